"""Pins of the reflective wall boundary in the oracle: a wall is the mirror
plane of the doubled domain (the halo holds the mirror image of the interior,
velocity and stretch tensor reflected), and a shock running into a wall
reflects with the Rankine-Hugoniot plateau.  CPU only."""
import numpy as np
import pytest

import workloads as W
from oracle import Oracle
from test_oracle_riemann import rh_reflected, run_to


def mirror(prim, L, dim, n, d, nv_map):
    """The mirror image of a primitive field in direction d (reversed order
    along d; u_d and the stretch components with exactly one index d negated)."""
    shp = (prim.shape[0],) + tuple(reversed(n))          # [var, (z), (y), x]
    a = prim.reshape(shp)
    axis = 1 + (dim - 1 - d)
    m = np.flip(a, axis=axis).copy()
    m[L["iu"] + d] *= -1.0
    for c, (p, q) in enumerate(nv_map):
        if (p == d) != (q == d):
            m[L["iv"] + c] *= -1.0
    return m


VMAP = {1: [(0, 0), (1, 1), (2, 2)], 2: [(0, 0), (0, 1), (1, 0), (1, 1), (2, 2)]}


def doubled(case):
    """A random state on the half domain with a wall on one side, and the
    doubled domain holding it and its mirror image."""
    dim = 1 if case.startswith("1d") else 2
    solid = "solid" in case
    nmat = 2 if ("two_fluid" in case or dim == 2) else 1
    side = 0 if "low" in case else 1
    d = 1 if case.endswith("_y") else 0
    n = (64,) if dim == 1 else (40, 24)
    wl = W.random_state(dim, n, nmat, solid, seed=31, amp=0.02 if solid else 0.1, body=(dim == 2))
    L = W.layout(dim, nmat, solid)
    half = wl.prim.reshape((wl.nvar,) + tuple(reversed(n)))
    m = mirror(wl.prim, L, dim, n, d, VMAP[dim] if solid else [])
    axis = 1 + (dim - 1 - d)
    full = np.concatenate([m, half] if side == 0 else [half, m], axis=axis)
    n_full = list(n)
    n_full[d] *= 2
    lo_full, hi_full = list(wl.lo), list(wl.hi)
    ext = wl.hi[d] - wl.lo[d]
    if side == 0:
        lo_full[d] -= ext
    else:
        hi_full[d] += ext
    walls = [0] * 6
    walls[2 * d + side] = 1
    a = Oracle(dim, n, wl.lo, wl.hi, wl.materials, solid)
    a.set_walls(walls)
    a.set_prim(wl.prim)
    b = Oracle(dim, n_full, lo_full, hi_full, wl.materials, solid)
    b.set_prim(full.reshape(wl.nvar, -1))
    sl = [slice(None)] * full.ndim
    sl[axis] = slice(n[d], None) if side == 0 else slice(0, n[d])

    def half_of(x):
        return x.reshape(full.shape)[tuple(sl)].reshape(wl.nvar, -1)
    return a, b, half_of, wl


def rel(x, ref):
    return np.abs(x - ref).sum(axis=1) / (np.abs(ref).sum(axis=1) + 1e-300)


CASES = ["1d_two_fluid_low", "1d_solid_high", "2d_solid_low_y", "2d_solid_high_x", "2d_two_fluid_high_x",
         "2d_two_fluid_low_y"]


@pytest.mark.parametrize("case", CASES)
def test_wall_operator_equals_mirror_plane(case):
    """D(U) next to a wall equals D of the doubled domain holding U and its
    mirror image (velocity and stretch tensor reflected), to rounding."""
    a, b, half_of, wl = doubled(case)
    err = rel(a.compute_D(), half_of(b.compute_D()))
    assert np.all(err < 1e-13), err


@pytest.mark.parametrize("case", [c for c in CASES if "solid" not in c])
def test_wall_run_equals_mirror_plane_of_doubled_domain(case):
    """25 steps: the fluid state next to a wall stays the half of the doubled
    domain's state.  (With a solid, the face value of the shear stretch is
    upwinded by S*, which is exactly 0 at a wall but only ~1e-16 at the
    doubled domain's mirror plane once rounding has broken the symmetry, so
    only the operator is compared there.)"""
    a, b, half_of, wl = doubled(case)
    for _ in range(25):
        dt = b.compute_dt(0.6)
        assert a.compute_dt(0.6) == pytest.approx(dt, rel=1e-14)
        a.step(dt)
        b.step(dt)
    err = rel(a.cons(), half_of(b.cons()))
    assert np.all(err < 1e-12), err


def test_shock_reflects_from_a_wall():
    """A Mach 2 shock in air running into a wall at x = 1: the plateau behind
    the reflected shock matches rho5, p5 and u = 0 within 1 %."""
    n = 400
    X = (np.arange(n) + 0.5) / n
    rho2, u2, p2 = W.ideal_shock_state(2.0, 1.4, 1.225, 1e5)
    w = np.zeros((4, n))
    post = X < 0.6
    w[0] = np.where(post, rho2, 1.225)
    w[1] = np.where(post, u2, 0.0)
    w[2] = np.where(post, p2, 1e5)
    o = Oracle(1, (n,), (0.0,), (1.0,), [W.AIR])
    o.set_walls([0, 1])
    o.set_prim(w)
    s = rh_reflected(2.0)
    # the incident shock reaches the wall after 0.4/vs1, then the reflected shock runs back
    vs1 = u2 * rho2 / (rho2 - 1.225)
    t = 0.4 / vs1 + 0.15 / s["vs"]
    run_to(o, t, cfl=0.8)
    wp = o.prim()
    plateau = (X > 0.9) & (X < 0.97)
    assert np.mean(wp[0, plateau]) == pytest.approx(s["rho5"], rel=0.01)
    assert np.mean(wp[2, plateau]) == pytest.approx(s["p5"], rel=0.01)
    assert np.max(np.abs(wp[1, plateau])) < 0.01 * u2
