"""Pins of the oracle's CFL time step and rigid-body update against values
computed here from textbook closed forms, not from the oracle's own formulas.

* Time step (Sec. 3.1 takes a fraction of the largest stable step; the
  reading is dt = CFL / max_cells sum_d (|u_d| + c)/dx_d, also covering the
  body speed sum_d |v_r,d|/dx_d): uniform single-material states, where the
  sound speed has the closed form c^2 = gamma (p + p_inf)/rho of the ideal
  and stiffened gases, in 1-D, 2-D and 3-D with dx_d all different, signed
  velocities in every direction, and a case where the body speed dominates;
  and a random state whose maximum the test finds by brute force.
* Body motion (a dynamic body driven by the pressure force, not in the
  paper, which imposes v_r): symplectic Euler v^{n+1} = v^n + dt F^n/m,
  x^{n+1} = x^n + dt v^{n+1}, with F^n the force of the step-start seeded
  state; the first F is known in closed form for a planar body face with a
  pressure that varies only along the face (so that the seeding copies it
  unchanged).  CPU only."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import Oracle


def gas_c(m, rho, p):
    """Textbook sound speed of an ideal (p_inf = 0) or stiffened gas."""
    return math.sqrt(m["gamma"] * (p + m.get("pinf", 0.0)) / rho)


def uniform(dim, n, lo, hi, mat, rho, u, p, r=0.0):
    o = Oracle(dim, n, lo, hi, [mat])
    L = W.layout(dim, 1, False)
    w = np.zeros((L["nvar"], int(np.prod(n))))
    w[L["irho"]] = rho
    for d in range(dim):
        w[L["iu"] + d] = u[d]
    w[L["ip"]] = p
    w[L["ir"]] = r
    o.set_prim(w)
    return o


CASES = [
    # dim, n, hi (lo = 0), material, rho, u, p
    (1, (40,), (0.8,), W.AIR, 1.225, (-230.0,), 1e5),
    (2, (24, 10), (1.0, 0.3), W.AIR, 2.0, (310.0, -75.0), 3.5e5),
    (2, (12, 16), (0.5, 1.7), W.WATER, 1000.0, (-12.0, 40.0), 1e5),
    (3, (6, 8, 5), (0.6, 1.2, 0.25), W.AIR, 0.9, (50.0, -120.0, 260.0), 8e4),
    (3, (5, 4, 6), (0.1, 0.3, 0.2), W.WATER, 1020.0, (3.0, -4.0, 7.5), 2e6),
]


@pytest.mark.parametrize("dim,n,hi,mat,rho,u,p", CASES)
@pytest.mark.parametrize("cfl", [0.8, 0.3])
def test_dt_uniform_state_closed_form(dim, n, hi, mat, rho, u, p, cfl):
    lo = (0.0,) * dim
    o = uniform(dim, n, lo, hi, mat, rho, u, p)
    c = gas_c(mat, rho, p)
    dx = [hi[d] / n[d] for d in range(dim)]
    expect = cfl / sum((abs(u[d]) + c) / dx[d] for d in range(dim))
    got = o.compute_dt(cfl)
    assert got == pytest.approx(expect, rel=1e-12)
    # the three plausible slips all move it by far more than that
    assert abs(cfl / max((abs(u[d]) + c) / dx[d] for d in range(dim)) - got) > 1e-3 * got or dim == 1
    assert abs(cfl / sum(c / dx[d] for d in range(dim)) - got) > 1e-3 * got


def test_dt_body_speed_dominates():
    """Quiescent air (sum_d c/dx_d = 2c/h) with a body moving at 1000 m/s in
    x and 300 in y: sum_d |v_r,d|/dx_d = 1300/h is the larger one."""
    n, h = 16, 1.0 / 16
    o = uniform(2, (n, n), (0.0, 0.0), (1.0, 1.0), W.AIR, 1.225, (0.0, 0.0), 1e5)
    c = gas_c(W.AIR, 1.225, 1e5)
    assert 2 * c < 1300.0
    o.set_body(v=(1000.0, -300.0, 0.0))
    assert o.compute_dt(0.8) == pytest.approx(0.8 * h / 1300.0, rel=1e-13)
    # a slower body leaves the gas term in charge
    o.set_body(v=(200.0, 100.0, 0.0))
    assert o.compute_dt(0.8) == pytest.approx(0.8 * h / (2 * c), rel=1e-12)


def test_dt_random_state_brute_force_maximum():
    """Random smooth + noisy ideal-gas state: the oracle's dt equals CFL over
    the largest per-cell sum, found here cell by cell with the gas's closed-form
    sound speed (and the cell it comes from is not the one of largest |u| or
    largest c alone)."""
    nx, ny = 20, 14
    hx, hy = 1.0 / nx, 0.6 / ny
    rng = np.random.default_rng(77)
    o = Oracle(2, (nx, ny), (0.0, 0.0), (1.0, 0.6), [W.AIR])
    w = np.zeros((5, nx * ny))
    w[0] = 1.0 + 0.8 * rng.random(nx * ny)
    w[1] = 400.0 * (rng.random(nx * ny) - 0.5)
    w[2] = 400.0 * (rng.random(nx * ny) - 0.5)
    w[3] = 1e5 * (1.0 + 2.0 * rng.random(nx * ny))
    o.set_prim(w)
    c = np.sqrt(1.4 * w[3] / w[0])
    per_cell = (np.abs(w[1]) + c) / hx + (np.abs(w[2]) + c) / hy
    assert o.compute_dt(0.8) == pytest.approx(0.8 / per_cell.max(), rel=1e-12)


def planar_body(n=32, m=2.0):
    """Body filling x > 0.7 (tanh profile in x only), air at rest at 1e5 Pa
    plus a pressure gradient along y (parallel to the body face)."""
    o = Oracle(2, (n, n), (0.0, 0.0), (1.0, 1.0), [W.AIR])
    X, Y, _ = W.cell_centres((n, n), (0.0, 0.0), (1.0, 1.0))
    w = np.zeros((5, n * n))
    w[0] = 1.225
    w[3] = 1e5 + 4e4 * Y
    w[4] = W.rigid_profile(0.7 - X, 1.0 / n)
    o.set_prim(w)
    o.set_body(v=(0.0, 0.0, 0.0), x=(0.7, 0.5, 0.0), mass=m, dynamic=True)
    return o, w


def test_first_force_closed_form():
    """With r = r(x) and p = p(y), the seeding copies p unchanged (the probe
    moves along x only) and F = sum p grad(r) dV telescopes row by row: with
    central differences and clamped end cells (r_{-1} = r_0, r_N = r_{N-1}),
    sum_i (r_{i+1} - r_{i-1})/2h over a row is (r_{N-1} - r_0)/h; F_y = 0."""
    n = 32
    o, w = planar_body(n)
    h = 1.0 / n
    r = w[4].reshape(n, n)[0]
    p = w[3].reshape(n, n)[:, 0]
    tele = (r[-1] - r[0]) / h
    expect_x = np.sum(p * tele * h * h)
    o.step(o.compute_dt(0.5))
    F, _, _ = o.body()
    assert F[0] == pytest.approx(expect_x, rel=1e-10)
    assert abs(F[1]) < 1e-9 * abs(expect_x)


def test_body_update_is_symplectic_euler():
    """Each step: v^{n+1} = v^n + dt F^n/m, then x^{n+1} = x^n + dt v^{n+1}
    (the new velocity), with F^n the force the step reports.  An explicit
    Euler position update (x^n + dt v^n) or a force taken after the stage
    update would differ by far more than the tolerance."""
    m = 2.0
    o, _ = planar_body(32, m)
    _, v, x = o.body()
    assert np.all(v == 0.0)
    dts, F_, V, X = [], [], [v.copy()], [x.copy()]
    for _ in range(6):
        dt = o.compute_dt(0.5)
        o.step(dt)
        F, v, x = o.body()
        dts.append(dt)
        F_.append(F.copy())
        V.append(v.copy())
        X.append(x.copy())
    explicit_gap = 0.0
    for k, dt in enumerate(dts):
        vk = V[k] + dt * F_[k] / m
        np.testing.assert_allclose(V[k + 1], vk, rtol=1e-14, atol=1e-14 * np.abs(vk).max())
        xk = X[k] + dt * V[k + 1]
        np.testing.assert_allclose(X[k + 1], xk, rtol=0, atol=1e-15)
        explicit_gap = max(explicit_gap, float(np.abs(X[k + 1] - (X[k] + dt * V[k])).max()))
    # the symplectic and explicit updates are told apart by the test
    assert explicit_gap > 1e-9
    # the force changes from step to step (the body moves): F^n is per step
    assert abs(F_[-1][0] - F_[0][0]) > 0.0


def test_static_body_does_not_move():
    o, _ = planar_body(32)
    o.set_body(v=(0.0, 0.0, 0.0), x=(0.7, 0.5, 0.0), mass=2.0, dynamic=False)
    for _ in range(3):
        o.step(o.compute_dt(0.5))
    F, v, x = o.body()
    assert np.all(v == 0.0) and x[0] == 0.7 and x[1] == 0.5
    assert F[0] > 0.0
