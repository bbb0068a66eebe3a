"""Pins of the two method variants: the Riemann-problem-based seeding of
Sec. 3.2 (step 5, second option) and the HLLC-LM flux option (named for the
cylinder test).  CPU only."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import Oracle
from test_oracle_riemann import rh_reflected, run_to


def test_hllc_lm_is_hllc_above_the_mach_limit():
    """phi = 1 when the larger normal Mach number is >= 0.1: the centred
    form then equals the HLLC flux."""
    o = Oracle(2, (4, 4), (0.0, 0.0), (1.0, 1.0), [W.AIR, W.AIR])
    # normal Mach numbers |u_d|/c above 0.1 in both sweep directions
    wL = np.array([0.7, 1.4, 1.3, 90.0, -80.0, 2e5, 0.0])
    wR = np.array([0.3, 1.1, 1.0, 60.0, 70.0, 1.3e5, 0.0])
    for d in (0, 1):
        o.set_variants(hllc_lm=False)
        F0, u0, _ = o.riemann(d, wL, wR)
        o.set_variants(hllc_lm=True)
        F1, u1, _ = o.riemann(d, wL, wR)
        np.testing.assert_allclose(F1, F0, rtol=1e-12, atol=1e-12 * np.abs(F0).max())
        np.testing.assert_allclose(u1, u0, rtol=1e-14)


def test_hllc_lm_consistent_and_less_dissipative_at_low_mach():
    o = Oracle(1, (4,), (0.0,), (1.0,), [W.AIR])
    o.set_variants(hllc_lm=True)
    w = np.array([1.2, 3.0, 1e5, 0.0])
    F, _, _ = o.riemann(0, w, w)
    q = o.prim_to_cons(w)
    np.testing.assert_allclose(F[:3], [q[1], q[1] * 3.0 + 1e5, (q[2] + 1e5) * 3.0], rtol=1e-13)
    # a pressure jump at rest: the low-Mach form damps the acoustic dissipation
    wL = np.array([1.2, 0.0, 1.001e5, 0.0])
    wR = np.array([1.2, 0.0, 1.0e5, 0.0])
    F1, _, _ = o.riemann(0, wL, wR)
    o.set_variants(hllc_lm=False)
    F0, _, _ = o.riemann(0, wL, wR)
    assert abs(F1[0]) < 0.1 * abs(F0[0])


def test_hllc_lm_run_stays_symmetric_and_close():
    wl = W.cylinder_2d(48)
    a = Oracle.from_workload(wl, hllc_lm=True)
    b = Oracle.from_workload(wl, hllc_lm=False)
    for _ in range(10):
        dt = b.compute_dt(0.8)
        a.step(dt)
        b.step(dt)
    wa = a.prim().reshape(5, 48, 48)
    assert np.max(np.abs(wa[0] - wa[0][::-1, :])) <= 1e-11 * wa[0].max()
    # the flux differs only in low-Mach regions: densities close to plain HLLC
    assert np.mean(np.abs(wa[0] - b.prim()[0].reshape(48, 48))) / np.mean(wa[0]) < 0.05


def normals(r, n, dx):
    """Outward normals -grad r/|grad r| by clamped central differences."""
    R = r.reshape(n, n)
    gx = (np.concatenate([R[:, 1:], R[:, -1:]], 1) - np.concatenate([R[:, :1], R[:, :-1]], 1)) / (2 * dx)
    gy = (np.concatenate([R[1:, :], R[-1:, :]], 0) - np.concatenate([R[:1, :], R[:-1, :]], 0)) / (2 * dx)
    g = np.hypot(gx, gy)
    return -gx / np.maximum(g, 1e-300), -gy / np.maximum(g, 1e-300)


@pytest.mark.parametrize("vbody", [(0.0, 0.0), (150.0, -60.0)])
def test_riemann_seeding_imposes_the_body_normal_velocity(vbody):
    """The star state of the symmetric problem (reflected | interpolated)
    moves at S* = v_r . n exactly, so every seeded cell gets u.n = v_r.n."""
    n = 40
    wl = W.random_state(2, (n, n), 1, False, seed=41, amp=0.1)
    o = Oracle.from_workload(wl, seed_variant=1)
    o.set_body(v=(vbody[0], vbody[1], 0.0))
    r = wl.prim[-1]
    before = o.cons()
    o.seed()
    after = o.cons()
    seeded = np.any(after != before, axis=0)
    assert seeded.sum() > 20
    w = o.prim()
    nx, ny = normals(r, n, 1.0 / n)
    un = w[1] * nx.ravel() + w[2] * ny.ravel()
    vn = vbody[0] * nx.ravel() + vbody[1] * ny.ravel()
    assert np.all(r[seeded] > 0.5)
    np.testing.assert_allclose(un[seeded], vn[seeded], rtol=0, atol=1e-9 * (400.0 + abs(vbody[0])))


def test_riemann_seeding_quiescent_and_comoving_unchanged():
    for u in ((0.0, 0.0), (120.0, -70.0)):
        nn = 32
        X, Y, _ = W.cell_centres((nn, nn), (0.0, 0.0), (1.0, 1.0))
        w = np.zeros((5, X.size))
        w[0], w[1], w[2], w[3] = 1.225, u[0], u[1], 1e5
        w[4] = W.rigid_profile(np.hypot(X - 0.45, Y - 0.55) - 0.2, 1.0 / nn)
        o = Oracle(2, (nn, nn), (0.0, 0.0), (1.0, 1.0), [W.AIR])
        o.set_variants(seed_variant=1)
        o.set_prim(w)
        o.set_body(v=(u[0], u[1], 0.0))
        for _ in range(5):
            o.step(o.compute_dt(0.5))
        wp = o.prim()
        np.testing.assert_allclose(wp[0], 1.225, rtol=1e-12)
        np.testing.assert_allclose(wp[3], 1e5, rtol=1e-11)
        np.testing.assert_allclose(wp[1], u[0], atol=1e-9 * 338)


def test_reflected_shock_with_riemann_seeding():
    wl = W.shock_reflection_1d(400)
    o = Oracle.from_workload(wl, seed_variant=1)
    s = rh_reflected(2.0)
    run_to(o, 8.874e-4, cfl=0.8)
    w = o.prim()
    x = (np.arange(400) + 0.5) / 400
    plateau = (x > 0.62) & (x < 0.68)
    assert np.mean(w[0, plateau]) == pytest.approx(s["rho5"], rel=0.01)
    assert np.mean(w[2, plateau]) == pytest.approx(s["p5"], rel=0.01)
