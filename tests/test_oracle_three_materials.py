"""Pins of the N-material form with three materials in the oracle: a material
split into two identical halves reproduces the two-material run, uniform
pressure and velocity survive three-material interfaces, and every partial
density is conserved.  CPU only."""
import numpy as np
import pytest

import workloads as W
from oracle import Oracle


@pytest.mark.parametrize("solid", [False, True])
@pytest.mark.parametrize("thinc", [True, False])
def test_identical_halves_reproduce_the_two_material_run(solid, thinc):
    """Materials (A, B) with fractions (phi_A, phi_B) against (A, B, B) with
    (phi_A, phi_B/2, phi_B/2): the mixture rules, the van Leer and THINC face
    values and the HLLC fluxes are all homogeneous of degree one in the
    split, so the sums of the split planes follow the two-material run."""
    dim, n = 2, (36, 30)
    wl2 = W.random_state(dim, n, 2, solid, seed=71, amp=0.02 if solid else 0.1)
    L2 = W.layout(dim, 2, solid)
    L3 = W.layout(dim, 3, solid)
    mats3 = wl2.materials + [wl2.materials[1]]
    p2 = wl2.prim.copy()
    # genuinely mixed cells everywhere (fractions in [0.15, 0.85]): the rule
    # for absent materials (fraction < 1e-6) is a switch that a split across
    # its threshold would see on one side only
    X, Y, _ = W.cell_centres(n, wl2.lo, wl2.hi)
    rng = np.random.default_rng(9)
    p2[L2["iphi"]] = 0.5 + 0.3 * np.sin(2 * np.pi * X) * np.cos(np.pi * Y) + 0.02 * rng.standard_normal(X.size)
    p3 = np.zeros((L3["nvar"], p2.shape[1]))
    phiA = p2[L2["iphi"]]
    p3[L3["iphi"]] = phiA
    p3[L3["iphi"] + 1] = 0.5 * (1.0 - phiA)
    p3[L3["irho"]] = p2[L2["irho"]]
    p3[L3["irho"] + 1] = p2[L2["irho"] + 1]
    p3[L3["irho"] + 2] = p2[L2["irho"] + 1]
    p3[L3["iu"]:] = p2[L2["iu"]:]
    o2 = Oracle(dim, n, wl2.lo, wl2.hi, wl2.materials, solid)
    o3 = Oracle(dim, n, wl2.lo, wl2.hi, mats3, solid)
    for o, p in ((o2, p2), (o3, p3)):
        o.set_options(use_thinc=thinc)
        o.set_prim(p)
    for _ in range(8):
        dt = o2.compute_dt(0.6)
        assert o3.compute_dt(0.6) == pytest.approx(dt, rel=1e-13)
        o2.step(dt)
        o3.step(dt)
    q2, q3 = o2.cons(), o3.cons()
    merged = np.concatenate([q3[L3["iphi"]: L3["iphi"] + 1],
                             q3[L3["irho"]: L3["irho"] + 1],
                             q3[L3["irho"] + 1: L3["irho"] + 2] + q3[L3["irho"] + 2: L3["irho"] + 3],
                             q3[L3["iu"]:]])
    scale = np.abs(q2).sum(axis=1) + 1e-300
    err = np.abs(merged - q2).sum(axis=1) / scale
    assert np.all(err < 1e-12), err
    # the two halves stay equal
    np.testing.assert_allclose(q3[L3["irho"] + 1], q3[L3["irho"] + 2], rtol=1e-13)


def test_uniform_pressure_and_velocity_across_three_materials():
    """Abgrall's condition with water, helium and air: p and u uniform at
    the start stay uniform (1-D, transmissive)."""
    n = 200
    X = (np.arange(n) + 0.5) / n
    L = W.layout(1, 3, False)
    w = np.zeros((L["nvar"], n))
    water = (X > 0.2) & (X < 0.45)
    helium = (X > 0.6) & (X < 0.8)
    w[L["iphi"]] = np.where(water, 1.0 - 2e-8, 1e-8)
    w[L["iphi"] + 1] = np.where(helium, 1.0 - 2e-8, 1e-8)
    w[L["irho"]] = 1000.0
    w[L["irho"] + 1] = 0.166
    w[L["irho"] + 2] = 1.225
    w[L["iu"]] = 50.0
    w[L["ip"]] = 1e5
    o = Oracle(1, (n,), (0.0,), (1.0,), [W.WATER, W.HELIUM, W.AIR])
    o.set_prim(w)
    for _ in range(30):
        o.step(o.compute_dt(0.5))
    wp = o.prim()
    np.testing.assert_allclose(wp[L["ip"]], 1e5, rtol=1e-7)
    np.testing.assert_allclose(wp[L["iu"]], 50.0, rtol=1e-7)


def test_three_material_partial_densities_conserved():
    wl = W.random_state(2, (32, 30), 3, False, seed=72, periodic=(1, 1), body=False)
    L = W.layout(2, 3, False)
    o = Oracle.from_workload(wl)
    m0 = o.cons()[L["irho"]: L["irho"] + 3].sum(axis=1)
    for _ in range(10):
        o.step(o.compute_dt(0.6))
    m1 = o.cons()[L["irho"]: L["irho"] + 3].sum(axis=1)
    np.testing.assert_allclose(m1, m0, rtol=1e-12)
