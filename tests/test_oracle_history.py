"""Pins of the equivalent-plastic-strain history planes (phi rho eps)_l of
Sec. 2.1.1 in the oracle: a constant eps is carried unchanged, the planes are
conserved, and the radial return adds the closed-form increment
sqrt(2/3) (1 - s) |d| to materials with a yield stress.  CPU only."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import Oracle


def test_layout_and_zero_history_changes_nothing_else():
    wl = W.impact_2d(64)
    wh = W.with_history(wl)
    assert wh.nvar == wl.nvar + 2
    a, b = Oracle.from_workload(wl), Oracle.from_workload(wh)
    for _ in range(3):
        dt = a.compute_dt(wl.cfl)
        assert b.compute_dt(wl.cfl) == dt
        a.step(dt)
        b.step(dt)
    np.testing.assert_array_equal(b.cons()[: wl.nvar], a.cons())


@pytest.mark.parametrize("dim,n", [(1, (200,)), (2, (40, 36))])
def test_constant_eps_is_carried_unchanged_below_yield(dim, n):
    """Below yield the planes are pure advection: eps = (phi rho eps)/(phi rho)
    stays exactly constant when it starts constant (the history flux is eps
    times the partial-density flux in every wave region)."""
    wl = W.random_state(dim, n, 2, True, seed=51, amp=0.002, body=False)
    wh = W.with_history(wl)
    L = W.layout(dim, 2, True, True)
    # stretch tensor near the identity: elastic everywhere (random_state's 1 % noise would yield)
    rng = np.random.default_rng(5)
    ident = [1.0, 1.0, 1.0] if dim == 1 else [1.0, 0.0, 0.0, 1.0, 1.0]
    for c, v in enumerate(ident):
        wh.prim[L["iv"] + c] = v + 1e-4 * rng.standard_normal(wh.ncell)
    # a uniform flow at uniform pressure carries the density and fraction variations
    for a in range(dim):
        wh.prim[L["iu"] + a] = 30.0 * (a + 1)
    wh.prim[L["ip"]] = 1e5
    wh.prim[L["ih"]] = 0.004
    wh.prim[L["ih"] + 1] = 0.0015
    o = Oracle.from_workload(wh)
    for _ in range(15):
        o.step(o.compute_dt(0.6))
    w = o.prim()
    assert np.all(np.isfinite(w))
    # no cell yields at this amplitude, so nothing is added
    np.testing.assert_allclose(w[L["ih"]], 0.004, rtol=1e-11)
    np.testing.assert_allclose(w[L["ih"] + 1], 0.0015, rtol=1e-10)


def test_history_planes_are_conserved_on_a_periodic_grid():
    """Random eps and velocities, stretch near the identity (elastic): the
    planes only move between cells."""
    wl = W.random_state(2, (32, 30), 2, True, seed=52, amp=0.002, periodic=(1, 1), body=False)
    wh = W.with_history(wl, seed=7, amp=0.01)
    L = W.layout(2, 2, True, True)
    rng = np.random.default_rng(6)
    for c, v in enumerate([1.0, 0.0, 0.0, 1.0, 1.0]):
        wh.prim[L["iv"] + c] = v + 1e-4 * rng.standard_normal(wh.ncell)
    o = Oracle.from_workload(wh)
    q0 = o.cons()[L["ih"]: L["ih"] + 2].sum(axis=1)
    for _ in range(10):
        o.step(o.compute_dt(0.6))
    q1 = o.cons()[L["ih"]: L["ih"] + 2].sum(axis=1)
    np.testing.assert_allclose(q1, q0, rtol=1e-12)


def test_radial_return_adds_the_closed_form_increment():
    """One 2-D aluminium cell stretched by V = diag(lam, 1/lam, 1): the
    deviatoric log-stretches are (ln lam, -ln lam, 0), |d| = sqrt(2) ln lam,
    sigma_vm = sqrt(3/2) 2 G |d|, s = sigma_Y / sigma_vm (mixture G and sigma_Y),
    and the return adds
    (phi rho)_l sqrt(2/3) (1 - s) |d| to the solid's plane only."""
    o = Oracle(2, (4, 4), (0.0, 0.0), (1.0, 1.0), [W.ALUMINIUM, W.AIR], solid=2)
    L = W.layout(2, 2, True, True)
    lam = 1.01
    w = np.zeros(L["nvar"])
    w[L["iphi"]] = 1.0 - 1e-8
    w[L["irho"]], w[L["irho"] + 1] = 2700.0, 1.225
    w[L["ip"]] = 1e5
    w[L["iv"]: L["iv"] + 5] = [lam, 0.0, 0.0, 1.0 / lam, 1.0]
    w[L["ih"]], w[L["ih"] + 1] = 0.002, 0.003
    q = o.prim_to_cons(w)
    cl = o.closure(q)          # mixture shear modulus and yield stress of the cell
    d = math.sqrt(2.0) * math.log(lam)
    svm = math.sqrt(1.5) * 2.0 * cl["G"] * d
    s = cl["sigY"] / svm
    assert s < 1.0
    qp = o.plastic_cons(q)
    ar = q[L["irho"]: L["irho"] + 2]
    deps = math.sqrt(2.0 / 3.0) * (1.0 - s) * d
    assert qp[L["ih"]] == pytest.approx(q[L["ih"]] + ar[0] * deps, rel=1e-12)
    assert qp[L["ih"] + 1] == q[L["ih"] + 1]          # the gas has no yield stress
    # below yield nothing changes
    w[L["iv"]: L["iv"] + 5] = [1.0001, 0.0, 0.0, 1.0 / 1.0001, 1.0]
    q2 = o.prim_to_cons(w)
    np.testing.assert_array_equal(o.plastic_cons(q2)[L["ih"]: L["ih"] + 2], q2[L["ih"]: L["ih"] + 2])


def test_impact_accumulates_plastic_strain_in_the_block_only():
    wh = W.with_history(W.impact_2d(96))
    L = W.layout(2, 2, True, True)
    o = Oracle.from_workload(wh)
    for _ in range(40):
        o.step(o.compute_dt(wh.cfl))
    w = o.prim()
    eps_al, eps_air = w[L["ih"]], w[L["ih"] + 1]
    assert eps_al.max() > 1e-3                         # the block yields where it hits the wedge
    assert np.all(eps_al >= -1e-14)
    assert np.abs(eps_air).max() == 0.0               # air has no yield stress and starts at 0
