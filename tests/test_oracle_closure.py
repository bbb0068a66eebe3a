"""Pins of the oracle's thermodynamics (Sec. 2.1.2-2.2): closed forms,
thermodynamic identities checked by finite differences, and the mixture
rules' reductions.  CPU only."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import Oracle

AL = W.ALUMINIUM


def single(mat, dim=1, solid=False):
    return Oracle(dim, (4,) * dim, (0.0,) * dim, (1.0,) * dim, [mat], solid=solid)


def test_ideal_gas_closed_form():
    o = single(W.AIR)
    rho, u, p = 1.7, 123.0, 2.3e5
    q = o.prim_to_cons([rho, u, p, 0.0])
    assert q[0] == pytest.approx(rho, rel=1e-15)
    assert q[2] == pytest.approx(p / 0.4 + 0.5 * rho * u * u, rel=1e-14)   # p = (gamma-1) rho e
    cl = o.closure(q)
    assert cl["p"] == pytest.approx(p, rel=1e-13)
    assert cl["c"] == pytest.approx(math.sqrt(1.4 * p / rho), rel=1e-13)


def test_stiffened_gas_closed_form():
    o = single(W.WATER)
    rho, p = 1000.0, 1.0e5
    q = o.prim_to_cons([rho, 0.0, p, 0.0])
    # p = (gamma-1) rho e - gamma p_inf  =>  rho e = (p + gamma p_inf)/(gamma-1)
    assert q[2] == pytest.approx((p + 4.4 * 6e8) / 3.4, rel=1e-14)
    cl = o.closure(q)
    assert cl["p"] == pytest.approx(p, rel=1e-9)
    assert cl["c"] == pytest.approx(math.sqrt(4.4 * (p + 6e8) / rho), rel=1e-13)


@pytest.mark.parametrize("x", [0.8, 1.0, 1.17])
@pytest.mark.parametrize("J2", [0.0, 3e-4])
def test_romenskii_reference_curves(x, J2):
    o = single(AL, solid=True)
    rho = AL["rho0"] * x
    r = o.material_ref(0, rho, J2)
    h = rho * 1e-6
    rp, rm = o.material_ref(0, rho + h, J2), o.material_ref(0, rho - h, J2)
    # p_ref = rho^2 de_ref/drho  (eq:Romenskii)
    dedr = (rp["eref"] - rm["eref"]) / (2 * h)
    tol = 1e-8 * AL["K0"]   # FD truncation ~ K0 (h/rho)^2
    assert r["pref"] == pytest.approx(rho * rho * dedr, rel=2e-6, abs=tol)
    assert r["deref"] == pytest.approx(dedr, rel=2e-6, abs=tol / rho ** 2)
    dpdr = (rp["pref"] - rm["pref"]) / (2 * h)
    assert r["dpref"] == pytest.approx(dpdr, rel=2e-6)
    assert r["G"] == pytest.approx(AL["G0"] * x ** (AL["beta"] + 1.0), rel=1e-14)
    assert r["Gamma"] == AL["Gamma0"]


def test_romenskii_bulk_modulus_at_reference_density():
    """rho dp_ref/drho = K0 at rho = rho0 (either form of the cold term)."""
    o = single(AL, solid=True)
    r = o.material_ref(0, AL["rho0"], 0.0)
    assert r["pref"] == 0.0 and r["eref"] == 0.0
    assert AL["rho0"] * r["dpref"] == pytest.approx(AL["K0"], rel=1e-14)


@pytest.mark.parametrize("x,p", [(1.0, 1e5), (1.1, 2e9), (0.93, -1e8)])
def test_romenskii_sound_speed_is_isentropic_derivative(x, p):
    """a^2 = (dp/drho)_S (Sec. 2.1.2): the closure's c^2 - 4/3 G/rho equals a
    finite-difference derivative of p along de = p/rho^2 drho."""
    o = single(AL, solid=True)
    rho = AL["rho0"] * x
    q0 = o.prim_to_cons([rho, 0.0, p, 1.0, 1.0, 1.0, 0.0])
    e0 = q0[2] / rho
    h = rho * 1e-6
    ps = []
    for s in (+1, -1):
        r1 = rho + s * h
        # second-order isentrope step: de = p/rho^2 drho, p evaluated midway
        pm = p
        for _ in range(3):
            e1 = e0 + s * h * pm / ((rho + 0.5 * s * h) ** 2)
            p1 = o.closure([r1, 0.0, r1 * e1, 1.0, 1.0, 1.0, 0.0])["p"]
            pm = 0.5 * (p + p1)
        ps.append(p1)
    a2_fd = (ps[0] - ps[1]) / (2 * h)
    cl = o.closure(q0)
    G = o.material_ref(0, rho, 0.0)["G"]
    a2 = cl["c"] ** 2 - 4.0 / 3.0 * G / rho
    assert a2 == pytest.approx(a2_fd, rel=1e-6)


@pytest.mark.parametrize("phi,tol", [(0.3, 1e-13), (1e-5, 1e-13), (0.999, 1e-13), (1e-8, 1e-7)])
def test_mixture_of_identical_materials_reduces_to_single(phi, tol):
    """Two copies of one gas at any volume fraction give the single-material
    pressure and sound speed (mixture rules, Sec. 2.2).  Below a volume
    fraction of 1e-6 a material is absent and takes its reference density, so
    the sound speed then agrees only to O(phi)."""
    one = single(W.AIR)
    two = Oracle(1, (4,), (0.0,), (1.0,), [W.AIR, W.AIR])
    rho, u, p = 1.3, 55.0, 3.3e5
    q1 = one.prim_to_cons([rho, u, p, 0.0])
    q2 = two.prim_to_cons([phi, rho, rho, u, p, 0.0])
    assert q2[1] + q2[2] == pytest.approx(q1[0], rel=1e-15)
    assert q2[4] == pytest.approx(q1[2], rel=1e-14)
    c1, c2 = one.closure(q1), two.closure(q2)
    assert c2["p"] == pytest.approx(c1["p"], rel=1e-13)
    assert c2["c"] == pytest.approx(c1["c"], rel=tol)


def test_absent_material_takes_reference_density():
    """A material below phi = 1e-6 (or with a slightly negative transported
    phi) is evaluated at its reference density, so an inconsistent trace of a
    stiff solid cannot set the pressure of the cell it sits in."""
    two = Oracle(1, (4,), (0.0,), (1.0,), [AL, W.AIR], solid=True)
    for phi_al, ar_al in ((-2.7e-6, 0.0118), (5e-7, 0.01), (0.0, 1e-5)):
        w_air = two.prim_to_cons([1e-8, 2700.0, 1.2, 0.0, 1e5, 1.0, 1.0, 1.0, 0.0])
        q = w_air.copy()
        q[0], q[1] = phi_al, ar_al
        q[4] = q[4] + 0.0
        cl = two.closure(q)
        assert cl["p"] == pytest.approx(1e5, rel=1e-3), (phi_al, cl)
        assert two.cons_to_prim(q)[1] == AL["rho0"]


def test_mixture_pure_limits():
    """phi -> 1 of one material recovers that material's closure."""
    two = Oracle(1, (4,), (0.0,), (1.0,), [W.AIR, W.WATER])
    w_air = two.closure(two.prim_to_cons([1.0, 1.2, 1000.0, 0.0, 2e5, 0.0]))
    assert w_air["p"] == pytest.approx(2e5, rel=1e-12)
    assert w_air["c"] == pytest.approx(math.sqrt(1.4 * 2e5 / 1.2), rel=1e-12)
    w_wat = two.closure(two.prim_to_cons([0.0, 1.2, 1000.0, 0.0, 2e5, 0.0]))
    assert w_wat["p"] == pytest.approx(2e5, rel=1e-8)
    assert w_wat["c"] == pytest.approx(math.sqrt(4.4 * (2e5 + 6e8) / 1000.0), rel=1e-12)


def test_mixture_pressure_is_gamma_weighted_component_pressure():
    """Sec. 2.2: the mixture pressure equals sum(phi_l p_l/Gamma_l)/sum(phi_l/Gamma_l)
    when each component is evaluated at its own energy; with a common p the
    mixture returns it, and the mixture shear modulus follows the same weights."""
    two = Oracle(2, (4, 4), (0.0, 0.0), (1.0, 1.0), [AL, W.AIR], solid=True)
    phi, p = 0.37, 4.0e7
    w = [phi, 2750.0, 1.5, 10.0, -3.0, p, 1.01, 0.002, -0.001, 0.99, 1.0 / (1.01 * 0.99 + 0.002 * 0.001), 0.0]
    q = two.prim_to_cons(w)
    cl = two.closure(q)
    assert cl["p"] == pytest.approx(p, rel=1e-12)
    rAl = two.material_ref(0, 2750.0, cl["J2"])
    G = (phi * rAl["G"] / AL["Gamma0"]) / (phi / AL["Gamma0"] + (1 - phi) / 0.4)
    assert cl["G"] == pytest.approx(G, rel=1e-13)


def test_cons_prim_roundtrip_two_material_solid():
    two = Oracle(2, (4, 4), (0.0, 0.0), (1.0, 1.0), [AL, W.AIR], solid=True)
    w = np.array([0.6, 2690.0, 1.1, 300.0, -20.0, 3e8, 1.02, 0.01, -0.02, 0.97, 1.0, 0.2])
    w2 = two.cons_to_prim(two.prim_to_cons(w))
    np.testing.assert_allclose(w2, w, rtol=1e-10)
