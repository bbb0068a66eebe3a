"""Pins of the oracle's Johnson-Cook flow stress (Table 2 constants of
copper; the law, reference temperature 298 K and reference rate 1/s are
readings) in the plastic update.  The von Mises stress after a return is
measured here from the returned stretch tensor with scipy's matrix
logarithm, independently of the oracle's eigen-solver:

* with c2 = c3 = 0 and no thermal softening the return is the perfectly
  plastic one at sigma_Y = c1 (bit for bit);
* the hardening curve at tabulated plastic strains, and along a sequence of
  isochoric uniaxial compressions whose plastic strain the history plane
  accumulates;
* the strain-rate factor 1 + c3 ln(rate) at the rate of the predictor return;
* thermal softening: half-way to melting, and at the melting temperature
  (no deviatoric stress left).  CPU only."""
import math

import numpy as np
import pytest
import scipy.linalg as sla

import workloads as W
from oracle import Oracle

CU = W.COPPER
T0 = 298.0


def cell(mat):
    """A 2-D one-cell copper grid with the plastic-strain plane:
    primitives rho, u, v, p, Vxx, Vxy, Vyx, Vyy, Vzz, r, eps."""
    return Oracle(2, (1, 1), (0.0, 0.0), (1.0, 1.0), [mat], solid=2)


def prim(A, eps=0.0, p=1e5, rho=8960.0):
    return [rho, 0.0, 0.0, p, A[0, 0], A[0, 1], A[1, 0], A[1, 1], A[2, 2], 0.0, eps]


def stretch(q):
    return np.array([[q[4], q[5], 0.0], [q[6], q[7], 0.0], [0.0, 0.0, q[8]]])


def von_mises(V, G):
    H = sla.logm(V).real
    Hd = H - np.trace(H) / 3.0 * np.eye(3)
    return math.sqrt(1.5) * 2.0 * G * np.linalg.norm(Hd), np.linalg.norm(Hd)


def sheared(s=0.03):
    """A symmetric, unimodular stretch far beyond yield."""
    return sla.expm(np.array([[s, 0.3 * s, 0.0], [0.3 * s, -s, 0.0], [0.0, 0.0, 0.0]]))


NO_RATE_NO_HEAT = dict(CU, jc_c3=0.0, jc_m=60.0)   # T* ~ 1e-5 -> T*^60 = 0


def test_reduces_to_perfect_plasticity_at_c1():
    jc = dict(NO_RATE_NO_HEAT, jc_c2=0.0)
    pp = {k: v for k, v in CU.items() if not k.startswith("jc_")}
    pp["sigY"] = CU["jc_c1"]
    a, b = cell(jc), cell(pp)
    q = a.prim_to_cons(prim(sheared()))
    np.testing.assert_array_equal(a.plastic_cons(q, 1e-8)[:10], b.plastic_cons(q, 1e-8)[:10])


@pytest.mark.parametrize("eps,expect", [
    (0.0, 0.09e9),
    (0.5, 0.09e9 + 0.292e9 * 0.5 ** 0.31),
    (1.0, 0.382e9),
    (2.0, 0.09e9 + 0.292e9 * 2.0 ** 0.31),
])
def test_hardening_at_tabulated_strains(eps, expect):
    o = cell(NO_RATE_NO_HEAT)
    q = o.prim_to_cons(prim(sheared(), eps=eps))
    q2 = o.plastic_cons(q, 1e-8)
    G = o.closure(q2)["G"]
    svm, _ = von_mises(stretch(q2), G)
    assert svm == pytest.approx(expect, rel=1e-9)
    # the plastic strain the return removed went into the history plane
    assert q2[10] > q[10]


def test_uniaxial_hardening_curve():
    """Forty isochoric compressions of 0.2 % along x, each followed by the
    return: past yield, the von Mises stress after each return is
    c1 + c2 eps^n at the plastic strain the cell had before it."""
    o = cell(NO_RATE_NO_HEAT)
    q = o.prim_to_cons(prim(np.eye(3)))
    d = 0.002
    F = np.diag([1.0 - d, (1.0 - d) ** -0.5, (1.0 - d) ** -0.5])
    yielded = 0
    for k in range(40):
        V = F @ stretch(q)
        q = q.copy()
        q[4], q[5], q[6], q[7], q[8] = V[0, 0], V[0, 1], V[1, 0], V[1, 1], V[2, 2]
        eps_before = q[10] / q[0]
        q = o.plastic_cons(q, 1e-8)
        svm, _ = von_mises(stretch(q), o.closure(q)["G"])
        if q[10] / q[0] > eps_before:
            yielded += 1
            assert svm == pytest.approx(0.09e9 + 0.292e9 * eps_before ** 0.31, rel=1e-8)
        else:
            assert svm < 0.09e9 * (1 + 1e-9)
    assert yielded > 20
    assert q[10] / q[0] > 0.02


def test_strain_rate_factor():
    """c3 > 0: the rate is the plastic strain a return at the rate-free yield
    stress would remove, over dt; the return then uses (1 + c3 ln rate)."""
    mat = dict(CU, jc_m=60.0)
    o = cell(mat)
    eps0, dt = 0.3, 2e-9
    q = o.prim_to_cons(prim(sheared(), eps=eps0))
    G = o.closure(q)["G"]
    svm_trial, nd = von_mises(stretch(q), G)
    sy0 = 0.09e9 + 0.292e9 * eps0 ** 0.31
    rate = math.sqrt(2.0 / 3.0) * (1.0 - sy0 / svm_trial) * nd / dt
    assert rate > 1e6
    q2 = o.plastic_cons(q, dt)
    svm, _ = von_mises(stretch(q2), G)
    assert svm == pytest.approx(sy0 * (1.0 + 0.025 * math.log(rate)), rel=1e-8)
    # without a step (dt = 0) there is no rate term
    svm0, _ = von_mises(stretch(o.plastic_cons(q, 0.0)), G)
    assert svm0 == pytest.approx(sy0, rel=1e-8)


def test_thermal_softening():
    """T from the thermal energy (p - p_ref)/(rho Gamma C_V): half-way to
    melting the yield stress is c1 (1 - 0.5^m); at melting it vanishes."""
    mat = dict(CU, jc_c3=0.0)
    o = cell(mat)
    A = sheared()
    J2 = von_mises(A, 1.0)[1] ** 2
    pref = o.material_ref(0, 8960.0, J2)["pref"]
    for frac, expect in ((0.5, 0.09e9 * (1.0 - 0.5 ** 1.09)), (1.0, 0.0)):
        p = pref + frac * (1358.0 - T0) * 8960.0 * 2.0 * 385.0
        q = o.prim_to_cons(prim(A, p=p))
        q2 = o.plastic_cons(q, 1e-8)
        svm, _ = von_mises(stretch(q2), o.closure(q2)["G"])
        if expect == 0.0:
            assert svm < 1e-6 * 0.09e9
        else:
            assert svm == pytest.approx(expect, rel=1e-8)
