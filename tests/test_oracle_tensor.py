"""Pins of the oracle's stretch-tensor algebra: the symmetric eigen solver,
the Hencky strain dev(H) = ln V (Sec. 2.1.2), the left polar decomposition
and the plastic radial return, against scipy's matrix functions and the
invariants they must satisfy.  CPU only."""
import math

import numpy as np
import pytest
import scipy.linalg as sla

import oracle
import workloads as W
from oracle import Oracle

AL = W.ALUMINIUM


def rand_A(rng, amp=0.2):
    A = np.eye(3) + amp * rng.standard_normal((3, 3))
    if np.linalg.det(A) < 0:
        A[:, 0] *= -1
    return A


@pytest.mark.parametrize("seed", range(5))
def test_sym_eig3_reconstructs(seed):
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((3, 3))
    B = M @ M.T + 0.1 * np.eye(3)
    lam, Q = oracle.sym_eig3(B)
    np.testing.assert_allclose(Q @ np.diag(lam) @ Q.T, B, rtol=0, atol=1e-13 * np.abs(B).max())
    np.testing.assert_allclose(Q.T @ Q, np.eye(3), atol=1e-14)
    np.testing.assert_allclose(np.sort(lam), np.linalg.eigvalsh(B), rtol=1e-13)


@pytest.mark.parametrize("seed", range(5))
def test_polar_decomposition(seed):
    A = rand_A(np.random.default_rng(seed))
    V, R = oracle.polar(A)
    np.testing.assert_allclose(V, V.T, atol=1e-14)
    assert np.all(np.linalg.eigvalsh(V) > 0)
    np.testing.assert_allclose(V @ R, A, atol=1e-13)
    np.testing.assert_allclose(R.T @ R, np.eye(3), atol=1e-13)
    np.testing.assert_allclose(V, sla.sqrtm(A @ A.T).real, atol=1e-12)


@pytest.mark.parametrize("seed", range(5))
def test_hencky_strain_against_logm(seed):
    A = rand_A(np.random.default_rng(100 + seed))
    dH, J2 = oracle.vbar_log(A)
    V = sla.sqrtm(A @ A.T).real
    H = sla.logm(V).real
    Hdev = H - np.trace(H) / 3.0 * np.eye(3)
    np.testing.assert_allclose(dH, Hdev, atol=1e-12)
    assert abs(np.trace(dH)) < 1e-14
    assert J2 == pytest.approx(np.sum(Hdev * Hdev), rel=1e-12)


def test_hencky_strain_identity_and_pure_rotation():
    dH, J2 = oracle.vbar_log(np.eye(3))
    assert J2 == 0.0 and np.all(dH == 0.0)
    th = 0.3
    R = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1]])
    dH, J2 = oracle.vbar_log(R)
    assert J2 < 1e-28


def _solid2d():
    return Oracle(2, (4, 4), (0.0, 0.0), (1.0, 1.0), [AL, W.AIR], solid=True)


def _vm(V, G):
    H = sla.logm(V).real
    Hd = H - np.trace(H) / 3 * np.eye(3)
    return math.sqrt(1.5) * 2 * G * np.linalg.norm(Hd)


def test_radial_return_lands_on_yield_surface():
    """Perfect plasticity: after the return the von Mises stress of the new
    (symmetric, unimodular) V equals the mixture yield stress."""
    o = _solid2d()
    phi = 1.0 - 1e-8
    s = 0.02  # 2 % shear strain: well beyond yield (sigma_Y/G ~ 0.01)
    A = np.array([[1 + s, 0.01, 0], [-0.004, 1 - s, 0], [0, 0, 1.0]])
    w = [phi, 2700.0, 1.225, 0.0, 0.0, 1e5, A[0, 0], A[0, 1], A[1, 0], A[1, 1], A[2, 2], 0.0]
    q = o.prim_to_cons(w)
    q2 = o.plastic_cons(q)
    V = np.array([[q2[6], q2[7], 0], [q2[8], q2[9], 0], [0, 0, q2[10]]])
    np.testing.assert_allclose(V, V.T, atol=1e-15)
    assert np.linalg.det(V) == pytest.approx(1.0, abs=1e-14)
    cl = o.closure(q2)
    assert _vm(V, cl["G"]) == pytest.approx(cl["sigY"], rel=1e-10)
    assert cl["sigY"] == pytest.approx(
        (phi * AL["sigY"] / AL["Gamma0"]) / (phi / AL["Gamma0"] + (1 - phi) / 0.4), rel=1e-13)
    # energy, mass and momentum are untouched by the return
    np.testing.assert_array_equal(q2[:6], q[:6])
    assert q2[11] == q[11]


def test_radial_return_elastic_state_only_symmetrised():
    """Below yield only the rotation is removed: V is the polar stretch of A
    made unimodular."""
    o = _solid2d()
    th = 0.2
    Rz = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1.0]])
    U = np.diag([1.001, 1.0 / 1.001, 1.0])
    A = U @ Rz
    w = [1 - 1e-8, 2700.0, 1.225, 0.0, 0.0, 1e5, A[0, 0], A[0, 1], A[1, 0], A[1, 1], A[2, 2], 0.0]
    q2 = o.plastic_cons(o.prim_to_cons(w))
    V = np.array([[q2[6], q2[7], 0], [q2[8], q2[9], 0], [0, 0, q2[10]]])
    np.testing.assert_allclose(V, U, atol=1e-13)
