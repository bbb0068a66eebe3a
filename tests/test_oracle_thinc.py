"""Pins of the oracle's THINC face values (Sec. 3.1, MUSCL-BVD-THINC): the
face values must be the end values of the tanh profile whose cell average is
the cell value, checked by quadrature of that profile; monotone cells only.
CPU only."""
import math

import numpy as np
import pytest

import oracle

BETA = 1.6


def profile_from_faces(qm, q0, qp, fm):
    """Recover the jump centre x_c from the left face value and return the
    tanh profile q(x) on [0,1]."""
    qmin, qmax = min(qm, qp), max(qm, qp)
    dq = qmax - qmin
    th = 1.0 if qp >= qm else -1.0
    t0 = (2.0 * (fm - qmin) / dq - 1.0) / th          # = tanh(-beta x_c)
    xc = -math.atanh(t0) / BETA
    return lambda x: qmin + 0.5 * dq * (1.0 + th * np.tanh(BETA * (x - xc)))


@pytest.mark.parametrize("qm,q0,qp", [(0.0, 0.3, 1.0), (1.0, 0.9, 0.0), (0.2, 0.21, 0.9),
                                      (1e-8, 0.5, 1.0 - 1e-8), (5.0, 4.0, -2.0)])
def test_thinc_face_values_match_cell_average(qm, q0, qp):
    res = oracle.thinc(qm, q0, qp, BETA)
    assert res is not None
    fm, fp = res
    q = profile_from_faces(qm, q0, qp, fm)
    # Gauss-Legendre quadrature of the profile over the cell
    xg, wg = np.polynomial.legendre.leggauss(60)
    avg = 0.5 * np.sum(wg * q(0.5 * (xg + 1.0)))
    assert avg == pytest.approx(q0, rel=1e-12, abs=1e-13)
    assert q(1.0) == pytest.approx(fp, rel=1e-12, abs=1e-13)
    lo, hi = min(qm, qp), max(qm, qp)
    assert lo <= fm <= hi and lo <= fp <= hi


def test_thinc_not_applied_to_extrema_or_flat():
    assert oracle.thinc(0.0, 1.0, 0.0, BETA) is None       # local maximum
    assert oracle.thinc(0.5, 0.5, 0.7, BETA) is None       # flat on one side
    assert oracle.thinc(0.0, 1e-10, 1.0, BETA) is None     # C below 1e-8


def test_thinc_mirror_symmetry():
    fm, fp = oracle.thinc(0.1, 0.35, 0.8, BETA)
    gm, gp = oracle.thinc(0.8, 0.35, 0.1, BETA)
    assert gm == pytest.approx(fp, rel=1e-14) and gp == pytest.approx(fm, rel=1e-14)


def test_thinc_centred_jump_is_symmetric():
    """C = 1/2: the jump sits in the cell centre and the face values are
    q_min + dq/2 (1 -/+ tanh(beta/2))."""
    fm, fp = oracle.thinc(0.0, 0.5, 1.0, BETA)
    assert fm == pytest.approx(0.5 * (1 - math.tanh(BETA / 2)), rel=1e-14)
    assert fp == pytest.approx(0.5 * (1 + math.tanh(BETA / 2)), rel=1e-14)
