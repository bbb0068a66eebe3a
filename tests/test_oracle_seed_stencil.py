"""Pin of the probe-stencil reading of the seeding (Sec. 3.2): a corner of
the probe point's enclosing cells whose multilinear weight is (near) zero is
not part of the stencil.  At whole-cell probe steps along an axis-aligned
normal the probe point lies on a cell centre, and the zero-weight corner is
the rigid cell itself for a body on one side and a fluid cell for a body on
the other; the seeding must not depend on which side the body is on.  CPU
only."""
import numpy as np
import pytest

import workloads as W
from oracle import Oracle


def planar_1d(n, body_right, rng):
    """Smooth random gas left of a body face at x = 0.7 (or its mirror
    image: body left of x = 0.3, state mirrored, velocity negated)."""
    X, _, _ = W.cell_centres((n,), (0.0,), (1.0,))
    w = np.zeros((4, n))
    w[0] = 1.2 + 0.3 * np.sin(7 * X) + 0.05 * rng.standard_normal(n)
    w[1] = 80.0 * np.cos(5 * X) + 10.0 * rng.standard_normal(n)
    w[2] = 1e5 * (1 + 0.2 * np.sin(3 * X))
    w[3] = W.rigid_profile(0.7 - X, 1.0 / n)
    if not body_right:
        w = w[:, ::-1].copy()
        w[1] = -w[1]
    o = Oracle(1, (n,), (0.0,), (1.0,), [W.AIR])
    o.set_prim(w)
    return o, w


@pytest.mark.parametrize("n", [64, 100, 257])
def test_seeding_is_mirror_symmetric(n):
    rng = np.random.default_rng(n)
    oR, wR = planar_1d(n, True, np.random.default_rng(n))
    oL, wL = planar_1d(n, False, np.random.default_rng(n))
    oR.seed()
    oL.seed()
    pR, pL = oR.prim(), oL.prim()
    mirror = pL[:, ::-1].copy()
    mirror[1] = -mirror[1]
    scale = np.abs(pR).max(axis=1, keepdims=True)
    assert np.max(np.abs(pR - mirror) / scale) < 1e-12
    # the seeding changed something (band cells exist on both sides)
    assert np.max(np.abs(pR - wR) / scale) > 1e-3


def test_first_band_cell_takes_its_neighbour_at_one_cell():
    """The first rigid cell next to the face: its s = 1.0 probe point is the
    centre of its fluid neighbour (weight 1), so it takes that cell's state
    with the velocity reflected, on either side."""
    n = 80
    for body_right in (True, False):
        o, w = planar_1d(n, body_right, np.random.default_rng(3))
        r = w[3]
        rigid = np.nonzero(r > 0.5)[0]
        i = rigid.min() if body_right else rigid.max()
        j = i - 1 if body_right else i + 1
        assert r[j] < 0.5
        o.seed()
        p = o.prim()
        assert p[0, i] == pytest.approx(w[0, j], rel=1e-13)
        assert p[2, i] == pytest.approx(w[2, j], rel=1e-13)
        assert p[1, i] == pytest.approx(-w[1, j], rel=1e-13)
