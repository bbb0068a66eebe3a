"""Pins of the seeding options of Sec. 3.2-3.3 in the oracle: the line/cell
geometry behind ELVIRA, the ELVIRA normal itself (exact for straight
interfaces, as the method is built to be), the fixed 1.5 dx probe, and the
use of the step-start state by every seeded cell.  CPU only."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import Oracle, cut_alpha, cut_fraction, elvira


def square_fraction(nx, ny, alpha, x0, y0, hx, hy):
    """Closed form of the area of {n.x <= alpha} in a rectangle: map to the
    unit square, flip negative coefficients, then inclusion-exclusion of the
    quadratic ramps (a^2 - (a-m1)^2_+ - (a-m2)^2_+ + (a-m1-m2)^2_+) / (2 m1 m2)."""
    a = alpha - nx * x0 - ny * y0
    m1, m2 = nx * hx, ny * hy
    if m1 < 0:
        a -= m1
        m1 = -m1
    if m2 < 0:
        a -= m2
        m2 = -m2
    if m1 < m2:
        m1, m2 = m2, m1
    if m2 <= 1e-9 * m1 or m1 == 0.0:       # a line parallel to a side: the linear limit
        if m1 == 0.0:
            return 1.0 if a >= 0 else 0.0
        return min(max(a / m1, 0.0), 1.0)
    r = lambda t: max(t, 0.0) ** 2
    return (r(a) - r(a - m1) - r(a - m2) + r(a - m1 - m2)) / (2.0 * m1 * m2)


def test_cut_fraction_matches_the_closed_form():
    rng = np.random.default_rng(3)
    for _ in range(2000):
        th = rng.uniform(0, 2 * math.pi)
        n = (math.cos(th), math.sin(th))
        if min(abs(n[0]), abs(n[1])) < 0.05:    # the closed form cancels badly near the axes
            continue
        x0, y0 = rng.uniform(-2, 2, 2)
        hx, hy = rng.uniform(0.3, 2.0, 2)
        cx, cy = x0 + hx / 2, y0 + hy / 2
        alpha = n[0] * cx + n[1] * cy + rng.uniform(-1, 1) * (abs(n[0]) * hx + abs(n[1]) * hy) * 0.6
        f = cut_fraction(n, alpha, x0, y0, hx, hy)
        assert f == pytest.approx(square_fraction(n[0], n[1], alpha, x0, y0, hx, hy), abs=1e-12)
        # the two sides of the line fill the cell
        assert f + cut_fraction((-n[0], -n[1]), -alpha, x0, y0, hx, hy) == pytest.approx(1.0, abs=1e-13)


def test_cut_fraction_axis_aligned_and_diagonal():
    assert cut_fraction((1.0, 0.0), 0.25, 0.0, 0.0, 1.0, 1.0) == pytest.approx(0.25, abs=1e-15)
    assert cut_fraction((0.0, -1.0), -0.6, 0.0, 0.0, 1.0, 1.0) == pytest.approx(0.4, abs=1e-15)
    s = 1 / math.sqrt(2)
    assert cut_fraction((s, s), 0.5 * s, 0.0, 0.0, 1.0, 1.0) == pytest.approx(0.125, abs=1e-15)
    assert cut_fraction((s, s), 10.0, 0.0, 0.0, 1.0, 1.0) == 1.0
    assert cut_fraction((s, s), -10.0, 0.0, 0.0, 1.0, 1.0) == 0.0


def test_cut_alpha_inverts_the_fraction():
    rng = np.random.default_rng(4)
    for _ in range(300):
        th = rng.uniform(0, 2 * math.pi)
        n = (math.cos(th), math.sin(th))
        hx, hy = rng.uniform(0.5, 1.5, 2)
        f = rng.uniform(0.0, 1.0)
        a = cut_alpha(n, f, -hx / 2, -hy / 2, hx, hy)
        assert square_fraction(n[0], n[1], a, -hx / 2, -hy / 2, hx, hy) == pytest.approx(f, abs=1e-12)


def line_block(theta, alpha, hx=1.0, hy=1.0):
    """r of the 3x3 block for the body {n.x <= alpha}, n = (cos, sin) outward,
    cell (k, l) centred at (k hx, l hy), from the closed form."""
    n = (math.cos(theta), math.sin(theta))
    return np.array([[square_fraction(n[0], n[1], alpha, (k - 0.5) * hx, (l - 0.5) * hy, hx, hy)
                      for k in (-1, 0, 1)] for l in (-1, 0, 1)])


def youngs(b, hx=1.0, hy=1.0):
    g = np.array([(b[1, 2] - b[1, 0]) / (2 * hx), (b[2, 1] - b[0, 1]) / (2 * hy)])
    return -g / np.linalg.norm(g)


@pytest.mark.parametrize("hx,hy", [(1.0, 1.0), (1.0, 0.8)])
def test_elvira_reproduces_straight_interfaces(hx, hy):
    """Pilliod & Puckett's property: a straight interface through the centre
    cell whose height function stays inside the block is recovered exactly,
    in every orientation; Youngs' normal is not."""
    rng = np.random.default_rng(5)
    worst_youngs = 0.0
    for axis in range(4):
        for _ in range(60):
            theta = axis * math.pi / 2 + rng.uniform(-0.55, 0.55)    # |tan| <= 0.62 off an axis
            alpha = rng.uniform(-0.15, 0.15) * min(hx, hy)
            b = line_block(theta, alpha, hx, hy)
            assert 0.0 < b[1, 1] < 1.0
            n = elvira(b, hx, hy)
            exact = np.array([math.cos(theta), math.sin(theta)])
            np.testing.assert_allclose(n, exact, atol=1e-11)
            worst_youngs = max(worst_youngs, np.abs(youngs(b, hx, hy) - exact).max())
    assert worst_youngs > 1e-2


def test_elvira_orientation_and_symmetry():
    b = line_block(math.pi / 2, 0.0)         # body below y = 0
    np.testing.assert_allclose(elvira(b), [0.0, 1.0], atol=1e-14)
    np.testing.assert_allclose(elvira(b[::-1, :]), [0.0, -1.0], atol=1e-14)     # mirrored in y
    np.testing.assert_allclose(elvira(b.T), [1.0, 0.0], atol=1e-14)            # body left of x = 0
    rng = np.random.default_rng(6)
    blk = np.clip(rng.uniform(-0.2, 1.2, (3, 3)), 0, 1)
    n = elvira(blk)
    assert abs(np.linalg.norm(n) - 1.0) < 1e-14
    # a quarter turn of the block turns the normal with it
    n_rot = elvira(np.rot90(blk, k=1))   # rot90 maps (k, l) -> (-l, k) in the array's (row=l, col=k) view
    assert abs(np.linalg.norm(n_rot) - 1.0) < 1e-14


def sharp_wall_state(n, theta, u_along, offset=0.013):
    """Quiescent-pressure air over a straight inclined wall through the domain
    centre, r from exact cell fractions, uniform flow along the wall."""
    lo, hi = (0.0, 0.0), (1.0, 1.0)
    h = 1.0 / n
    X, Y, _ = W.cell_centres((n, n), lo, hi)
    nx, ny = math.cos(theta), math.sin(theta)
    alpha = nx * 0.5 + ny * 0.5 + offset
    r = np.array([square_fraction(nx, ny, alpha, x - h / 2, y - h / 2, h, h) for x, y in zip(X, Y)])
    w = np.zeros((5, n * n))
    w[0], w[3] = 1.225, 1e5
    w[1], w[2] = -ny * u_along, nx * u_along
    w[4] = r
    return w, np.array([nx, ny])


@pytest.mark.parametrize("theta", [0.3, 2.0, 4.4])
def test_elvira_seeding_normals_exact_on_a_straight_wall(theta):
    n = 40
    w, nrm = sharp_wall_state(n, theta, 80.0)
    o = Oracle(2, (n, n), (0.0, 0.0), (1.0, 1.0), [W.AIR])
    o.set_variants(normal_method=1)
    o.set_prim(w)
    o.seed()
    ns = o.seed_normals()
    I, J = np.meshgrid(np.arange(n), np.arange(n))
    interior = ((I > 0) & (I < n - 1) & (J > 0) & (J < n - 1)).ravel()    # 3x3 block inside the grid
    cut = (w[4] > 0.5) & (w[4] < 1.0 - 1e-9) & (np.abs(ns).sum(axis=0) > 0) & interior
    assert cut.sum() > 10
    np.testing.assert_allclose(ns[0, cut], nrm[0], atol=1e-11)
    np.testing.assert_allclose(ns[1, cut], nrm[1], atol=1e-11)
    # the flow along the wall is reflected into itself: seeded cut cells keep the free stream
    wp = o.prim()
    np.testing.assert_allclose(wp[1, cut], w[1, cut], atol=1e-9)
    np.testing.assert_allclose(wp[2, cut], w[2, cut], atol=1e-9)
    # Youngs normals on the same field are not exact
    o2 = Oracle(2, (n, n), (0.0, 0.0), (1.0, 1.0), [W.AIR])
    o2.set_prim(w)
    o2.seed()
    ny_ = o2.seed_normals()
    assert np.abs(ny_[:2, cut] - nrm[:, None]).max() > 1e-3


@pytest.mark.parametrize("side", ["left", "right"])
def test_fixed_probe_interpolates_at_one_and_a_half_cells(side):
    """A planar body face normal to x and density, pressure linear in x: the
    fixed probe reads the state at x_c + 1.5 dx n exactly (multilinear
    interpolation of a linear field), from the state before seeding even where
    the probe's cells are themselves seeded (body on the right: the probe looks
    back over cells the loop has already visited)."""
    nx_, ny_ = 40, 6
    lo, hi = (0.0, 0.0), (1.0, 0.15)
    X, Y, _ = W.cell_centres((nx_, ny_), lo, hi)
    dx = 1.0 / nx_
    s = (X - 0.5) if side == "left" else (0.5 - X)      # signed distance, positive outside the body
    w = np.zeros((5, X.size))
    w[0] = 1.0 + 0.3 * X
    w[3] = 1e5 * (1.0 + 0.2 * X)
    w[4] = W.rigid_profile(s, dx)
    o = Oracle(2, (nx_, ny_), lo, hi, [W.AIR])
    o.set_variants(probe_mode=1)
    o.set_prim(w)
    o.seed()
    seeded = np.abs(o.seed_normals()).sum(axis=0) > 0
    assert seeded.sum() >= 2 * ny_
    sign = 1.0 if side == "left" else -1.0
    xp = X + sign * 1.5 * dx
    wp = o.prim()
    np.testing.assert_allclose(wp[0, seeded], 1.0 + 0.3 * xp[seeded], rtol=1e-13)
    np.testing.assert_allclose(wp[3, seeded], 1e5 * (1.0 + 0.2 * xp[seeded]), rtol=1e-13)


def test_stepped_probe_unchanged_by_the_options():
    """Youngs + stepped probe is the default; the plain reflected shock still
    matches its committed behaviour when the other options are left off."""
    wl = W.cylinder_2d(48)
    a = Oracle.from_workload(wl)
    b = Oracle.from_workload(wl, normal_method=0, probe_mode=0)
    for _ in range(3):
        dt = a.compute_dt(0.8)
        a.step(dt)
        b.step(dt)
    np.testing.assert_array_equal(a.cons(), b.cons())


@pytest.mark.parametrize("opts", [dict(normal_method=1), dict(probe_mode=1), dict(normal_method=1, probe_mode=1)])
def test_options_keep_quiescent_and_comoving_states(opts):
    for u in ((0.0, 0.0), (120.0, -70.0)):
        nn = 32
        X, Y, _ = W.cell_centres((nn, nn), (0.0, 0.0), (1.0, 1.0))
        w = np.zeros((5, X.size))
        w[0], w[1], w[2], w[3] = 1.225, u[0], u[1], 1e5
        w[4] = W.rigid_profile(np.hypot(X - 0.45, Y - 0.55) - 0.2, 1.0 / nn)
        o = Oracle(2, (nn, nn), (0.0, 0.0), (1.0, 1.0), [W.AIR])
        o.set_variants(**opts)
        o.set_prim(w)
        o.set_body(v=(u[0], u[1], 0.0))
        for _ in range(4):
            o.step(o.compute_dt(0.5))
        wp = o.prim()
        np.testing.assert_allclose(wp[0], 1.225, rtol=1e-12)
        np.testing.assert_allclose(wp[3], 1e5, rtol=1e-11)
        np.testing.assert_allclose(wp[1], u[0], atol=1e-9 * 338)
