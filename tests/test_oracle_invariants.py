"""Invariant pins of the oracle: uniform pressure/velocity across material
interfaces (Abgrall), quiescent and co-moving bodies, conservation on a
periodic grid, THINC translation of a step in r, mirror symmetry, and the
summation-by-parts identity of the pressure-force sum.  CPU only."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import Oracle


def steps(o, k, cfl=0.5):
    for _ in range(k):
        o.step(o.compute_dt(cfl))


def two_fluid_interface(dim, n):
    nn = (n,) * dim
    o = Oracle(dim, nn, (0.0,) * dim, (1.0,) * dim, [W.AIR, W.WATER], periodic=(1,) * dim)
    X, Y, _ = W.cell_centres(nn, (0.0,) * dim, (1.0,) * dim)
    blob = (np.hypot(X - 0.5, Y - 0.5) < 0.3) if dim == 2 else (np.abs(X - 0.5) < 0.25)
    L = W.layout(dim, 2, False)
    w = np.zeros((L["nvar"], X.size))
    w[0] = np.where(blob, 1e-8, 1 - 1e-8)
    w[0] += 0.3 * np.exp(-((X - 0.5) ** 2) / 0.02) * (w[0] > 0.5) * 0   # sharp interface
    w[1] = np.where(blob, 1.0, 1.2)
    w[2] = 1000.0
    w[L["iu"]] = 50.0
    if dim == 2:
        w[L["iu"] + 1] = -20.0
    w[L["ip"]] = 1e5
    o.set_prim(w)
    return o, L


@pytest.mark.parametrize("dim,n,k", [(1, 64, 60), (2, 32, 20)])
def test_abgrall_uniform_pressure_velocity(dim, n, k):
    o, L = two_fluid_interface(dim, n)
    steps(o, k)
    w = o.prim()
    assert np.max(np.abs(w[L["ip"]] / 1e5 - 1)) < 1e-9
    assert np.max(np.abs(w[L["iu"]] / 50.0 - 1)) < 1e-9
    if dim == 2:
        assert np.max(np.abs(w[L["iu"] + 1] / -20.0 - 1)) < 1e-9
    # the interface moved and stayed sharp (THINC): few mixed cells
    phi = w[0]
    assert np.count_nonzero((phi > 0.01) & (phi < 0.99)) < 6 * (n if dim == 2 else 1) * (2 if dim == 2 else 2)


def body_state(u=(0.0, 0.0), vr=(0.0, 0.0), n=32):
    nn = (n, n)
    o = Oracle(2, nn, (0.0, 0.0), (1.0, 1.0), [W.AIR])
    X, Y, _ = W.cell_centres(nn, (0.0, 0.0), (1.0, 1.0))
    w = np.zeros((5, X.size))
    w[0] = 1.225
    w[1], w[2] = u
    w[3] = 1e5
    w[4] = W.rigid_profile(np.hypot(X - 0.45, Y - 0.55) - 0.2, 1.0 / n)
    o.set_prim(w)
    o.set_body(v=(vr[0], vr[1], 0.0))
    return o


def test_quiescent_gas_with_static_body_is_unchanged():
    o = body_state()
    q0 = o.cons()
    steps(o, 10)
    q1 = o.cons()
    scales = [1.225, 1.225 * 338.0, 1.225 * 338.0, 2.5e5, 1.0]   # rho, rho c, rho c, rho E, r
    for v in range(q0.shape[0]):
        np.testing.assert_allclose(q1[v], q0[v], rtol=1e-13, atol=1e-13 * scales[v])


def test_uniform_flow_with_comoving_body_stays_uniform():
    u = (120.0, -70.0)
    o = body_state(u=u, vr=u)
    steps(o, 10)
    w = o.prim()
    np.testing.assert_allclose(w[0], 1.225, rtol=1e-12)
    np.testing.assert_allclose(w[1], u[0], rtol=1e-11)
    np.testing.assert_allclose(w[2], u[1], rtol=1e-11)
    np.testing.assert_allclose(w[3], 1e5, rtol=1e-11)


def test_conservation_periodic_two_materials():
    wl = W.random_state(2, (24, 20), 2, False, seed=7, periodic=(1, 1), body=False)
    o = Oracle(2, wl.n, wl.lo, wl.hi, wl.materials, periodic=(1, 1))
    o.set_prim(wl.prim)
    q0 = o.cons().sum(axis=1)
    steps(o, 5)
    q1 = o.cons().sum(axis=1)
    scale = np.abs(o.cons()).sum(axis=1)
    # phasic masses, momenta, energy are conserved; phi and r are not conserved variables
    for v in (1, 2, 3, 4, 5):
        assert abs(q1[v] - q0[v]) <= 1e-13 * scale[v], v


def test_conservation_periodic_solid():
    wl = W.random_state(2, (20, 16), 2, True, seed=3, periodic=(1, 1), body=False, amp=0.02)
    o = Oracle(2, wl.n, wl.lo, wl.hi, wl.materials, solid=True, periodic=(1, 1))
    o.set_prim(wl.prim)
    q0 = o.cons().sum(axis=1)
    for _ in range(3):
        o.step(o.compute_dt(0.5))   # no mask (r = 0); plastic return keeps mass/momentum/energy
    q1 = o.cons().sum(axis=1)
    scale = np.abs(o.cons()).sum(axis=1)
    for v in (1, 2, 3, 4, 5):
        assert abs(q1[v] - q0[v]) <= 1e-13 * scale[v], v


def r_step_translation(use_thinc, n=64, periods=1.0):
    v = 100.0
    o = Oracle(1, (n,), (0.0,), (1.0,), [W.AIR], periodic=(1,))
    o.set_options(use_thinc=use_thinc)
    x = (np.arange(n) + 0.5) / n
    w = np.zeros((4, n))
    w[0] = 1.225
    w[1] = v            # gas co-moving with the body: the flow stays uniform
    w[2] = 1e5
    w[3] = np.where((x > 0.25) & (x < 0.6), 1.0, 0.0)
    o.set_prim(w)
    o.set_body(v=(v, 0, 0))
    t_end = periods * 1.0 / v
    t = 0.0
    while t < t_end * (1 - 1e-13):
        dt = min(o.compute_dt(0.4), t_end - t)
        o.step(dt)
        t += dt
    return x, o.prim()[3], w[3]


def test_thinc_translation_of_rigid_field():
    x, r, r0 = r_step_translation(True)
    assert r.sum() == pytest.approx(r0.sum(), rel=1e-12)
    width = np.count_nonzero((r > 0.05) & (r < 0.95))
    assert width <= 2 * 3          # two interfaces, at most 3 cells each
    _, r_m, _ = r_step_translation(False)
    assert np.count_nonzero((r_m > 0.05) & (r_m < 0.95)) > width   # MUSCL alone is more diffuse
    assert np.mean(np.abs(r - r0)) < np.mean(np.abs(r_m - r0))


def test_mirror_symmetry_cylinder():
    wl = W.cylinder_2d(48)
    o = Oracle.from_workload(wl)
    for _ in range(15):
        o.step(o.compute_dt(0.8))
    w = o.prim().reshape(5, 48, 48)        # [var, y, x]
    flip = w[:, ::-1, :]
    for v, sgn in ((0, 1), (1, 1), (2, -1), (3, 1), (4, 1)):
        scale = np.abs(w[v]).max()
        assert np.max(np.abs(w[v] - sgn * flip[v])) <= 1e-11 * scale, v


def test_force_uniform_pressure_is_boundary_flux_only():
    """Uniform p: the central-difference sum telescopes, leaving only the
    (tiny) values of r on the transmissive boundary."""
    n = 32
    o = body_state(n=n)
    F = o.force()
    r = o.prim()[4].reshape(n, n)          # [y, x]
    h = 1.0 / n
    Fx = 1e5 * h * np.sum(r[:, -1] - r[:, 0])
    Fy = 1e5 * h * np.sum(r[-1, :] - r[0, :])
    scale = 1e5 * 0.4
    assert abs(F[0] - Fx) < 1e-12 * scale and abs(F[1] - Fy) < 1e-12 * scale
    assert abs(F[0]) < 1e-6 * scale and abs(F[1]) < 1e-6 * scale


def test_force_linear_pressure_summation_by_parts():
    """p = p0 + g . x gives sum p grad(r) dV = -g sum r dV exactly (discrete
    summation by parts; r vanishes near the boundary)."""
    n = 40
    nn = (n, n)
    o = Oracle(2, nn, (0.0, 0.0), (1.0, 1.0), [W.AIR])
    X, Y, _ = W.cell_centres(nn, (0.0, 0.0), (1.0, 1.0))
    g = np.array([3.0e5, -1.2e5])
    w = np.zeros((5, X.size))
    w[0] = 1.225
    w[3] = 1e5 + g[0] * X + g[1] * Y
    r = W.rigid_profile(np.hypot(X - 0.5, Y - 0.5) - 0.2, 1.0 / n)
    w[4] = r
    o.set_prim(w)
    F = o.force()
    dV = 1.0 / n ** 2
    expect = -g * r.sum() * dV
    np.testing.assert_allclose(F[:2], expect, rtol=1e-9)
