"""Pins of the oracle's hyperbolic update against exact solutions: Sod and a
water/air stiffened-gas shock tube (exact Riemann solver in
tests/exact_riemann.py), the Rankine-Hugoniot reflected-shock state at a
static rigid wall (the 1-D 400-cell workload), and consistency of the HLLC
flux with the physical flux of Sec. 2.1.1.  CPU only."""
import math

import numpy as np
import pytest

import exact_riemann as ER
import workloads as W
from oracle import Oracle


def run_to(o, t_end, cfl=0.8, max_steps=100000):
    t, steps = 0.0, 0
    while t < t_end * (1 - 1e-14) and steps < max_steps:
        dt = o.compute_dt(cfl)
        if t + dt > t_end:
            dt = t_end - t
        o.step(dt)
        t += dt
        steps += 1
    return steps


def sod(n):
    o = Oracle(1, (n,), (0.0,), (1.0,), [dict(kind="ideal", gamma=1.4)])
    x = (np.arange(n) + 0.5) / n
    left = x < 0.5
    w = np.zeros((4, n))
    w[0] = np.where(left, 1.0, 0.125)
    w[2] = np.where(left, 1.0, 0.1)
    o.set_prim(w)
    run_to(o, 0.2, cfl=0.6)
    rho_ex, _, p_ex, _ = ER.sample(ER.Side(1.0, 0.0, 1.0, 1.4), ER.Side(0.125, 0.0, 0.1, 1.4), (x - 0.5) / 0.2)
    return o.prim(), rho_ex, p_ex, x


def test_sod_converges_to_exact_solution():
    errs = []
    for n in (100, 200, 400):
        w, rho_ex, p_ex, x = sod(n)
        errs.append(np.mean(np.abs(w[0] - rho_ex)))
    assert errs[0] < 0.02
    assert errs[1] < 0.75 * errs[0] and errs[2] < 0.75 * errs[1]
    # shock position (exact 0.5 + 1.7522*0.2) within 2 cells at n = 400
    w, rho_ex, p_ex, x = sod(400)
    grad = np.abs(np.diff(w[0]))
    xs = x[np.argmax(grad[x[:-1] > 0.8]) + np.searchsorted(x, 0.8)]
    assert abs(xs - (0.5 + 1.75215573 * 0.2)) < 2.5 / 400


def test_water_air_shock_tube_two_materials():
    """Stiffened-gas water (rho 1000, p 1e9) against air (rho 50, p 1e5),
    interface at x = 0.7, t = 240 us: the mixture density follows the exact
    solution and the material interface stays within two cells of it."""
    n = 400
    water = dict(kind="stiffened", gamma=4.4, pinf=6e8)
    air = dict(kind="ideal", gamma=1.4)
    o = Oracle(1, (n,), (0.0,), (1.0,), [water, air])
    x = (np.arange(n) + 0.5) / n
    left = x < 0.7
    w = np.zeros((6, n))
    w[0] = np.where(left, 1 - 1e-8, 1e-8)
    w[1] = 1000.0
    w[2] = 50.0
    w[4] = np.where(left, 1e9, 1e5)
    o.set_prim(w)
    t_end = 240e-6
    run_to(o, t_end, cfl=0.6)
    wp = o.prim()
    phi = wp[0]
    rho = phi * wp[1] + (1 - phi) * wp[2]
    L, R = ER.Side(1000.0, 0.0, 1e9, 4.4, 6e8), ER.Side(50.0, 0.0, 1e5, 1.4, 0.0)
    rho_ex, u_ex, p_ex, side = ER.sample(L, R, (x - 0.7) / t_end)
    rel_l1 = np.mean(np.abs(rho - rho_ex)) / np.mean(rho_ex)
    assert rel_l1 < 0.02
    ps, us = ER.star_state(L, R)
    xi = x[np.argmin(np.abs(phi - 0.5))]
    assert abs(xi - (0.7 + us * t_end)) < 2.0 / n
    # pressure and velocity stay continuous and close to the star state at the contact
    k = np.argmin(np.abs(x - (0.7 + us * t_end)))
    assert wp[4, k] == pytest.approx(ps, rel=0.05)
    assert wp[3, k] == pytest.approx(us, rel=0.05)


def rh_reflected(mach, g=1.4, rho1=1.225, p1=1e5):
    """Closed-form Rankine-Hugoniot incident and wall-reflected states."""
    rho2, u2, p2 = W.ideal_shock_state(mach, g, rho1, p1)
    rhs = mach / (mach * mach - 1) * math.sqrt(1 + 2 * (g - 1) / (g + 1) ** 2 * (mach * mach - 1) * (g + 1 / mach ** 2))
    # M_R/(M_R^2-1) = rhs  ->  M_R = (1 + sqrt(1 + 4 rhs^2)) / (2 rhs)
    MR = (1 + math.sqrt(1 + 4 * rhs * rhs)) / (2 * rhs)
    p5 = p2 * (1 + 2 * g / (g + 1) * (MR * MR - 1))
    rho5 = rho2 * (g + 1) * MR * MR / ((g - 1) * MR * MR + 2)
    c2 = math.sqrt(g * p2 / rho2)
    vs = MR * c2 - u2   # reflected shock speed in the lab (leftward)
    return dict(rho2=rho2, u2=u2, p2=p2, MR=MR, p5=p5, rho5=rho5, vs=vs)


def test_rh_reflected_values():
    """The closed form reproduces the textbook numbers for M = 2 in air."""
    s = rh_reflected(2.0)
    assert s["p5"] == pytest.approx(1.5e6, rel=1e-9)
    assert s["rho5"] == pytest.approx(7.35, rel=1e-9)
    assert s["vs"] == pytest.approx(338.0617, rel=1e-6)


def test_reflected_shock_at_static_rigid_body():
    """1-D workload (400 cells, M2 shock at 0.3, rigid surface at 0.7):
    the plateau behind the reflected shock matches p5, rho5, u5 = 0 within 1 %
    and the reflected shock is within two cells of its exact position."""
    wl = W.shock_reflection_1d(400)
    o = Oracle.from_workload(wl)
    s = rh_reflected(2.0)
    c1 = math.sqrt(1.4e5 / 1.225)
    t_hit = 0.4 / (2.0 * c1)
    t_end = 8.874e-4
    run_to(o, t_end, cfl=0.8)
    w = o.prim()
    x = (np.arange(400) + 0.5) / 400
    plateau = (x > 0.62) & (x < 0.68)
    assert np.mean(w[0, plateau]) == pytest.approx(s["rho5"], rel=0.01)
    assert np.mean(w[2, plateau]) == pytest.approx(s["p5"], rel=0.01)
    assert np.max(np.abs(w[1, plateau])) < 0.01 * s["u2"]
    x_exact = 0.7 - s["vs"] * (t_end - t_hit)
    sel = (x > 0.5) & (x < 0.69)
    xs = x[sel][np.argmax(np.abs(np.gradient(w[0, sel])))]
    assert abs(xs - x_exact) < 2.0 / 400


def physical_flux_2d(o, w, d):
    """Flux of Sec. 2.1.1 from a primitive state (two-material solid, 2-D)."""
    import oracle as ORC
    q = o.prim_to_cons(w)
    cl = o.closure(q)
    A = np.array([[w[6], w[7], 0], [w[8], w[9], 0], [0, 0, w[10]]])
    dH, _ = ORC.vbar_log(A)
    p, G = cl["p"], cl["G"]
    u = np.array([w[3], w[4], 0.0])
    sig = -p * np.eye(3) + 2 * G * dH
    rho = q[1] + q[2]
    F = np.zeros(12)
    F[0] = w[0] * u[d]
    F[1], F[2] = q[1] * u[d], q[2] * u[d]
    for a in range(2):
        F[3 + a] = rho * u[a] * u[d] - sig[a, d]
    F[5] = q[5] * u[d] - u @ sig[:, d]
    comps = [(0, 0), (0, 1), (1, 0), (1, 1), (2, 2)]
    for c, (a, b) in enumerate(comps):
        F[6 + c] = A[a, b] * u[d] - A[d, b] * u[a]
    return F


@pytest.mark.parametrize("d", [0, 1])
def test_hllc_consistency_with_physical_flux(d):
    o = Oracle(2, (4, 4), (0.0, 0.0), (1.0, 1.0), [W.ALUMINIUM, W.AIR], solid=True)
    w = np.array([0.7, 2710.0, 1.3, 210.0, -75.0, 2e8, 1.01, 0.02, -0.01, 0.985, 1.003, 0.3])
    F, us, vrow = o.riemann(d, w, w)
    Fp = physical_flux_2d(o, w, d)
    np.testing.assert_allclose(F[:11], Fp[:11], rtol=1e-12, atol=1e-12 * np.abs(Fp).max())
    assert us[d] == pytest.approx(w[3 + d], rel=1e-13)


def test_hllc_mirror_symmetry():
    """Swapping left/right and reversing the normal velocity reverses the
    mass and energy flux and keeps the normal-momentum flux."""
    o = Oracle(1, (4,), (0.0,), (1.0,), [W.AIR, W.WATER])
    wL = np.array([0.9, 1.5, 1000.0, 120.0, 3e5, 0.0])
    wR = np.array([0.2, 1.1, 1010.0, -40.0, 1e5, 0.0])
    F1, us1, _ = o.riemann(0, wL, wR)
    mL, mR = wL.copy(), wR.copy()
    mL[3], mR[3] = -wL[3], -wR[3]
    F2, us2, _ = o.riemann(0, mR, mL)
    np.testing.assert_allclose(F2[[0, 1, 2, 4]], -F1[[0, 1, 2, 4]], rtol=1e-12)
    assert F2[3] == pytest.approx(F1[3], rel=1e-12)
    assert us2[0] == pytest.approx(-us1[0], rel=1e-12)


def test_gas_solid_face_transmits_no_shear():
    """A sheared, sliding solid against gas at rest: the tangential traction at
    the face is the gas's, zero, so the tangential momentum flux is only the
    momentum carried by the mass flux, however large the solid's shear stress,
    and the face tangential velocity is the solid's (free slip)."""
    o = Oracle(2, (4, 4), (0.0, 0.0), (1.0, 1.0), [W.ALUMINIUM, W.AIR], solid=True)
    air = np.array([0.0, 2700.0, 1.225, 0.0, 0.0, 1e5, 1.0, 0.0, 0.0, 1.0, 1.0, 0.0])
    s = 0.01
    al = np.array([1.0, 2700.0, 1.225, 400.0, 0.0, 1e5, 1.0, s, 0.0, 1.0, 1.0, 0.0])
    F, us, _ = o.riemann(1, air, al)          # face normal to y, gas below, solid above
    mass = F[1] + F[2]
    ux_up = 0.0 if us[1] >= 0.0 else 400.0     # tangential velocity carried across
    sig_xy = 2 * o.closure(o.prim_to_cons(al))["G"] * oracle_devH_xy(s)
    assert abs(F[3] - mass * ux_up) <= 1e-9 * abs(sig_xy)
    # the solid's shear stress is released by a shear wave: u* = u + sigma_xy / Z
    Z = math.sqrt(2700.0 * o.closure(o.prim_to_cons(al))["G"])
    assert us[0] == pytest.approx(400.0 + sig_xy / Z, rel=1e-12)
    F2, _, _ = o.riemann(1, al, al)
    assert F2[3] == pytest.approx(-sig_xy, rel=1e-9)  # the solid alone does carry shear


def oracle_devH_xy(s):
    import oracle as ORC
    dH, _ = ORC.vbar_log(np.array([[1.0, s, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]]))
    return dH[0, 1]
