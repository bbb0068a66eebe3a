"""Seeded synthetic workloads shaped like the paper's tests.

This module is the one piece that both sides of the parity tests use: it
produces initial PRIMITIVE fields (volume fractions, phasic densities,
velocity, pressure, stretch tensor, rigid field r) as float64 numpy arrays,
plus the grid, the materials and the body.  It holds none of the method's
arithmetic: conversion to conserved variables, closures, fluxes and steps are
done separately by the oracle and by the CUDA library.

Primitive plane order (N materials, d dimensions, nv stretch components):
    phi_1..phi_{N-1}, rho_1..rho_N, u_1..u_d, p, V_1..V_nv, r
with nv = 0 for fluids and 3 / 5 / 9 for solids in 1-D / 2-D / 3-D, the
stored stretch components being (xx, yy, zz) in 1-D, (xx, xy, yx, yy, zz)
in 2-D and all nine (row-major) in 3-D.  Cell (i, j, k) is at flat index
i + nx * (j + ny * k).

Every workload is drawn from numpy.random.Generator(PCG64(seed)) with
seed = 1111806 + workload index (batched instance i: 1111806 * 1000 + i).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

SEED_BASE = 1111806

# Material records: the parameters each closure needs.  rho0 of a gas is the
# reference density its phasic density takes where it is absent from a cell.
AIR = dict(kind="ideal", gamma=1.4, rho0=1.225)
WATER = dict(kind="stiffened", gamma=4.4, pinf=6.0e8, rho0=1000.0)
# Aluminium-like Romenskii solid: rho0, K0, G0 and the yield stress are the
# impact workload's; alpha, beta, Gamma0 are the paper's Table 1 aluminium row.
HELIUM = dict(kind="ideal", gamma=1.67, rho0=0.166)
ALUMINIUM = dict(kind="romenskii", rho0=2700.0, K0=76.0e9, G0=26.0e9, alpha=0.627,
                 beta=2.288, Gamma0=1.484, sigY=0.3e9)

# Copper: the paper's Table 1 Romenskii constants and Table 2 Johnson-Cook
# constants (c1, c2 in Pa, T_melt in K, C_V in J/(kg K)).
COPPER = dict(kind="romenskii", rho0=8960.0, K0=130.1e9, G0=43.33e9, alpha=1.0, beta=3.0, Gamma0=2.0,
              jc_c1=0.09e9, jc_c2=0.292e9, jc_c3=0.025, jc_n=0.31, jc_m=1.09, jc_tmelt=1358.0, jc_cv=385.0)

PHI_PURE = 1.0e-8   # residual volume fraction of an absent material


@dataclasses.dataclass
class Workload:
    name: str
    dim: int
    n: tuple
    lo: tuple
    hi: tuple
    periodic: tuple
    materials: list
    solid: bool
    prim: np.ndarray          # (nvar, ncell) float64
    body_v: tuple = (0.0, 0.0, 0.0)
    body_x: tuple = (0.0, 0.0, 0.0)
    body_mass: float = 0.0
    body_dynamic: bool = False
    cfl: float = 0.8
    steps: int = 1
    t_end: Optional[float] = None
    walls: tuple = (0, 0, 0, 0, 0, 0)   # reflective wall on the low / high side of each direction
    history: bool = False               # solids: one plastic-strain plane per material after r

    @property
    def nmat(self) -> int:
        return len(self.materials)

    @property
    def nvar(self) -> int:
        return self.prim.shape[0]

    @property
    def ncell(self) -> int:
        return int(np.prod(self.n))


def layout(dim: int, nmat: int, solid: bool, history: bool = False) -> dict:
    """Plane offsets of the primitive / conserved vectors (history planes, one
    per material, after r for solids with plastic-strain history)."""
    nv = (3 if dim == 1 else 5 if dim == 2 else 9) if solid else 0
    iphi = 0
    irho = nmat - 1
    iu = 2 * nmat - 1
    ip = iu + dim
    iv = ip + 1
    ir = iv + nv
    nh = nmat if (solid and history) else 0
    return dict(nv=nv, iphi=iphi, irho=irho, iu=iu, ip=ip, iv=iv, ir=ir, ih=ir + 1, nh=nh, nvar=ir + 1 + nh)


def cell_centres(n, lo, hi):
    """Cell-centre coordinate arrays, flattened with x fastest."""
    axes = []
    for d in range(3):
        if d < len(n):
            dx = (hi[d] - lo[d]) / n[d]
            axes.append(lo[d] + (np.arange(n[d]) + 0.5) * dx)
        else:
            axes.append(np.zeros(1))
    Z, Y, X = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
    return X.ravel(), Y.ravel(), Z.ravel()


def ideal_shock_state(mach: float, gamma: float, rho1: float, p1: float):
    """Post-shock (rho2, u2, p2) of a right-running ideal-gas shock of Mach
    number `mach` into gas at rest (Rankine-Hugoniot)."""
    g = gamma
    c1 = math.sqrt(g * p1 / rho1)
    p2 = p1 * (1.0 + 2.0 * g / (g + 1.0) * (mach * mach - 1.0))
    rho2 = rho1 * (g + 1.0) * mach * mach / ((g - 1.0) * mach * mach + 2.0)
    u2 = mach * c1 * (1.0 - rho1 / rho2)
    return rho2, u2, p2


def rigid_profile(sdist: np.ndarray, dx: float) -> np.ndarray:
    """r = (1 - tanh(s/dx))/2 with s the signed distance, positive outside the
    body: a diffuse field about 2 cells wide, r = 0.5 on the surface."""
    return 0.5 * (1.0 - np.tanh(sdist / dx))


def _empty_prim(dim, nmat, solid, ncell):
    L = layout(dim, nmat, solid)
    w = np.zeros((L["nvar"], ncell))
    if solid:  # stretch tensor starts at the identity
        diag = {1: [0, 1, 2], 2: [0, 3, 4], 3: [0, 4, 8]}[dim]
        for c in diag:
            w[L["iv"] + c] = 1.0
    return w, L


# --------------------------------------------------------------- workloads

def shock_reflection_1d(n: int = 400, mach: float = 2.0) -> Workload:
    """1-D Mach `mach` shock at x=0.3 running into a static rigid body whose
    surface is at x=0.7 (body on the right), ideal-gas air at rest
    (rho 1.225, p 1e5)."""
    lo, hi = (0.0,), (1.0,)
    X, _, _ = cell_centres((n,), lo, hi)
    dx = 1.0 / n
    w, L = _empty_prim(1, 1, False, n)
    rho1, p1 = 1.225, 1.0e5
    rho2, u2, p2 = ideal_shock_state(mach, 1.4, rho1, p1)
    post = X < 0.3
    w[L["irho"]] = np.where(post, rho2, rho1)
    w[L["iu"]] = np.where(post, u2, 0.0)
    w[L["ip"]] = np.where(post, p2, p1)
    w[L["ir"]] = rigid_profile(0.7 - X, dx)
    return Workload("shock_reflection_1d_%d" % n, 1, (n,), lo, hi, (0,), [AIR], False, w,
                    cfl=0.8, steps=0, t_end=None)


def cylinder_2d(n: int = 512, mach: float = 3.0, radius: float = 0.1, ny: Optional[int] = None) -> Workload:
    """2-D planar Mach `mach` shock at x=0.2 over a static rigid cylinder of
    radius 0.1 at (0.5, 0.5) on [0,1]^2, air at rest (rho 1.225, p 1e5)."""
    ny = n if ny is None else ny
    lo, hi = (0.0, 0.0), (1.0, 1.0)
    X, Y, _ = cell_centres((n, ny), lo, hi)
    dx = min(1.0 / n, 1.0 / ny)
    w, L = _empty_prim(2, 1, False, n * ny)
    rho1, p1 = 1.225, 1.0e5
    rho2, u2, p2 = ideal_shock_state(mach, 1.4, rho1, p1)
    post = X < 0.2
    w[L["irho"]] = np.where(post, rho2, rho1)
    w[L["iu"]] = np.where(post, u2, 0.0)
    w[L["ip"]] = np.where(post, p2, p1)
    sd = np.hypot(X - 0.5, Y - 0.5) - radius
    w[L["ir"]] = rigid_profile(sd, dx)
    return Workload("cylinder_2d_%dx%d" % (n, ny), 2, (n, ny), lo, hi, (0, 0), [AIR], False, w,
                    cfl=0.8, steps=500)


def dynamic_body_2d(nx: int = 1024, ny: int = 512, mach: float = 3.0) -> Workload:
    """Free circular body (radius 0.05, density 7.6 x air) at (0.15, 0.05) on
    [0,2]x[0,1], air (gamma 1.4) over a water layer (stiffened gas, gamma 4.4,
    p_inf 6e8) below y = 0.03, Mach `mach` shock at x = 0.05 in the air."""
    lo, hi = (0.0, 0.0), (2.0, 1.0)
    X, Y, _ = cell_centres((nx, ny), lo, hi)
    dx = min(2.0 / nx, 1.0 / ny)
    w, L = _empty_prim(2, 2, False, nx * ny)
    rho_air, p1, rho_w = 1.225, 1.0e5, 1000.0
    rho2, u2, p2 = ideal_shock_state(mach, 1.4, rho_air, p1)
    water = Y < 0.03
    post = (X < 0.05) & ~water
    # material 1 is the water: its volume fraction is the stored one, so that
    # its 1e-8 trace in the air (whose p_inf term dominates the trace's share
    # of the mixture pressure) keeps full relative precision in FP32 storage
    w[L["iphi"]] = np.where(water, 1.0 - PHI_PURE, PHI_PURE)      # phi of water
    w[L["irho"]] = rho_w                                           # rho of water
    w[L["irho"] + 1] = np.where(post, rho2, rho_air)               # rho of air
    w[L["iu"]] = np.where(post, u2, 0.0)
    w[L["ip"]] = np.where(post, p2, p1)
    R = 0.05
    sd = np.hypot(X - 0.15, Y - 0.05) - R
    w[L["ir"]] = rigid_profile(sd, dx)
    mass = 7.6 * rho_air * math.pi * R * R
    return Workload("dynamic_body_2d_%dx%d" % (nx, ny), 2, (nx, ny), lo, hi, (0, 0), [WATER, AIR], False, w,
                    body_x=(0.15, 0.05, 0.0), body_mass=mass, body_dynamic=True, cfl=0.8, steps=2000)


def wedge_distance(X, Y, apex=(0.06, 0.05), half_angle_deg=30.0):
    """Signed distance (positive outside) to the infinite wedge with apex
    `apex`, axis +x and the given half-angle."""
    th = math.radians(half_angle_deg)
    xi = X - apex[0]
    eta = np.abs(Y - apex[1])
    proj = xi * math.cos(th) + eta * math.sin(th)
    line = -xi * math.sin(th) + eta * math.cos(th)
    return np.where(proj >= 0.0, line, np.hypot(xi, eta))


def wedge_2d(nx: int = 1200, mach: float = 10.0, angle_deg: float = 30.0) -> Workload:
    """Shock reflection from a wedge (the paper's wedge tests): non-dimensional
    ideal gas (gamma 1.4) at rest with rho 1.4, p 1 on [0,3]x[0,2], a planar
    Mach `mach` shock at x = 0.25, a rigid wedge rising from the floor at
    x = 0.5 at `angle_deg`; the floor y = 0 is a reflective wall, the other
    sides transmissive.  nx = 1200 (ny = 800) is the resolution of the
    paper's finest level (300x200 base with two refinements by 2); CFL 0.4."""
    ny = nx * 2 // 3
    lo, hi = (0.0, 0.0), (3.0, 2.0)
    X, Y, _ = cell_centres((nx, ny), lo, hi)
    dx = min(3.0 / nx, 2.0 / ny)
    gas = dict(kind="ideal", gamma=1.4)
    w, L = _empty_prim(2, 1, False, nx * ny)
    rho1, p1 = 1.4, 1.0
    rho2, u2, p2 = ideal_shock_state(mach, 1.4, rho1, p1)
    post = X < 0.25
    w[L["irho"]] = np.where(post, rho2, rho1)
    w[L["iu"]] = np.where(post, u2, 0.0)
    w[L["ip"]] = np.where(post, p2, p1)
    th = math.radians(angle_deg)
    sx, sy = X - 0.5, Y
    along = sx * math.cos(th) + sy * math.sin(th)
    above = -sx * math.sin(th) + sy * math.cos(th)
    sd = np.where(along >= 0.0, above, np.hypot(sx, sy))     # signed distance, positive in the gas
    w[L["ir"]] = rigid_profile(sd, dx)
    return Workload("wedge_2d_%dx%d_mach%g_%gdeg" % (nx, ny, mach, angle_deg), 2, (nx, ny), lo, hi, (0, 0), [gas],
                    False, w, cfl=0.4, steps=0, t_end=0.2 if mach >= 5 else 1.2, walls=(0, 0, 1, 0, 0, 0))


def impact_2d(n: int = 1024, seed_index: int = 4, solid_material: Optional[dict] = None) -> Workload:
    """Aluminium-like block [0.005,0.025]x[0.03,0.07] m moving at 400 m/s into
    a static rigid wedge (apex (0.06,0.05), half-angle 30 deg) on [0,0.1]^2,
    surrounded by air at rest; V starts at the identity; 1e-6 x 400 m/s
    Gaussian noise on both velocity components.  solid_material replaces the
    aluminium (e.g. COPPER, with its Johnson-Cook flow stress)."""
    mat = ALUMINIUM if solid_material is None else solid_material
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + seed_index))
    lo, hi = (0.0, 0.0), (0.1, 0.1)
    X, Y, _ = cell_centres((n, n), lo, hi)
    dx = 0.1 / n
    w, L = _empty_prim(2, 2, True, n * n)
    block = (X >= 0.005) & (X <= 0.025) & (Y >= 0.03) & (Y <= 0.07)
    w[L["iphi"]] = np.where(block, 1.0 - PHI_PURE, PHI_PURE)     # phi of the solid
    w[L["irho"]] = mat["rho0"]
    w[L["irho"] + 1] = 1.225
    noise = 1.0e-6 * 400.0 * rng.standard_normal((2, n * n))
    w[L["iu"]] = np.where(block, 400.0, 0.0) + noise[0]
    w[L["iu"] + 1] = noise[1]
    w[L["ip"]] = 1.0e5
    w[L["ir"]] = rigid_profile(wedge_distance(X, Y), dx)
    return Workload("impact_2d_%d" % n, 2, (n, n), lo, hi, (0, 0), [mat, AIR], True, w,
                    cfl=0.8, steps=3000)


def ellipse_instance(i: int, n: Optional[int] = None) -> Workload:
    """One instance of the batched workload: an n x n grid on [0,1]^2 with n
    drawn from {128,192,256,384,512}, a rigid ellipse centred at (0.5,0.5)
    with semi-axes U[0.05,0.15] and angle U[0,pi), and a shock of Mach
    U[1.5,3] at x = 0.2 in air at rest."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE * 1000 + i))
    sizes = (128, 192, 256, 384, 512)
    nn = int(sizes[rng.integers(0, len(sizes))])
    a, b = rng.uniform(0.05, 0.15, size=2)
    ang = rng.uniform(0.0, math.pi)
    mach = rng.uniform(1.5, 3.0)
    if n is not None:
        nn = n
    lo, hi = (0.0, 0.0), (1.0, 1.0)
    X, Y, _ = cell_centres((nn, nn), lo, hi)
    dx = 1.0 / nn
    w, L = _empty_prim(2, 1, False, nn * nn)
    rho1, p1 = 1.225, 1.0e5
    rho2, u2, p2 = ideal_shock_state(mach, 1.4, rho1, p1)
    post = X < 0.2
    w[L["irho"]] = np.where(post, rho2, rho1)
    w[L["iu"]] = np.where(post, u2, 0.0)
    w[L["ip"]] = np.where(post, p2, p1)
    ca, sa = math.cos(ang), math.sin(ang)
    xr = (X - 0.5) * ca + (Y - 0.5) * sa
    yr = -(X - 0.5) * sa + (Y - 0.5) * ca
    F = np.sqrt((xr / a) ** 2 + (yr / b) ** 2)
    gx, gy = xr / (a * a * np.maximum(F, 1e-30)), yr / (b * b * np.maximum(F, 1e-30))
    sd = (F - 1.0) / np.maximum(np.hypot(gx, gy), 1e-30)
    w[L["ir"]] = rigid_profile(sd, dx)
    return Workload("ellipse_%d_%d" % (i, nn), 2, (nn, nn), lo, hi, (0, 0), [AIR], False, w,
                    cfl=0.8, steps=300)


def batch_sizes(count: int = 256) -> List[int]:
    """Grid sizes of the batched workload's instances (cheap: no fields)."""
    out = []
    sizes = (128, 192, 256, 384, 512)
    for i in range(count):
        rng = np.random.Generator(np.random.PCG64(SEED_BASE * 1000 + i))
        out.append(int(sizes[rng.integers(0, len(sizes))]))
    return out


def sphere_3d(n: int = 256, mach: float = 2.5) -> Workload:
    """3-D Mach 2.5 air shock at x = 0.2 over a static rigid sphere of radius
    0.1 at the centre of [0,1]^3."""
    lo, hi = (0.0, 0.0, 0.0), (1.0, 1.0, 1.0)
    X, Y, Z = cell_centres((n, n, n), lo, hi)
    dx = 1.0 / n
    w, L = _empty_prim(3, 1, False, n ** 3)
    rho1, p1 = 1.225, 1.0e5
    rho2, u2, p2 = ideal_shock_state(mach, 1.4, rho1, p1)
    post = X < 0.2
    w[L["irho"]] = np.where(post, rho2, rho1)
    w[L["iu"]] = np.where(post, u2, 0.0)
    w[L["ip"]] = np.where(post, p2, p1)
    sd = np.sqrt((X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2) - 0.1
    w[L["ir"]] = rigid_profile(sd, dx)
    return Workload("sphere_3d_%d" % n, 3, (n, n, n), lo, hi, (0, 0, 0), [AIR], False, w,
                    cfl=0.8, steps=200)


def random_state(dim, n, nmat, solid, seed, periodic=None, body=True, amp=0.1):
    """Smooth-plus-noise random state for parity tests: every primitive is
    perturbed so that every branch of the update is exercised (interfaces in
    phi and r, shear in V, non-zero velocities)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = tuple(n)
    lo = tuple(0.0 for _ in range(dim))
    hi = tuple(1.0 * (n[d] / n[0]) for d in range(dim))
    X, Y, Z = cell_centres(n, lo, hi)
    nc = int(np.prod(n))
    w, L = _empty_prim(dim, nmat, solid, nc)
    mats = [AIR] if nmat == 1 else ([ALUMINIUM, AIR] if solid else [AIR, WATER])
    if nmat == 1 and solid:
        mats = [ALUMINIUM]
    if nmat == 3:
        mats = [ALUMINIUM, WATER, AIR] if solid else [WATER, HELIUM, AIR]
    if nmat == 2:
        blob = np.hypot(X - 0.4, Y - 0.5) < 0.25
        w[L["iphi"]] = np.where(blob, 1.0 - PHI_PURE, PHI_PURE)
        w[L["iphi"]] = np.clip(w[L["iphi"]] + 0.02 * rng.standard_normal(nc) * (
            (w[L["iphi"]] > 0.5) - 0.5), PHI_PURE, 1.0 - PHI_PURE)
    if nmat == 3:
        # two blobs (materials 1 and 2) in the third
        b1 = np.hypot(X - 0.35, Y - 0.45) < 0.2
        b2 = (np.hypot(X - 0.7, Y - 0.6) < 0.18) & ~b1 if dim > 1 else (np.abs(X - 0.75) < 0.1)
        f1 = np.where(b1, 1.0 - 2 * PHI_PURE, PHI_PURE)
        f2 = np.where(b2, 1.0 - 2 * PHI_PURE, PHI_PURE)
        f1 = np.clip(f1 + 0.01 * rng.standard_normal(nc) * (f1 > 0.5), PHI_PURE, 1.0 - 2 * PHI_PURE)
        w[L["iphi"]] = f1
        w[L["iphi"] + 1] = np.where(b1, PHI_PURE, f2)
    for l, m in enumerate(mats):
        base = {"ideal": 1.2, "stiffened": 1000.0, "romenskii": m.get("rho0", 1.0)}[m["kind"]]
        w[L["irho"] + l] = base * (1.0 + amp * 0.5 * rng.standard_normal(nc) * 0.2 + amp * np.sin(2 * np.pi * X))
    cs = 400.0 if not solid else 2000.0
    for a in range(dim):
        w[L["iu"] + a] = cs * amp * (np.sin(2 * np.pi * (X + 0.3 * a)) + 0.3 * rng.standard_normal(nc))
    w[L["ip"]] = 1.0e5 * (1.0 + amp * (np.cos(2 * np.pi * Y) + 0.5 * rng.standard_normal(nc) * 0.3))
    if solid:
        for c in range(L["nv"]):
            w[L["iv"] + c] += 0.01 * rng.standard_normal(nc)
    if body:
        sd = np.hypot(X - 0.6, Y - 0.45) - 0.2 if dim > 1 else (0.7 - X)
        if dim == 3:
            sd = np.sqrt((X - 0.6) ** 2 + (Y - 0.45) ** 2 + (Z - 0.5) ** 2) - 0.2
        dx = min((hi[d] - lo[d]) / n[d] for d in range(dim))
        w[L["ir"]] = rigid_profile(sd, dx)
    per = tuple(periodic) if periodic is not None else tuple(0 for _ in range(dim))
    return Workload("random_%dd" % dim, dim, n, lo, hi, per, mats, solid, w)


def with_history(wl: Workload, seed: Optional[int] = None, amp: float = 0.0) -> Workload:
    """The same workload carrying one equivalent-plastic-strain plane per
    material after r: zero, or uniform random in [0, amp) with `seed`."""
    assert wl.solid
    extra = np.zeros((wl.nmat, wl.ncell))
    if seed is not None and amp > 0.0:
        rng = np.random.Generator(np.random.PCG64(seed))
        extra = amp * rng.random((wl.nmat, wl.ncell))
    prim = np.concatenate([wl.prim, extra], axis=0)
    return dataclasses.replace(wl, prim=prim, history=True, name=wl.name + "_history")


def material_params(m: dict) -> tuple:
    """(kind_code, gamma, pinf, rho0, K0, G0, alpha, beta, Gamma0, sigY)."""
    kind = {"ideal": 0, "stiffened": 1, "romenskii": 2}[m["kind"]]
    return (kind, m.get("gamma", 0.0), m.get("pinf", 0.0), m.get("rho0", 0.0), m.get("K0", 0.0),
            m.get("G0", 0.0), m.get("alpha", 0.0), m.get("beta", 0.0), m.get("Gamma0", 0.0),
            m.get("sigY", 0.0))
