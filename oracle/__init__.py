"""Python handle on the plain FP64 CPU oracle (oracle.c).

TEST INFRASTRUCTURE: only tests/, the smoke check in __graft_entry__ and the
CPU-baseline leg of bench.py use this package.  It never imports the CUDA
library and the CUDA library never imports it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so with gcc (plain -O2, no FMA
    contraction so results match across x86-64 and aarch64 hosts)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            L.o_create.restype = ctypes.c_void_p
            L.o_create.argtypes = [ctypes.c_int, _ip, _dp, _dp, _ip, ctypes.c_int, ctypes.c_int]
            L.o_destroy.argtypes = [ctypes.c_void_p]
            L.o_nvar.argtypes = [ctypes.c_void_p]
            L.o_set_material.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int] + [ctypes.c_double] * 9
            L.o_set_options.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_double]
            L.o_set_variants.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
            L.o_set_walls.argtypes = [ctypes.c_void_p, _ip]
            L.o_set_seed_stages.argtypes = [ctypes.c_void_p, ctypes.c_int]
            L.o_get_stage_input.argtypes = [ctypes.c_void_p, ctypes.c_int, _dp]
            L.o_seed_normals.argtypes = [ctypes.c_void_p, _dp]
            L.o_cut_fraction.argtypes = [ctypes.c_double] * 7
            L.o_cut_fraction.restype = ctypes.c_double
            L.o_cut_alpha.argtypes = [ctypes.c_double] * 7
            L.o_cut_alpha.restype = ctypes.c_double
            L.o_elvira.argtypes = [_dp, ctypes.c_double, ctypes.c_double, _dp]
            for name in ("o_set_prim", "o_get_prim", "o_set_cons", "o_get_cons", "o_compute_D"):
                getattr(L, name).argtypes = [ctypes.c_void_p, _dp]
            L.o_set_body.argtypes = [ctypes.c_void_p, _dp, _dp, ctypes.c_double, ctypes.c_int]
            L.o_get_body.argtypes = [ctypes.c_void_p, _dp, _dp, _dp]
            L.o_compute_dt.argtypes = [ctypes.c_void_p, ctypes.c_double]
            L.o_compute_dt.restype = ctypes.c_double
            L.o_step.argtypes = [ctypes.c_void_p, ctypes.c_double]
            L.o_seed_state.argtypes = [ctypes.c_void_p]
            L.o_force_state.argtypes = [ctypes.c_void_p, _dp]
            L.o_plastic_state.argtypes = [ctypes.c_void_p, ctypes.c_double]
            L.o_cell_closure.argtypes = [ctypes.c_void_p, _dp, _dp]
            L.o_cell_prim_to_cons.argtypes = [ctypes.c_void_p, _dp, _dp]
            L.o_cell_cons_to_prim.argtypes = [ctypes.c_void_p, _dp, _dp]
            L.o_material_ref.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_double, _dp]
            L.o_riemann.argtypes = [ctypes.c_void_p, ctypes.c_int, _dp, _dp, _dp, _dp, _dp]
            L.o_plastic_cons.argtypes = [ctypes.c_void_p, _dp, ctypes.c_double]
            L.o_set_jc.argtypes = [ctypes.c_void_p, ctypes.c_int] + [ctypes.c_double] * 7
            L.o_thinc.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, _dp, _dp]
            L.o_thinc.restype = ctypes.c_int
            L.o_sym_eig3.argtypes = [_dp, _dp, _dp]
            L.o_vbar_log.argtypes = [_dp, _dp, _dp, _dp, _dp]
            L.o_polar.argtypes = [_dp, _dp, _dp]
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _arr(x, n=None):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if n is not None:
        b = np.zeros(n)
        b[: a.size] = a.ravel()
        a = b
    return a


class Oracle:
    """One grid of the oracle solver."""

    def __init__(self, dim, n, lo, hi, materials, solid=False, periodic=None):
        L = lib()
        self.dim = dim
        self.n = tuple(int(x) for x in n)
        n3 = np.array(list(self.n) + [1] * (3 - dim), dtype=np.int32)
        lo3 = _arr(lo, 3)
        hi3 = _arr(hi, 3)
        per = np.array(list(periodic or [0] * dim) + [0] * (3 - dim), dtype=np.int32)
        # solid: False / True, or 2 for a solid with plastic-strain history planes
        self._h = L.o_create(dim, n3.ctypes.data_as(_ip), _p(lo3), _p(hi3), per.ctypes.data_as(_ip),
                             len(materials), 2 if solid == 2 else int(bool(solid)))
        self.nmat = len(materials)
        self.solid = bool(solid)
        for l, m in enumerate(materials):
            self.set_material(l, m)
        self.nvar = L.o_nvar(self._h)
        self.ncell = int(np.prod(self.n))

    @classmethod
    def from_workload(cls, wl, use_thinc=True, thinc_beta=1.6, hllc_lm=False, seed_variant=0, normal_method=0,
                      probe_mode=0, seed_stages=False):
        solid = 2 if (wl.solid and getattr(wl, "history", False)) else wl.solid
        o = cls(wl.dim, wl.n, wl.lo, wl.hi, wl.materials, solid, wl.periodic)
        o.set_options(use_thinc, thinc_beta)
        o.set_variants(hllc_lm, seed_variant, normal_method, probe_mode)
        o.set_seed_stages(seed_stages)
        o.set_walls(getattr(wl, "walls", (0,) * 6))
        o.set_prim(wl.prim)
        o.set_body(wl.body_v, wl.body_x, wl.body_mass, wl.body_dynamic)
        return o

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().o_destroy(h)
            self._h = None

    def set_material(self, l, m):
        kind = {"ideal": 0, "stiffened": 1, "romenskii": 2}[m["kind"]]
        lib().o_set_material(self._h, l, kind, m.get("gamma", 0.0), m.get("pinf", 0.0), m.get("rho0", 0.0),
                             m.get("K0", 0.0), m.get("G0", 0.0), m.get("alpha", 0.0), m.get("beta", 0.0),
                             m.get("Gamma0", 0.0), m.get("sigY", 0.0))
        lib().o_set_jc(self._h, l, *[float(m.get(k, 0.0)) for k in
                                     ("jc_c1", "jc_c2", "jc_c3", "jc_n", "jc_m", "jc_tmelt", "jc_cv")])

    def set_options(self, use_thinc=True, thinc_beta=1.6):
        lib().o_set_options(self._h, int(bool(use_thinc)), float(thinc_beta))

    def set_variants(self, hllc_lm=False, seed_variant=0, normal_method=0, probe_mode=0):
        """HLLC-LM flux (True/False), seeding variant (0 original, 1 Riemann),
        normal method (0 Youngs, 1 ELVIRA in 2-D), probe (0 stepped, 1 fixed 1.5 dx)."""
        lib().o_set_variants(self._h, int(bool(hllc_lm)), int(seed_variant), int(normal_method), int(probe_mode))

    def set_seed_stages(self, on=True):
        """Seed every stage input (U1 before stage 2, U3 before stage 3) as
        well as the step-start state (on), or the step-start state only."""
        lib().o_set_seed_stages(self._h, int(bool(on)))

    def stage_input(self, k):
        """Conserved planes of the last step's input of stage k+1 (k = 1: U1,
        k = 2: U3), as that stage read them."""
        out = np.zeros((self.nvar, self.ncell))
        lib().o_get_stage_input(self._h, int(k), out.ctypes.data_as(_dp))
        return out

    def set_walls(self, walls):
        """Reflective walls: walls[2d], walls[2d+1] for the low / high side of direction d."""
        a = np.zeros(6, dtype=np.int32)
        a[: len(walls)] = [int(bool(x)) for x in walls]
        lib().o_set_walls(self._h, a.ctypes.data_as(_ip))

    def seed_normals(self):
        a = np.zeros((3, self.ncell))
        lib().o_seed_normals(self._h, _p(a))
        return a

    def set_prim(self, prim):
        a = _arr(prim).reshape(self.nvar, self.ncell)
        lib().o_set_prim(self._h, _p(a))

    def prim(self):
        a = np.zeros((self.nvar, self.ncell))
        lib().o_get_prim(self._h, _p(a))
        return a

    def set_cons(self, cons):
        a = _arr(cons).reshape(self.nvar, self.ncell)
        lib().o_set_cons(self._h, _p(a))

    def cons(self):
        a = np.zeros((self.nvar, self.ncell))
        lib().o_get_cons(self._h, _p(a))
        return a

    def set_body(self, v=(0, 0, 0), x=(0, 0, 0), mass=0.0, dynamic=False):
        lib().o_set_body(self._h, _p(_arr(v, 3)), _p(_arr(x, 3)), float(mass), int(bool(dynamic)))

    def body(self):
        f, v, x = np.zeros(3), np.zeros(3), np.zeros(3)
        lib().o_get_body(self._h, _p(f), _p(v), _p(x))
        return f, v, x

    def compute_dt(self, cfl):
        return lib().o_compute_dt(self._h, float(cfl))

    def step(self, dt):
        lib().o_step(self._h, float(dt))

    def run(self, steps, cfl, t_end=None):
        t = 0.0
        for _ in range(steps):
            dt = self.compute_dt(cfl)
            if t_end is not None and t + dt > t_end:
                dt = t_end - t
            if dt <= 0.0:
                break
            self.step(dt)
            t += dt
        return t

    def compute_D(self):
        a = np.zeros((self.nvar, self.ncell))
        lib().o_compute_D(self._h, _p(a))
        return a

    def seed(self):
        lib().o_seed_state(self._h)

    def force(self):
        f = np.zeros(3)
        lib().o_force_state(self._h, _p(f))
        return f

    def plastic(self, dt=0.0):
        """The plastic update of every cell (dt: the step, for the strain rate
        of Johnson-Cook materials; 0 = no rate term)."""
        lib().o_plastic_state(self._h, float(dt))

    # ---- single-cell / single-face pieces, for pins
    def closure(self, q):
        out = np.zeros(5)
        lib().o_cell_closure(self._h, _p(_arr(q)), _p(out))
        return dict(p=out[0], c=out[1], G=out[2], sigY=out[3], J2=out[4])

    def prim_to_cons(self, w):
        q = np.zeros(self.nvar)
        lib().o_cell_prim_to_cons(self._h, _p(_arr(w)), _p(q))
        return q

    def cons_to_prim(self, q):
        w = np.zeros(self.nvar)
        lib().o_cell_cons_to_prim(self._h, _p(_arr(q)), _p(w))
        return w

    def material_ref(self, l, rho, J2=0.0):
        out = np.zeros(6)
        lib().o_material_ref(self._h, l, float(rho), float(J2), _p(out))
        return dict(Gamma=out[0], eref=out[1], pref=out[2], deref=out[3], dpref=out[4], G=out[5])

    def riemann(self, d, wL, wR):
        F = np.zeros(self.nvar)
        us, vr = np.zeros(3), np.zeros(3)
        lib().o_riemann(self._h, d, _p(_arr(wL)), _p(_arr(wR)), _p(F), _p(us), _p(vr))
        return F, us, vr

    def plastic_cons(self, q, dt=0.0):
        a = _arr(q).copy()
        lib().o_plastic_cons(self._h, _p(a), float(dt))
        return a


def thinc(qm, q0, qp, beta=1.6):
    fm, fp = ctypes.c_double(), ctypes.c_double()
    ok = lib().o_thinc(qm, q0, qp, beta, ctypes.byref(fm), ctypes.byref(fp))
    return (fm.value, fp.value) if ok else None


def cut_fraction(n, alpha, x0, y0, hx, hy):
    """Fraction of the rectangle [x0,x0+hx]x[y0,y0+hy] on the side n.x <= alpha."""
    return lib().o_cut_fraction(float(n[0]), float(n[1]), float(alpha), float(x0), float(y0), float(hx), float(hy))


def cut_alpha(n, f, x0, y0, hx, hy):
    return lib().o_cut_alpha(float(n[0]), float(n[1]), float(f), float(x0), float(y0), float(hx), float(hy))


def elvira(block, hx=1.0, hy=1.0):
    """ELVIRA outward normal of the centre of a 3x3 block of r, block[l][k] = r(i+k-1, j+l-1)."""
    b = _arr(block).ravel().copy()
    out = np.zeros(2)
    lib().o_elvira(_p(b), float(hx), float(hy), _p(out))
    return out


def sym_eig3(B):
    lam, Q = np.zeros(3), np.zeros(9)
    lib().o_sym_eig3(_p(_arr(B).ravel().copy()), _p(lam), _p(Q))
    return lam, Q.reshape(3, 3)


def vbar_log(A):
    dH, J2, lam, Q = np.zeros(9), np.zeros(1), np.zeros(3), np.zeros(9)
    lib().o_vbar_log(_p(_arr(A).ravel().copy()), _p(dH), _p(J2), _p(lam), _p(Q))
    return dH.reshape(3, 3), J2[0]


def polar(A):
    V, R = np.zeros(9), np.zeros(9)
    lib().o_polar(_p(_arr(A).ravel().copy()), _p(V), _p(R))
    return V.reshape(3, 3), R.reshape(3, 3)
