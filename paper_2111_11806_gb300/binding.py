"""ctypes binding of libdfvrb.so (include/dfvrb.h): the same entry points,
argument marshalling only.  PyTorch supplies the device workspace and the
CUDA stream; every step of the solver runs in the library's kernels.  There is
no CPU fallback: without the built library or a CUDA device the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdfvrb.so")

DFV_OK = 0
DFV_ERR = {-1: "DFV_ERR_ARG", -2: "DFV_ERR_CUDA", -3: "DFV_ERR_NONPHYSICAL", -4: "DFV_ERR_TIMEOUT",
           -5: "DFV_ERR_WORKSPACE", -6: "DFV_ERR_UNSUPPORTED", -7: "DFV_ERR_TOO_LARGE"}
DFV_NOALLOC_MAX_CELLS = 16 * 1024 * 1024
DFV_FP64, DFV_FP32 = 0, 1
DFV_BC_TRANSMISSIVE, DFV_BC_PERIODIC, DFV_BC_REFLECTIVE = 0, 1, 2
DFV_FIELDS_CONSERVED, DFV_FIELDS_PRIMITIVE = 0, 1
MAT_KIND = {"ideal": 0, "stiffened": 1, "romenskii": 2}

EXPORTS = ("dfv_workspace_bytes", "dfv_create_grid", "dfv_add_material", "dfv_set_fields", "dfv_get_fields",
           "dfv_set_body", "dfv_get_body", "dfv_compute_dt", "dfv_step", "dfv_run", "dfv_check",
           "dfv_profile", "dfv_launch_count", "dfv_state_layout", "dfv_destroy", "dfv_last_error",
           "dfv_compute_dt_noalloc",
           "dfv_batch_workspace_bytes", "dfv_batch_create", "dfv_batch_add_material", "dfv_batch_set_fields",
           "dfv_batch_get_fields", "dfv_batch_run", "dfv_batch_autotune", "dfv_batch_set_schedule",
           "dfv_batch_get_time", "dfv_batch_profile", "dfv_batch_launch_count", "dfv_batch_destroy",
           "dfv_batch_last_error", "dfv_batch_set_all_fields", "dfv_batch_get_all_fields",
           "dfv_set_fields_pitched", "dfv_get_fields_pitched", "dfv_set_state")


class dfv_material_params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in
                ("gamma", "pinf", "rho0", "K0", "G0", "alpha", "beta", "Gamma0", "sigma_y",
                 "jc_c1", "jc_c2", "jc_c3", "jc_n", "jc_m", "jc_tmelt", "jc_cv")]


class dfv_options(ctypes.Structure):
    _fields_ = [("nmat", ctypes.c_int), ("solid", ctypes.c_int), ("use_thinc", ctypes.c_int),
                ("thinc_beta", ctypes.c_double), ("hllc_lm", ctypes.c_int), ("seed_variant", ctypes.c_int),
                ("normal_method", ctypes.c_int), ("probe_mode", ctypes.c_int), ("general_stage", ctypes.c_int),
                ("gas_rows", ctypes.c_int), ("seed_stages", ctypes.c_int)]


class dfv_instance_desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
                ("bc", ctypes.c_int * 6), ("v_body", ctypes.c_double * 3)]


class DfvError(RuntimeError):
    pass


_lib = None
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_vp = ctypes.c_void_p


def load(path: str = LIB_PATH):
    """Load libdfvrb.so and declare the prototypes of include/dfvrb.h."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise DfvError("libdfvrb.so is not built (%s); run __graft_entry__.build()" % path)
    L = ctypes.CDLL(path)
    L.dfv_workspace_bytes.argtypes = [ctypes.c_int, _ip, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      ctypes.POINTER(ctypes.c_size_t)]
    L.dfv_create_grid.argtypes = [ctypes.c_int, _ip, _dp, _dp, _ip, ctypes.c_int, ctypes.POINTER(dfv_options),
                                  _vp, ctypes.c_size_t, _vp, ctypes.POINTER(_vp)]
    L.dfv_add_material.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(dfv_material_params), _ip]
    L.dfv_set_fields.argtypes = [_vp, _vp, ctypes.c_int]
    L.dfv_get_fields.argtypes = [_vp, _vp, ctypes.c_int, ctypes.c_int]
    L.dfv_set_fields_pitched.argtypes = [_vp, _vp, ctypes.c_longlong, ctypes.c_int]
    L.dfv_set_state.argtypes = [_vp, _vp, ctypes.c_int]
    L.dfv_get_fields_pitched.argtypes = [_vp, _vp, ctypes.c_longlong, ctypes.c_int, ctypes.c_int]
    L.dfv_set_body.argtypes = [_vp, _dp, _dp, ctypes.c_double, ctypes.c_int]
    L.dfv_get_body.argtypes = [_vp, _dp, _dp, _dp]
    L.dfv_compute_dt.argtypes = [_vp, ctypes.c_double, _dp]
    L.dfv_step.argtypes = [_vp, ctypes.c_double]
    L.dfv_run.argtypes = [_vp, ctypes.c_int, ctypes.c_double, ctypes.c_double, _dp]
    L.dfv_check.argtypes = [_vp, ctypes.c_int]
    L.dfv_profile.argtypes = [_vp, ctypes.c_int, _dp, ctypes.POINTER(ctypes.c_longlong)]
    L.dfv_launch_count.argtypes = [_vp, ctypes.POINTER(ctypes.c_longlong)]
    L.dfv_state_layout.argtypes = [_vp, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_longlong), _ip, _ip]
    L.dfv_destroy.argtypes = [_vp]
    _bp = ctypes.POINTER(dfv_instance_desc)
    L.dfv_batch_workspace_bytes.argtypes = [ctypes.c_int, ctypes.c_int, _bp, ctypes.c_int, ctypes.POINTER(dfv_options),
                                            ctypes.POINTER(ctypes.c_size_t)]
    L.dfv_batch_create.argtypes = [ctypes.c_int, ctypes.c_int, _bp, ctypes.c_int, ctypes.POINTER(dfv_options), _vp,
                                   ctypes.c_size_t, _vp, ctypes.POINTER(_vp)]
    L.dfv_batch_add_material.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(dfv_material_params)]
    L.dfv_batch_set_fields.argtypes = [_vp, ctypes.c_int, _vp, ctypes.c_int]
    L.dfv_batch_get_fields.argtypes = [_vp, ctypes.c_int, _vp, ctypes.c_int, ctypes.c_int]
    L.dfv_batch_set_all_fields.argtypes = [_vp, ctypes.POINTER(_vp), ctypes.c_int]
    L.dfv_batch_get_all_fields.argtypes = [_vp, ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_int]
    L.dfv_batch_run.argtypes = [_vp, ctypes.c_int, ctypes.c_double, ctypes.c_double]
    L.dfv_batch_autotune.argtypes = [_vp, ctypes.c_int, ctypes.c_double, _ip]
    L.dfv_batch_set_schedule.argtypes = [_vp, ctypes.c_int, ctypes.c_int]
    L.dfv_batch_get_time.argtypes = [_vp, ctypes.c_int, _dp, _dp]
    L.dfv_batch_profile.argtypes = [_vp, ctypes.c_int, _dp, ctypes.POINTER(ctypes.c_longlong)]
    L.dfv_batch_launch_count.argtypes = [_vp, ctypes.POINTER(ctypes.c_longlong)]
    L.dfv_batch_destroy.argtypes = [_vp]
    L.dfv_batch_last_error.argtypes = [_vp]
    L.dfv_batch_last_error.restype = ctypes.c_char_p
    L.dfv_compute_dt_noalloc.argtypes = [ctypes.c_int, _ip, _dp, _dp, ctypes.c_int, ctypes.POINTER(dfv_options),
                                         _ip, ctypes.POINTER(dfv_material_params), _vp, ctypes.c_longlong, _dp,
                                         ctypes.c_double, _vp, _dp]
    L.dfv_last_error.argtypes = [_vp]
    L.dfv_last_error.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("dfv_last_error", "dfv_batch_last_error"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(status, handle=None, what=""):
    if status != DFV_OK:
        msg = ""
        if handle:
            m = load().dfv_last_error(handle)
            msg = m.decode() if m else ""
        raise DfvError("%s: %s %s" % (what, DFV_ERR.get(status, status), msg))


def _d3(x):
    a = np.zeros(3)
    a[: len(x)] = x
    return a


def material_struct(m: dict) -> dfv_material_params:
    p = dfv_material_params()
    p.gamma = m.get("gamma", 0.0)
    p.pinf = m.get("pinf", 0.0)
    p.rho0 = m.get("rho0", 0.0)
    p.K0 = m.get("K0", 0.0)
    p.G0 = m.get("G0", 0.0)
    p.alpha = m.get("alpha", 0.0)
    p.beta = m.get("beta", 0.0)
    p.Gamma0 = m.get("Gamma0", 0.0)
    p.sigma_y = m.get("sigY", 0.0)
    for k in ("jc_c1", "jc_c2", "jc_c3", "jc_n", "jc_m", "jc_tmelt", "jc_cv"):
        setattr(p, k, m.get(k, 0.0))
    return p


def workspace_bytes(dim, n, nmat, solid, precision) -> int:
    n3 = (ctypes.c_int * 3)(*(list(n) + [1] * (3 - len(n))))
    out = ctypes.c_size_t()
    _check(load().dfv_workspace_bytes(dim, n3, nmat, 2 if solid == 2 else int(bool(solid)), precision, ctypes.byref(out)),
           what="dfv_workspace_bytes")
    return out.value


def compute_dt_noalloc(dim, n, lo, hi, materials, cons_ptr, plane_pitch, cfl, precision=DFV_FP64, solid=False,
                       v_body=(0.0, 0.0, 0.0), stream=0, use_thinc=True, thinc_beta=1.6, hllc_lm=False,
                       seed_variant=0, normal_method=0, probe_mode=0):
    """dfv_compute_dt_noalloc: the CFL dt of a conserved state the caller
    holds on the device (cons_ptr: device address of the planes, plane_pitch
    elements apart), computed with the library's fixed scratch array instead
    of an allocated workspace -- for callers that cannot allocate device
    memory.  Calls that overlap on the GPU share that scratch and race."""
    L = load()
    n3 = (ctypes.c_int * 3)(*(list(n) + [1] * (3 - dim)))
    lo3, hi3 = _d3(lo), _d3(hi)
    opt = dfv_options(len(materials), int(bool(solid)), int(bool(use_thinc)), float(thinc_beta), int(bool(hllc_lm)),
                      int(seed_variant), int(normal_method), int(probe_mode))
    kinds = (ctypes.c_int * len(materials))(*[MAT_KIND[m["kind"]] for m in materials])
    params = (dfv_material_params * len(materials))(*[material_struct(m) for m in materials])
    vb = _d3(v_body)
    dt = ctypes.c_double()
    _check(L.dfv_compute_dt_noalloc(dim, n3, lo3.ctypes.data_as(_dp), hi3.ctypes.data_as(_dp), precision,
                                    ctypes.byref(opt), kinds, params, _vp(cons_ptr), int(plane_pitch),
                                    vb.ctypes.data_as(_dp), float(cfl), _vp(stream), ctypes.byref(dt)),
           None, "dfv_compute_dt_noalloc")
    return dt.value


def bc_codes(dim, periodic=None, walls=None):
    """bc[6] of dfv_create_grid: periodic directions, else a reflective wall
    where walls[2d + side] is set, else transmissive."""
    per = list(periodic or [0] * dim)
    wal = list(walls or [0] * 6)
    out = [DFV_BC_TRANSMISSIVE] * 6
    for d in range(dim):
        for side in range(2):
            if per[d]:
                out[2 * d + side] = DFV_BC_PERIODIC
            elif wal[2 * d + side]:
                out[2 * d + side] = DFV_BC_REFLECTIVE
    return out


class Grid:
    """One grid of the CUDA library.  Device memory: one torch uint8 tensor
    (the workspace), owned by this object.  Stream: torch's current stream on
    `device` unless one is given."""

    def __init__(self, dim, n, lo, hi, materials, solid=False, precision=DFV_FP64, periodic=None,
                 use_thinc=True, thinc_beta=1.6, hllc_lm=False, seed_variant=0, normal_method=0, probe_mode=0,
                 walls=None, device="cuda:0", stream=None, general_stage=False, workspace=None, gas_rows=0,
                 seed_stages=False):
        import torch
        if not torch.cuda.is_available():
            raise DfvError("a CUDA device is required (no CPU fallback)")
        L = load()
        self.torch = torch
        self.device = torch.device(device)
        self.dim = dim
        self.n = tuple(int(x) for x in n)
        self.nmat = len(materials)
        self.solid = bool(solid)
        self.history = solid == 2          # solid with plastic-strain planes
        self.precision = precision
        self.ncell = int(np.prod(self.n))
        skind = 2 if self.history else int(self.solid)
        nbytes = workspace_bytes(dim, self.n, self.nmat, skind, precision)
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            if workspace is None:
                self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
            else:
                # a caller-owned uint8 device tensor of at least nbytes + 256 bytes
                assert workspace.dtype == torch.uint8 and workspace.is_cuda and workspace.numel() >= nbytes + 256
                self.workspace = workspace
        self.workspace_bytes = nbytes
        base = self.workspace.data_ptr()
        aligned = (base + 255) & ~255
        bc = (ctypes.c_int * 6)(*bc_codes(dim, periodic, walls))
        n3 = (ctypes.c_int * 3)(*(list(self.n) + [1] * (3 - dim)))
        lo3 = _d3(lo)
        hi3 = _d3(hi)
        opt = dfv_options(self.nmat, skind, int(bool(use_thinc)), float(thinc_beta), int(bool(hllc_lm)),
                          int(seed_variant), int(normal_method), int(probe_mode), int(bool(general_stage)),
                          int(gas_rows), int(bool(seed_stages)))
        h = _vp()
        with torch.cuda.device(self.device):
            st = L.dfv_create_grid(dim, n3, lo3.ctypes.data_as(_dp), hi3.ctypes.data_as(_dp), bc, precision,
                                   ctypes.byref(opt), _vp(aligned), nbytes, _vp(self.stream.cuda_stream),
                                   ctypes.byref(h))
        _check(st, None, "dfv_create_grid")
        self._h = h
        for m in materials:
            p = material_struct(m)
            _check(L.dfv_add_material(self._h, MAT_KIND[m["kind"]], ctypes.byref(p), None), self._h,
                   "dfv_add_material")
        self.nvar = (self.nmat - 1) + self.nmat + dim + 1 + ((3 if dim == 1 else 5 if dim == 2 else 9)
                                                            if solid else 0) + 1 + (self.nmat if self.history else 0)

    @classmethod
    def from_workload(cls, wl, precision=DFV_FP64, **kw):
        solid = 2 if (wl.solid and getattr(wl, "history", False)) else wl.solid
        g = cls(wl.dim, wl.n, wl.lo, wl.hi, wl.materials, solid=solid, precision=precision,
                periodic=wl.periodic, walls=getattr(wl, "walls", None), **kw)
        g.set_fields(wl.prim)
        g.set_body(wl.body_v, wl.body_x, wl.body_mass, wl.body_dynamic)
        return g

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            try:
                self.stream.synchronize()
            except Exception:
                pass
            load().dfv_destroy(h)
            self._h = None

    def _ctx(self):
        return self.torch.cuda.device(self.device)

    # ---- fields
    def set_fields(self, prim):
        """prim: numpy (host) or torch cuda float64 array of shape (nvar, ncell)."""
        if hasattr(prim, "is_cuda") and prim.is_cuda:
            t = prim.contiguous()
            assert t.dtype == self.torch.float64 and t.numel() == self.nvar * self.ncell
            with self._ctx():
                _check(load().dfv_set_fields(self._h, _vp(t.data_ptr()), 1), self._h, "dfv_set_fields")
            self._keep = t
            return
        a = np.ascontiguousarray(np.asarray(prim, dtype=np.float64)).reshape(self.nvar, self.ncell)
        with self._ctx():
            _check(load().dfv_set_fields(self._h, _vp(a.ctypes.data), 0), self._h, "dfv_set_fields")

    def set_state(self, cons):
        """Restore FP64 conserved planes (nvar, ncell) saved with cons() (checkpoint/resume)."""
        a = np.ascontiguousarray(np.asarray(cons, dtype=np.float64)).reshape(self.nvar, self.ncell)
        with self._ctx():
            _check(load().dfv_set_state(self._h, _vp(a.ctypes.data), 0), self._h, "dfv_set_state")

    def set_fields_pitched(self, prim):
        """prim: a host float64 array of shape (nvar, pitch), pitch >= ncell (a
        padded buffer; columns ncell .. pitch-1 of each plane are not read)."""
        a = np.asarray(prim, dtype=np.float64)
        assert a.ndim == 2 and a.shape[0] == self.nvar and a.flags.c_contiguous
        with self._ctx():
            _check(load().dfv_set_fields_pitched(self._h, _vp(a.ctypes.data), int(a.shape[1]), 0), self._h,
                   "dfv_set_fields_pitched")

    def get_fields_pitched(self, out, which=DFV_FIELDS_CONSERVED):
        """Into a host float64 array of shape (nvar, pitch), pitch >= ncell."""
        assert out.dtype == np.float64 and out.ndim == 2 and out.shape[0] == self.nvar and out.flags.c_contiguous
        with self._ctx():
            _check(load().dfv_get_fields_pitched(self._h, _vp(out.ctypes.data), int(out.shape[1]), which, 0),
                   self._h, "dfv_get_fields_pitched")
        return out

    def get_fields(self, which=DFV_FIELDS_CONSERVED, out=None):
        if out is not None and hasattr(out, "is_cuda") and out.is_cuda:
            with self._ctx():
                _check(load().dfv_get_fields(self._h, _vp(out.data_ptr()), which, 1), self._h, "dfv_get_fields")
            return out
        a = np.zeros((self.nvar, self.ncell)) if out is None else out
        with self._ctx():
            _check(load().dfv_get_fields(self._h, _vp(a.ctypes.data), which, 0), self._h, "dfv_get_fields")
        return a

    def cons(self):
        return self.get_fields(DFV_FIELDS_CONSERVED)

    def prim(self):
        return self.get_fields(DFV_FIELDS_PRIMITIVE)

    # ---- body
    def set_body(self, v=(0, 0, 0), x=(0, 0, 0), mass=0.0, dynamic=False):
        with self._ctx():
            _check(load().dfv_set_body(self._h, _d3(v).ctypes.data_as(_dp), _d3(x).ctypes.data_as(_dp),
                                       float(mass), int(bool(dynamic))), self._h, "dfv_set_body")

    def body(self):
        f, v, x = np.zeros(3), np.zeros(3), np.zeros(3)
        with self._ctx():
            _check(load().dfv_get_body(self._h, f.ctypes.data_as(_dp), v.ctypes.data_as(_dp),
                                       x.ctypes.data_as(_dp)), self._h, "dfv_get_body")
        return f, v, x

    # ---- time stepping
    def compute_dt(self, cfl):
        dt = ctypes.c_double()
        with self._ctx():
            _check(load().dfv_compute_dt(self._h, float(cfl), ctypes.byref(dt)), self._h, "dfv_compute_dt")
        return dt.value

    def step(self, dt):
        with self._ctx():
            _check(load().dfv_step(self._h, float(dt)), self._h, "dfv_step")

    def run(self, steps, cfl, t_end=0.0, sync=True):
        t = ctypes.c_double()
        with self._ctx():
            _check(load().dfv_run(self._h, int(steps), float(cfl), float(t_end or 0.0),
                                  ctypes.byref(t) if sync else None), self._h, "dfv_run")
        return t.value if sync else None

    def check(self, timeout_ms=0):
        with self._ctx():
            _check(load().dfv_check(self._h, int(timeout_ms)), self._h, "dfv_check")

    def profile(self, enable):
        """Start (enable=True) or stop per-kernel event timing; returns
        (ms[seed, stage1, stage2, stage3, finalize], steps) recorded so far."""
        ms = np.zeros(5)
        n = ctypes.c_longlong()
        with self._ctx():
            _check(load().dfv_profile(self._h, int(bool(enable)), ms.ctypes.data_as(_dp), ctypes.byref(n)),
                   self._h, "dfv_profile")
        return ms, n.value

    def launch_count(self):
        c = ctypes.c_longlong()
        _check(load().dfv_launch_count(self._h, ctypes.byref(c)), self._h, "dfv_launch_count")
        return c.value

    def state_layout(self):
        """(byte offsets of U^n, U1, U3 from the workspace's aligned base,
        plane pitch in elements, planes, bytes per element)."""
        off = (ctypes.c_size_t * 3)()
        pitch, nvar, eb = ctypes.c_longlong(), ctypes.c_int(), ctypes.c_int()
        _check(load().dfv_state_layout(self._h, off, ctypes.byref(pitch), ctypes.byref(nvar), ctypes.byref(eb)),
               self._h, "dfv_state_layout")
        return tuple(off), pitch.value, nvar.value, eb.value

    def aligned_offset(self):
        """Offset of the library's 256-byte aligned workspace base in self.workspace."""
        base = self.workspace.data_ptr()
        return ((base + 255) & ~255) - base


def _bcheck(status, handle, what):
    if status != DFV_OK:
        m = load().dfv_batch_last_error(handle) if handle else b""
        raise DfvError("%s: %s %s" % (what, DFV_ERR.get(status, status), m.decode() if m else ""))


class Batch:
    """A batch of independent 2-D instances (dfv_batch_*): each workload in
    `workloads` (same materials, fluid, 2-D) becomes one instance with its own
    grid, body velocity and time step.  Device memory: one torch workspace."""

    def __init__(self, workloads, precision=DFV_FP32, use_thinc=True, thinc_beta=1.6, hllc_lm=False, seed_variant=0,
                 normal_method=0, probe_mode=0, device="cuda:0", stream=None, general_stage=False, gas_rows=0,
                 seed_stages=False):
        import torch
        if not torch.cuda.is_available():
            raise DfvError("a CUDA device is required (no CPU fallback)")
        L = load()
        self.torch = torch
        self.device = torch.device(device)
        self.wls = list(workloads)
        self.count = len(self.wls)
        mats = self.wls[0].materials
        self.nmat = len(mats)
        self.precision = precision
        descs = (dfv_instance_desc * self.count)()
        for i, wl in enumerate(self.wls):
            assert wl.dim == 2 and not wl.solid and len(wl.materials) == self.nmat
            d = descs[i]
            for k in range(2):
                d.n[k] = wl.n[k]
                d.lo[k] = wl.lo[k]
                d.hi[k] = wl.hi[k]
            codes = bc_codes(2, wl.periodic, getattr(wl, "walls", None))
            for k in range(4):
                d.bc[k] = codes[k]
            d.n[2] = 1
            for k in range(3):
                d.v_body[k] = wl.body_v[k] if k < len(wl.body_v) else 0.0
        self._descs = descs
        opt = dfv_options(self.nmat, 0, int(bool(use_thinc)), float(thinc_beta), int(bool(hllc_lm)), int(seed_variant),
                          int(normal_method), int(probe_mode), int(bool(general_stage)), int(gas_rows),
                          int(bool(seed_stages)))
        nbytes = ctypes.c_size_t()
        _check(L.dfv_batch_workspace_bytes(2, self.count, descs, precision, ctypes.byref(opt), ctypes.byref(nbytes)),
               None, "dfv_batch_workspace_bytes")
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            self.workspace = torch.empty(nbytes.value + 256, dtype=torch.uint8, device=self.device)
        aligned = (self.workspace.data_ptr() + 255) & ~255
        h = _vp()
        with torch.cuda.device(self.device):
            _check(L.dfv_batch_create(2, self.count, descs, precision, ctypes.byref(opt), _vp(aligned),
                                      nbytes.value, _vp(self.stream.cuda_stream), ctypes.byref(h)),
                   None, "dfv_batch_create")
        self._h = h
        for m in mats:
            _bcheck(L.dfv_batch_add_material(self._h, MAT_KIND[m["kind"]], ctypes.byref(material_struct(m))),
                    self._h, "dfv_batch_add_material")
        self.cells = [int(np.prod(wl.n)) for wl in self.wls]
        self.total_cells = int(sum(self.cells))
        self.nvar = (self.nmat - 1) + self.nmat + 2 + 1 + 1

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            try:
                self.stream.synchronize()
            except Exception:
                pass
            load().dfv_batch_destroy(h)
            self._h = None

    def _ctx(self):
        return self.torch.cuda.device(self.device)

    def set_fields(self, i, prim):
        a = np.ascontiguousarray(np.asarray(prim, dtype=np.float64))
        with self._ctx():
            _bcheck(load().dfv_batch_set_fields(self._h, int(i), _vp(a.ctypes.data), 0), self._h,
                    "dfv_batch_set_fields")

    def set_all_fields(self, prims=None):
        """Every instance's primitive fields in one call (dfv_batch_set_all_fields);
        prims: one FP64 array per instance (default: the workloads' own)."""
        prims = [wl.prim for wl in self.wls] if prims is None else list(prims)
        arrs = [np.ascontiguousarray(np.asarray(p, dtype=np.float64)) for p in prims]
        assert len(arrs) == self.count
        ptrs = (_vp * self.count)(*[_vp(a.ctypes.data) for a in arrs])
        with self._ctx():
            _bcheck(load().dfv_batch_set_all_fields(self._h, ptrs, 0), self._h, "dfv_batch_set_all_fields")

    def get_all_fields(self, which=DFV_FIELDS_CONSERVED, outs=None):
        """Every instance's fields in one call (dfv_batch_get_all_fields); outs:
        one C-contiguous FP64 array of nvar x cells per instance (default: new)."""
        outs = [np.zeros((self.nvar, c)) for c in self.cells] if outs is None else list(outs)
        assert len(outs) == self.count
        for a, c in zip(outs, self.cells):
            assert a.dtype == np.float64 and a.flags.c_contiguous and a.size == self.nvar * c
        ptrs = (_vp * self.count)(*[_vp(a.ctypes.data) for a in outs])
        with self._ctx():
            _bcheck(load().dfv_batch_get_all_fields(self._h, ptrs, which, 0), self._h, "dfv_batch_get_all_fields")
        return outs

    def get_fields(self, i, which=DFV_FIELDS_CONSERVED, out=None):
        a = np.zeros((self.nvar, self.cells[i])) if out is None else out
        assert a.dtype == np.float64 and a.flags.c_contiguous and a.size == self.nvar * self.cells[i]
        with self._ctx():
            _bcheck(load().dfv_batch_get_fields(self._h, int(i), _vp(a.ctypes.data), which, 0), self._h,
                    "dfv_batch_get_fields")
        return a

    def run(self, steps, cfl, t_end=0.0):
        with self._ctx():
            _bcheck(load().dfv_batch_run(self._h, int(steps), float(cfl), float(t_end or 0.0)), self._h,
                    "dfv_batch_run")

    def autotune(self, trial_steps=3, cfl=0.8):
        c = (ctypes.c_int * 2)()
        with self._ctx():
            _bcheck(load().dfv_batch_autotune(self._h, int(trial_steps), float(cfl), c), self._h,
                    "dfv_batch_autotune")
        return int(c[0]), int(c[1])

    def set_schedule(self, ctas_per_sm, schedule):
        _bcheck(load().dfv_batch_set_schedule(self._h, int(ctas_per_sm), int(schedule)), self._h,
                "dfv_batch_set_schedule")

    def time(self, i):
        t, dt = ctypes.c_double(), ctypes.c_double()
        with self._ctx():
            _bcheck(load().dfv_batch_get_time(self._h, int(i), ctypes.byref(t), ctypes.byref(dt)), self._h,
                    "dfv_batch_get_time")
        return t.value, dt.value

    def profile(self, enable):
        ms = np.zeros(4)
        n = ctypes.c_longlong()
        with self._ctx():
            _bcheck(load().dfv_batch_profile(self._h, int(bool(enable)), ms.ctypes.data_as(_dp), ctypes.byref(n)),
                    self._h, "dfv_batch_profile")
        return ms, n.value

    def launch_count(self):
        c = ctypes.c_longlong()
        _bcheck(load().dfv_batch_launch_count(self._h, ctypes.byref(c)), self._h, "dfv_batch_launch_count")
        return c.value
