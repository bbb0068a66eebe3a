"""Failure paths made on the host, without faulting the GPU:

* a host wait that runs out: a legitimate long run is enqueued and
  dfv_check is given 1 ms; it reports DFV_ERR_TIMEOUT, nothing is left
  hanging, and after draining the stream the fields equal those of an
  uninterrupted run;
* writes outside the state: the caller's workspace is filled with a canary
  byte pattern before the grid is created; after steps on small grids of odd
  sizes (every precision and dimension, the gas and general stage kernels,
  solids, walls) the padding elements of every plane of U^n, U1, U3 and the
  bytes past the workspace's end still hold the canary;
* reads outside the state: a workspace filled with 0xFF bytes (NaN in FP32
  and FP64) before creation gives the same bits as one filled with zeros, so
  that no kernel lets plane padding or workspace it has not written reach its
  arithmetic (a NaN read would spread into the fields or set the error
  word)."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

B = pytest.importorskip("paper_2111_11806_gb300.binding")

CANARY = 0xA5


def test_host_wait_times_out_then_drains():
    import torch
    wl = W.sphere_3d(160)
    g1 = B.Grid.from_workload(wl, precision=B.DFV_FP32)
    g2 = B.Grid.from_workload(wl, precision=B.DFV_FP32)
    g1.check(timeout_ms=0)
    g1.run(40, wl.cfl, sync=False)      # about 40 x 1 ms of device work, enqueued
    with pytest.raises(B.DfvError, match="TIMEOUT"):
        g1.check(timeout_ms=1)
    g1.check(timeout_ms=0)              # drain with no limit
    g2.run(40, wl.cfl)
    np.testing.assert_array_equal(g1.cons(), g2.cons())


def with_walls(wl, walls):
    wl.walls = tuple(walls)
    return wl


CASES = [
    ("1d_101_fp64", lambda: W.random_state(1, (101,), 1, False, seed=301), B.DFV_FP64, False),
    ("2d_37x29_fp32_general", lambda: W.random_state(2, (37, 29), 1, False, seed=302), B.DFV_FP32, False),
    ("2d_100x37_fp32_gas", lambda: W.random_state(2, (100, 37), 1, False, seed=303), B.DFV_FP32, False),
    ("2d_100x37_fp32_gas_walls", lambda: with_walls(W.random_state(2, (100, 37), 1, False, seed=304),
                                                    (1, 1, 1, 1)), B.DFV_FP32, False),
    ("2d_41x23_two_fluid_fp32", lambda: W.random_state(2, (41, 23), 2, False, seed=305), B.DFV_FP32, False),
    ("2d_30x21_solid_fp64", lambda: W.random_state(2, (30, 21), 2, True, seed=306, amp=0.02), B.DFV_FP64, False),
    ("3d_13x11x9_fp32", lambda: W.random_state(3, (13, 11, 9), 1, False, seed=307), B.DFV_FP32, False),
    ("3d_13x11x9_fp64", lambda: W.random_state(3, (13, 11, 9), 1, False, seed=308), B.DFV_FP64, False),
]


@pytest.mark.parametrize("name,make,prec,_", CASES, ids=[c[0] for c in CASES])
def test_no_write_outside_the_state(name, make, prec, _):
    import torch
    wl = make()
    solid = 2 if (wl.solid and getattr(wl, "history", False)) else wl.solid
    nbytes = B.workspace_bytes(wl.dim, wl.n, wl.nmat, int(bool(solid)), prec)
    tail = 65536
    ws = torch.full((nbytes + 256 + tail,), CANARY, dtype=torch.uint8, device="cuda")
    g = B.Grid(wl.dim, wl.n, wl.lo, wl.hi, wl.materials, solid=solid, precision=prec, periodic=wl.periodic,
               walls=getattr(wl, "walls", None), workspace=ws)
    g.set_fields(wl.prim)
    g.set_body(wl.body_v, wl.body_x, wl.body_mass, wl.body_dynamic)
    g.run(5, 0.6)
    for _k in range(2):
        g.step(g.compute_dt(0.6))
    g.check(timeout_ms=60000)
    base = g.aligned_offset()
    off, pitch, nvar, eb = g.state_layout()
    assert pitch >= wl.ncell and nvar == wl.nvar
    host = ws.cpu().numpy()
    for o in off:
        for v in range(nvar):
            a = base + o + (v * pitch + wl.ncell) * eb
            b = base + o + (v + 1) * pitch * eb
            assert np.all(host[a:b] == CANARY), (name, o, v)
    # past the workspace the library was given
    assert np.all(host[base + nbytes:] == CANARY)


def _run_in(ws, wl, prec, solid):
    g = B.Grid(wl.dim, wl.n, wl.lo, wl.hi, wl.materials, solid=solid, precision=prec, periodic=wl.periodic,
               walls=getattr(wl, "walls", None), workspace=ws)
    g.set_fields(wl.prim)
    g.set_body(wl.body_v, wl.body_x, wl.body_mass, wl.body_dynamic)
    g.run(5, 0.6)
    for _k in range(2):
        g.step(g.compute_dt(0.6))
    g.check(timeout_ms=60000)
    return g.cons()


@pytest.mark.parametrize("name,make,prec,_", CASES, ids=[c[0] for c in CASES])
def test_no_read_outside_the_state(name, make, prec, _):
    import torch
    wl = make()
    solid = 2 if (wl.solid and getattr(wl, "history", False)) else wl.solid
    nbytes = B.workspace_bytes(wl.dim, wl.n, wl.nmat, int(bool(solid)), prec)
    nan_ws = torch.full((nbytes + 256,), 0xFF, dtype=torch.uint8, device="cuda")
    zero_ws = torch.zeros((nbytes + 256,), dtype=torch.uint8, device="cuda")
    a = _run_in(nan_ws, wl, prec, solid)
    b = _run_in(zero_ws, wl, prec, solid)
    assert np.all(np.isfinite(a))
    np.testing.assert_array_equal(a, b)
