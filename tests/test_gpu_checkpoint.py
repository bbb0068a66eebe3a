"""Checkpoint and resume through the C ABI: the conserved state saved with
dfv_get_fields(DFV_FIELDS_CONSERVED) and the body state saved with
dfv_get_body, restored into a fresh grid with dfv_set_state and dfv_set_body,
continue the run bit for bit (FP64 stored as it is, FP32 narrowed back from
its exact FP64 widening), in every stage-kernel form."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

B = pytest.importorskip("paper_2111_11806_gb300.binding")

CASES = [
    ("cylinder_64_fp32", lambda: W.cylinder_2d(64), B.DFV_FP32),                 # 2-D gas kernel
    ("dynamic_body_128x64_fp64", lambda: W.dynamic_body_2d(128, 64), B.DFV_FP64),   # moving body
    ("dynamic_body_128x64_fp32", lambda: W.dynamic_body_2d(128, 64), B.DFV_FP32),
    ("impact_96_fp32", lambda: W.impact_2d(96), B.DFV_FP32),                     # solids, plastic update
    ("sphere_3d_36x20x18_fp32", lambda: W.random_state(3, (36, 20, 18), 1, False, seed=15), B.DFV_FP32),
]


@pytest.mark.parametrize("name,make,prec", CASES, ids=[c[0] for c in CASES])
def test_resume_continues_bit_for_bit(name, make, prec):
    wl = make()
    a = B.Grid.from_workload(wl, precision=prec)
    dts = []
    for k in range(20):
        dt = a.compute_dt(wl.cfl)
        dts.append(dt)
        a.step(dt)
        if k == 9:
            saved = a.cons()
            _, v, x = a.body()
    b = B.Grid.from_workload(wl, precision=prec)
    b.set_state(saved)
    b.set_body(v, x, wl.body_mass, wl.body_dynamic)
    for dt in dts[10:]:
        b.step(dt)
    np.testing.assert_array_equal(b.cons(), a.cons())
    for p, q in zip(b.body(), a.body()):
        np.testing.assert_array_equal(p, q)


def test_device_driven_resume():
    """dfv_run for 10 steps, checkpoint, 10 more in a fresh grid: the same bits
    as 20 uninterrupted device-driven steps (the restored grid computes its
    first time step from the restored state)."""
    wl = W.cylinder_2d(80, ny=72)
    a = B.Grid.from_workload(wl, precision=B.DFV_FP64)
    a.run(10, 0.8)
    saved = a.cons()
    a.run(10, 0.8)
    b = B.Grid.from_workload(wl, precision=B.DFV_FP64)
    b.set_state(saved)
    b.run(10, 0.8)
    np.testing.assert_array_equal(b.cons(), a.cons())


def test_set_state_refuses_null():
    g = B.Grid.from_workload(W.cylinder_2d(32), precision=B.DFV_FP64)
    with pytest.raises(B.DfvError):
        B._check(B.load().dfv_set_state(g._h, None, 0), g._h, "dfv_set_state")
