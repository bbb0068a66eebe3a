"""The batched form: independent 2-D instances of different sizes (own body,
own Mach number, own time step) advanced by persistent launches over a work
list.  Each instance must evolve exactly as the single-grid path does for the
same instance (same tile code, same per-instance dt), under every schedule;
FP64 instances match the oracle."""
import numpy as np
import pytest

import workloads as W
from gpu_util import rel_l1, same_kernel_bits

pytestmark = pytest.mark.gpu

B = pytest.importorskip("paper_2111_11806_gb300.binding")

SIZES = [40, 64, 97, 33, 128, 72]



def instances():
    return [W.ellipse_instance(i, n=n) for i, n in enumerate(SIZES)]


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32"])
def test_batch_instances_equal_single_grids(precision):
    wls = instances()
    b = B.Batch(wls, precision=precision)
    b.set_all_fields()
    steps = 6
    b.run(steps, 0.8)
    for i, wl in enumerate(wls):
        g = B.Grid.from_workload(wl, precision=precision)
        t = g.run(steps, 0.8)
        same_kernel_bits(b.get_fields(i), g.cons(), wl, precision)
        tb, _ = b.time(i)
        assert tb == pytest.approx(t, rel=1e-13 if precision == 0 else 1e-6)


@pytest.mark.parametrize("schedule", [0, 1, 2])
@pytest.mark.parametrize("ctas", [0, 1, 2])
def test_batch_schedules_are_equivalent(schedule, ctas):
    wls = instances()
    ref = B.Batch(wls, precision=B.DFV_FP32)
    ref.set_all_fields()
    ref.run(4, 0.8)
    b = B.Batch(wls, precision=B.DFV_FP32)
    b.set_all_fields()
    b.set_schedule(ctas, schedule)
    b.run(4, 0.8)
    for i in range(len(wls)):
        np.testing.assert_array_equal(b.get_fields(i), ref.get_fields(i))


def test_batch_fp64_matches_oracle_with_per_instance_dt():
    from oracle import Oracle
    wls = instances()[:3]
    b = B.Batch(wls, precision=B.DFV_FP64)
    b.set_all_fields()
    b.run(1, 0.8)
    dts = []
    for i, wl in enumerate(wls):
        o = Oracle.from_workload(wl)
        dt = o.compute_dt(0.8)
        dts.append(dt)
        o.step(dt)
        err = rel_l1(b.get_fields(i), o.cons(), wl)
        assert np.all(err <= 1e-12), (i, err)
        t, _ = b.time(i)
        assert t == pytest.approx(dt, rel=1e-13)
    assert len(set(np.round(dts, 15))) > 1     # the instances really step with their own dt


def test_batch_autotune_restores_state():
    wls = instances()
    b = B.Batch(wls, precision=B.DFV_FP32)
    b.set_all_fields()
    b.run(2, 0.8)
    before = [b.get_fields(i) for i in range(len(wls))]
    t_before = [b.time(i)[0] for i in range(len(wls))]
    ctas, sched = b.autotune(trial_steps=2, cfl=0.8)
    assert ctas >= 0 and sched in (0, 1, 2)
    for i in range(len(wls)):
        np.testing.assert_array_equal(b.get_fields(i), before[i])
        assert b.time(i)[0] == t_before[i]
    b.run(3, 0.8)   # the chosen schedule runs (graph path)
    ref = B.Batch(wls, precision=B.DFV_FP32)
    ref.set_all_fields()
    ref.run(5, 0.8)
    for i in range(len(wls)):
        np.testing.assert_array_equal(b.get_fields(i), ref.get_fields(i))


def test_full_size_batch_sampled_instances_match_oracle():
    """The benchmark's workload in the benchmark's launch configuration: the
    256-instance FP32 batch, autotuned, one step.  The smallest, a middle and
    the largest instance against the FP64 oracle stepped with that instance's
    own time step (relative L1 per conserved plane <= 1e-4); every instance's
    error word clear (dfv_batch_get_time raises otherwise)."""
    from oracle import Oracle
    wls = [W.ellipse_instance(i) for i in range(256)]
    b = B.Batch(wls, precision=B.DFV_FP32)
    b.set_all_fields()
    b.autotune(trial_steps=2, cfl=0.8)          # restores the state it tuned on
    b.run(1, 0.8)
    order = np.argsort([wl.ncell for wl in wls], kind="stable")
    for i in (int(order[0]), int(order[len(order) // 2]), int(order[-1])):
        t, _ = b.time(i)
        o = Oracle.from_workload(wls[i])
        o.step(t)
        err = rel_l1(b.get_fields(i), o.cons(), wls[i])
        assert np.all(err <= 1e-4), (i, wls[i].n, err)
    for i in range(len(wls)):
        b.time(i)


def test_all_instance_field_io_matches_per_instance_calls():
    """dfv_batch_set_all_fields / get_all_fields against the per-instance
    calls: the same bits; a null instance pointer is refused."""
    wls = instances()
    a = B.Batch(wls, precision=B.DFV_FP32)
    a.set_all_fields()
    a.run(3, 0.8)
    b = B.Batch(wls, precision=B.DFV_FP32)
    for i, wl in enumerate(wls):
        b.set_fields(i, wl.prim)
    b.run(3, 0.8)
    for which in (B.DFV_FIELDS_CONSERVED, B.DFV_FIELDS_PRIMITIVE):
        got = a.get_all_fields(which)
        for i in range(len(wls)):
            np.testing.assert_array_equal(got[i], b.get_fields(i, which))
    ptrs = (B._vp * len(wls))(*([None] * len(wls)))
    with pytest.raises(B.DfvError):
        B._bcheck(B.load().dfv_batch_set_all_fields(a._h, ptrs, 0), a._h, "dfv_batch_set_all_fields")


MIXTURE_SIZES = [(70, 45), (33, 64), (96, 40)]


@pytest.mark.parametrize("nmat", [2, 3])
@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32"])
def test_batch_of_mixtures_equals_single_grids(nmat, precision):
    """Two- and three-material fluid instances (blobs of water and helium in
    air around a rigid body) step in the batch exactly as single grids do."""
    wls = [W.random_state(2, n, nmat, False, seed=40 + i) for i, n in enumerate(MIXTURE_SIZES)]
    b = B.Batch(wls, precision=precision)
    b.set_all_fields()
    b.run(4, 0.6)
    for i, wl in enumerate(wls):
        g = B.Grid.from_workload(wl, precision=precision)
        g.run(4, 0.6)
        same_kernel_bits(b.get_fields(i), g.cons(), wl, precision)


def test_batch_of_three_material_mixtures_matches_oracle():
    from oracle import Oracle
    wls = [W.random_state(2, n, 3, False, seed=50 + i) for i, n in enumerate(MIXTURE_SIZES)]
    b = B.Batch(wls, precision=B.DFV_FP64)
    b.set_all_fields()
    b.run(1, 0.6)
    for i, wl in enumerate(wls):
        o = Oracle.from_workload(wl)
        o.step(o.compute_dt(0.6))
        err = rel_l1(b.get_fields(i), o.cons(), wl)
        assert np.all(err <= 1e-12), (i, err)


def test_batch_refuses_four_materials():
    wl = W.ellipse_instance(0, n=32)
    wl.materials = [W.AIR] * 4
    with pytest.raises(B.DfvError):
        B.Batch([wl], precision=B.DFV_FP32)


def test_page_locked_host_fields_match_pageable():
    """Fields in page-locked host memory are converted in place (no staging
    copy); the bits in and out are those of the pageable-memory path."""
    import torch
    wls = instances()
    pin_in = [torch.empty(wl.prim.shape, dtype=torch.float64, pin_memory=True) for wl in wls]
    for h, wl in zip(pin_in, wls):
        h.numpy()[:] = wl.prim
    a = B.Batch(wls, precision=B.DFV_FP32)
    a.set_all_fields([h.numpy() for h in pin_in])
    a.run(3, 0.8)
    b = B.Batch(wls, precision=B.DFV_FP32)
    b.set_all_fields([wl.prim.copy() for wl in wls])
    b.run(3, 0.8)
    for which in (B.DFV_FIELDS_CONSERVED, B.DFV_FIELDS_PRIMITIVE):
        pin_out = [torch.empty(wl.prim.shape, dtype=torch.float64, pin_memory=True) for wl in wls]
        pin_out[0].numpy()[:] = np.nan
        a.get_all_fields(which, outs=[h.numpy() for h in pin_out])
        ref = b.get_all_fields(which)
        for i in range(len(wls)):
            np.testing.assert_array_equal(pin_out[i].numpy(), ref[i])
            np.testing.assert_array_equal(a.get_fields(i, which), ref[i])
