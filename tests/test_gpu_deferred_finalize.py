"""Device-driven steps of a static body leave their finalize (CFL maximum,
time, next dt, rigid box) to the seeding launch of the next step; any call
that reads or writes the control block runs it first.  These tests check that
the deferral is invisible: split runs, runs without reading the time, runs
followed by host-dt steps, body and field calls in between -- all give
bit-identical fields and times to one uninterrupted run."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

B = pytest.importorskip("paper_2111_11806_gb300.binding")


def fresh(precision=None, wl=None):
    wl = wl or W.cylinder_2d(80, ny=72)
    return B.Grid.from_workload(wl, precision=B.DFV_FP64 if precision is None else precision)


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32"])
def test_split_runs_equal_one_run(precision):
    g1 = fresh(precision)
    t1 = g1.run(12, 0.8)
    g2 = fresh(precision)
    g2.run(5, 0.8, sync=False)
    g2.run(4, 0.8, sync=False)
    t2 = g2.run(3, 0.8)
    assert t2 == t1
    np.testing.assert_array_equal(g1.cons(), g2.cons())


def test_run_then_host_steps_equal_host_loop():
    """run(6) without reading the time, then six compute_dt + step: the same
    as twelve compute_dt + step (compute_dt runs the pending finalize)."""
    g1 = fresh()
    for _ in range(12):
        g1.step(g1.compute_dt(0.8))
    g2 = fresh()
    g2.run(6, 0.8, sync=False)
    for _ in range(6):
        g2.step(g2.compute_dt(0.8))
    np.testing.assert_array_equal(g1.cons(), g2.cons())
    assert g2.run(0, 0.8) == pytest.approx(g1.run(0, 0.8), rel=0, abs=0)


def test_calls_between_runs_see_the_finalized_state():
    g1 = fresh()
    t_ref = g1.run(8, 0.8)
    f1, v1, x1 = g1.body()
    g2 = fresh()
    g2.run(4, 0.8, sync=False)
    g2.check(timeout_ms=60000)          # runs the pending finalize
    g2.run(4, 0.8, sync=False)
    f2, v2, x2 = g2.body()               # so does reading the body
    np.testing.assert_array_equal(v1, v2)
    np.testing.assert_array_equal(x1, x2)
    assert g2.run(0, 0.8) == t_ref
    np.testing.assert_array_equal(g1.cons(), g2.cons())


def test_new_cfl_and_new_fields_after_a_deferred_step():
    wl = W.cylinder_2d(64)
    g1 = fresh(wl=wl)
    g1.run(3, 0.8)
    t1 = g1.run(3, 0.5)
    g2 = fresh(wl=W.cylinder_2d(64))
    g2.run(3, 0.8, sync=False)
    t2 = g2.run(3, 0.5)                  # a new CFL number: the pending finalize runs first
    assert t2 == t1
    np.testing.assert_array_equal(g1.cons(), g2.cons())
    # new fields after a deferred step: the next run starts from them alone
    g2.run(2, 0.8, sync=False)
    g2.set_fields(W.cylinder_2d(64).prim)
    g3 = fresh(wl=W.cylinder_2d(64))
    np.testing.assert_array_equal(g2.cons(), g3.cons())
    tb = g2.run(0, 0.8)
    ta = g2.run(4, 0.8)
    assert ta - tb == pytest.approx(g3.run(4, 0.8), rel=1e-13)
    np.testing.assert_array_equal(g2.cons(), g3.cons())


def test_deferred_step_launches_four_kernels():
    g = fresh()
    g.run(2, 0.8)
    c0 = g.launch_count()
    g.run(10, 0.8, sync=False)
    # seeding (with the previous finalize), three stages
    assert g.launch_count() - c0 == 40
