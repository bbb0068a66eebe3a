"""GPU parity of the stage kernels of single-gas FP32 grids (2-D: warp-marching
strips, dfv_gasw.cuh; 3-D: marching columns, dfv_gas3.cuh, whose plane boxes
come by TMA when rows are 16-byte multiples (widths 40, 48 below) and by
per-thread asynchronous copies otherwise (widths 33-37)): against the FP64
oracle (relative L1 per conserved plane <= 1e-4) on grids with ragged last
strips and chunks, odd widths, a single strip, grids narrower than the halo,
reflective walls on every side, a stiffened gas, with and without a body;
against the general stage kernel on the same input (both FP32: they differ by
rounding only); and across chunk lengths (bit-identical: a cell's arithmetic
does not depend on how the grid is cut into work items)."""
import numpy as np
import pytest

import workloads as W
from gpu_util import rel_l1, run_both

pytestmark = pytest.mark.gpu

B = pytest.importorskip("paper_2111_11806_gb300.binding")


def walled(wl, walls):
    wl.walls = tuple(walls)
    return wl


def water(wl):
    """The same random state as a single stiffened gas (water)."""
    L = W.layout(2, 1, False)
    rng = np.random.default_rng(5)
    wl.materials = [W.WATER]
    wl.prim[L["irho"]] = 1000.0 * (1.0 + 0.02 * rng.standard_normal(wl.ncell))
    wl.prim[L["ip"]] = 1e5 * (1.0 + 50.0 * rng.random(wl.ncell))
    return wl


CASES = [
    ("ragged_100x37", lambda: W.random_state(2, (100, 37), 1, False, seed=201)),
    ("two_strips_32x16", lambda: W.random_state(2, (32, 16), 1, False, seed=202)),
    ("tiny_4x3", lambda: W.random_state(2, (4, 3), 1, False, seed=203, body=False)),
    ("thin_128x8", lambda: W.random_state(2, (128, 8), 1, False, seed=204)),
    ("walls_all_68x50", lambda: walled(W.random_state(2, (68, 50), 1, False, seed=205), (1, 1, 1, 1))),
    ("walls_low_72x33", lambda: walled(W.random_state(2, (72, 33), 1, False, seed=206), (1, 0, 1, 0))),
    ("water_64x40", lambda: water(W.random_state(2, (64, 40), 1, False, seed=207))),
    ("no_body_96x48", lambda: W.random_state(2, (96, 48), 1, False, seed=208, body=False)),
    ("cylinder_192", lambda: W.cylinder_2d(192)),
    ("odd_37x29", lambda: W.random_state(2, (37, 29), 1, False, seed=211)),
    ("walls_odd_45x31", lambda: walled(W.random_state(2, (45, 31), 1, False, seed=212), (1, 1, 1, 1))),
    ("one_row_57x1", lambda: W.random_state(2, (57, 1), 1, False, seed=213, body=False)),
    ("narrow_3x40_walls", lambda: walled(W.random_state(2, (3, 40), 1, False, seed=214, body=False), (1, 1, 0, 0))),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_gas_kernel_matches_oracle(name, make):
    wl = make()
    for steps in (1, 20):
        o, g = run_both(wl, steps, B.DFV_FP32)
        err = rel_l1(g.cons(), o.cons(), wl)
        assert np.all(err <= 1e-4), (steps, err)


@pytest.mark.parametrize("name,make", [CASES[0], CASES[4], CASES[8]], ids=[CASES[i][0] for i in (0, 4, 8)])
def test_gas_kernel_matches_general_kernel(name, make):
    wl = make()
    g1 = B.Grid.from_workload(wl, precision=B.DFV_FP32)
    g2 = B.Grid.from_workload(wl, precision=B.DFV_FP32, general_stage=True)
    t1 = g1.run(10, 0.8)
    t2 = g2.run(10, 0.8)
    assert t1 == pytest.approx(t2, rel=1e-5)
    err = rel_l1(g1.cons(), g2.cons(), wl)
    assert np.all(err <= 1e-5), err


@pytest.mark.parametrize("name,make", [CASES[0], CASES[4], CASES[8], CASES[10]],
                         ids=[CASES[i][0] for i in (0, 4, 8, 10)])
def test_gas_kernel_chunk_lengths_are_bit_identical(name, make):
    """Work items of 1, 3, 8, 64 and 4096 rows: the same bits."""
    wl = make()
    ref = B.Grid.from_workload(wl, precision=B.DFV_FP32, gas_rows=8)
    t_ref = ref.run(6, 0.8)
    for rows in (1, 3, 64, 4096):
        g = B.Grid.from_workload(wl, precision=B.DFV_FP32, gas_rows=rows)
        assert g.run(6, 0.8) == t_ref
        np.testing.assert_array_equal(g.cons(), ref.cons())


def test_gas_kernel_batch_with_long_chunks_matches_single_grids():
    """A batch whose work items are 64 rows long (the length the 256-instance
    batch takes) against single grids with 8-row items: the same bits."""
    wls = [W.ellipse_instance(i, n=n) for i, n in enumerate((150, 97, 64, 130))]
    b = B.Batch(wls, precision=B.DFV_FP32, gas_rows=64)
    b.set_all_fields()
    b.run(5, 0.8)
    for i, wl in enumerate(wls):
        g = B.Grid.from_workload(wl, precision=B.DFV_FP32, gas_rows=8)
        g.run(5, 0.8)
        np.testing.assert_array_equal(b.get_fields(i), g.cons())


def test_gas_rows_out_of_range_is_rejected():
    wl = W.cylinder_2d(64)
    for rows in (-1, 4097):
        with pytest.raises(B.DfvError):
            B.Grid.from_workload(wl, precision=B.DFV_FP32, gas_rows=rows)


def test_gas_kernel_device_dt_run():
    """dfv_run with the device time step (graph replay, deferred finalize,
    the rigid box folded by stage 3) against the oracle's own time steps."""
    wl = W.random_state(2, (100, 37), 1, False, seed=209)
    o, g = run_both(wl, 15, B.DFV_FP32, use_run=True)
    err = rel_l1(g.cons(), o.cons(), wl)
    assert np.all(err <= 1e-4), err


def test_moving_body_takes_the_general_kernel():
    """A body moving at 30 m/s needs the upwind r flux: the general kernel
    runs the stages, and the result still matches the oracle."""
    wl = W.random_state(2, (64, 48), 1, False, seed=210)
    wl.body_v = (30.0, -20.0, 0.0)
    o, g = run_both(wl, 10, B.DFV_FP32)
    err = rel_l1(g.cons(), o.cons(), wl)
    assert np.all(err <= 1e-4), err


# ---- the 3-D gas kernel (dfv_gas3.cuh): marching columns, ring of planes

CASES3 = [
    ("three_chunks_40x30x75", lambda: W.random_state(3, (40, 30, 75), 1, False, seed=221)),
    ("ragged_37x21x33", lambda: W.random_state(3, (37, 21, 33), 1, False, seed=222)),
    ("walls_all_34x18x40", lambda: walled(W.random_state(3, (34, 18, 40), 1, False, seed=223), (1, 1, 1, 1, 1, 1))),
    ("walls_z_33x26x40", lambda: walled(W.random_state(3, (33, 26, 40), 1, False, seed=224), (0, 0, 0, 0, 1, 1))),
    ("thin_z_35x9x3", lambda: W.random_state(3, (35, 9, 3), 1, False, seed=225)),
    ("one_plane_40x10x1", lambda: W.random_state(3, (40, 10, 1), 1, False, seed=226, body=False)),
    ("sphere_48", lambda: W.sphere_3d(48)),
]


@pytest.mark.parametrize("name,make", CASES3, ids=[c[0] for c in CASES3])
def test_gas3_kernel_matches_oracle(name, make):
    wl = make()
    for steps in (1, 10):
        o, g = run_both(wl, steps, B.DFV_FP32)
        err = rel_l1(g.cons(), o.cons(), wl)
        assert np.all(err <= 1e-4), (steps, err)


@pytest.mark.parametrize("name,make", [CASES3[0], CASES3[2], CASES3[6]], ids=[CASES3[i][0] for i in (0, 2, 6)])
def test_gas3_kernel_matches_general_kernel(name, make):
    wl = make()
    g1 = B.Grid.from_workload(wl, precision=B.DFV_FP32)
    g2 = B.Grid.from_workload(wl, precision=B.DFV_FP32, general_stage=True)
    t1 = g1.run(8, 0.8)
    t2 = g2.run(8, 0.8)
    assert t1 == pytest.approx(t2, rel=1e-5)
    err = rel_l1(g1.cons(), g2.cons(), wl)
    assert np.all(err <= 1e-5), err
