"""GPU parity of the 3-D single-material FP32 update, whose stage kernel
marches along z in chunks of planes: grids of several chunks with a ragged
last chunk, chunks shorter than the stencil halo, periodic and reflective z
boundaries, a body moving in z (upwind r flux on the z faces), the device
CFL maximum and the rigid box it folds, against the FP64 oracle (relative L1
per conserved plane <= 1e-4 after one step and after 10 steps)."""
import numpy as np
import pytest

import workloads as W
from gpu_util import rel_l1, run_both

pytestmark = pytest.mark.gpu

B = pytest.importorskip("paper_2111_11806_gb300.binding")


def with_walls(wl, walls):
    wl.walls = tuple(walls)
    return wl


def moving(wl, v):
    wl.body_v = tuple(v)
    return wl


CASES = [
    # 3 chunks of planes (32, 32, 11), x and y tiles ragged
    ("three_chunks_40x30x75", lambda: W.random_state(3, (40, 30, 75), 1, False, seed=91)),
    ("periodic_z_33x25x70", lambda: W.random_state(3, (33, 25, 70), 1, False, seed=92, periodic=(0, 0, 1))),
    # fully periodic without a body (the seeded sphere profile is not periodic)
    ("periodic_all_32x16x64", lambda: W.random_state(3, (32, 16, 64), 1, False, seed=93, periodic=(1, 1, 1),
                                                     body=False)),
    ("walls_z_35x26x40", lambda: with_walls(W.random_state(3, (35, 26, 40), 1, False, seed=94),
                                           (0, 1, 0, 0, 1, 1))),
    ("walls_xy_33x26x40", lambda: with_walls(W.random_state(3, (33, 26, 40), 1, False, seed=101),
                                            (1, 1, 1, 1, 0, 0))),
    ("body_moving_z_36x30x66", lambda: moving(W.random_state(3, (36, 30, 66), 1, False, seed=95),
                                              (30.0, -20.0, 45.0))),
    ("thin_z_35x9x4", lambda: W.random_state(3, (35, 9, 4), 1, False, seed=96)),
    ("one_plane_40x10x1", lambda: W.random_state(3, (40, 10, 1), 1, False, seed=97, body=False)),
    ("exact_chunk_32x8x32", lambda: W.random_state(3, (32, 8, 32), 1, False, seed=98)),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_fp32_one_step(name, make):
    wl = make()
    o, g = run_both(wl, 1, B.DFV_FP32)
    err = rel_l1(g.cons(), o.cons(), wl)
    assert np.all(err <= 1e-4), err


@pytest.mark.parametrize("name,make", [CASES[0], CASES[3], CASES[4]], ids=[CASES[i][0] for i in (0, 3, 4)])
def test_fp32_ten_steps_device_dt(name, make):
    """dfv_run: dt from the stage-3 CFL maximum, seeding from the rigid box
    that stage 3 folds, ten steps."""
    wl = make()
    o, g = run_both(wl, 10, B.DFV_FP32, use_run=True)
    err = rel_l1(g.cons(), o.cons(), wl)
    assert np.all(err <= 1e-4), err


def test_fp64_three_chunks_unchanged():
    """The FP64 3-D path keeps the tiled kernel: 1e-12 after one step on the
    multi-chunk grid."""
    wl = CASES[0][1]()
    o, g = run_both(wl, 1, B.DFV_FP64)
    err = rel_l1(g.cons(), o.cons(), wl)
    assert np.all(err <= 1e-12), err


def test_fp32_dt_matches_oracle():
    wl = W.random_state(3, (40, 30, 75), 1, False, seed=99)
    from oracle import Oracle
    o = Oracle.from_workload(wl)
    g = B.Grid.from_workload(wl, precision=B.DFV_FP32)
    for _ in range(3):
        dt_o, dt_g = o.compute_dt(0.6), g.compute_dt(0.6)
        # the wave speeds are formed in FP32 on the device
        assert dt_g == pytest.approx(dt_o, rel=1e-5)
        o.step(dt_o)
        g.step(dt_o)


def test_split_runs_equal_one_run():
    """Device-driven steps of a static body: the finalize of each step runs
    in the next step's seeding launch; split runs, with and without reading
    the time, give bit-identical fields and time to one run."""
    wl = CASES[0][1]()
    g1 = B.Grid.from_workload(wl, precision=B.DFV_FP32)
    t1 = g1.run(9, 0.6)
    g2 = B.Grid.from_workload(wl, precision=B.DFV_FP32)
    g2.run(4, 0.6, sync=False)
    g2.run(2, 0.6, sync=False)
    t2 = g2.run(3, 0.6)
    assert t2 == t1
    np.testing.assert_array_equal(g1.cons(), g2.cons())
