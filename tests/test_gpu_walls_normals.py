"""GPU parity of the seeding options of Sec. 3.2-3.3 and of reflective walls
against the oracle: ELVIRA normals (2-D), the fixed 1.5 dx probe (seeded
from the step-start state in two launches), slip walls, alone and combined,
including the Mach 10 wedge with its floor wall.  FP64: relative L1 per plane
<= 1e-12 after one step, <= 1e-8 after 100 steps; FP32 <= 1e-4."""
import numpy as np
import pytest

import workloads as W
from gpu_util import rel_l1, run_both, same_kernel_bits

pytestmark = pytest.mark.gpu

B = pytest.importorskip("paper_2111_11806_gb300.binding")

EL = dict(normal_method=1)
FX = dict(probe_mode=1)
ELFX = dict(normal_method=1, probe_mode=1)


def with_walls(wl, walls):
    wl.walls = tuple(walls)
    return wl


ONE_STEP = [
    ("cylinder_64_elvira", lambda: W.cylinder_2d(64), EL),
    ("cylinder_96x80_fixed", lambda: W.cylinder_2d(96, ny=80), FX),
    ("impact_96_elvira_fixed", lambda: W.impact_2d(96), ELFX),
    ("dynamic_body_128x64_elvira", lambda: W.dynamic_body_2d(128, 64), EL),
    ("reflection_1d_400_fixed", lambda: W.shock_reflection_1d(400), FX),
    ("sphere_3d_36x20x18_fixed", lambda: W.random_state(3, (36, 20, 18), 1, False, seed=15), FX),
    ("two_fluid_body_70x45_elvira_fixed", lambda: W.random_state(2, (70, 45), 2, False, seed=11), ELFX),
    ("wedge_120x80_elvira", lambda: W.wedge_2d(120), EL),
    ("wedge_mach1.7_25deg_90x60", lambda: W.wedge_2d(90, 1.7, 25.0), {}),
    ("solid_two_mat_40x37_walls", lambda: with_walls(
        W.random_state(2, (40, 37), 2, True, seed=12, amp=0.02), (1, 0, 0, 1)), {}),
    ("two_fluid_70x45_all_walls",
     lambda: with_walls(W.random_state(2, (70, 45), 2, False, seed=11), (1, 1, 1, 1)), ELFX),
    ("solid_1d_300_walls", lambda: with_walls(W.random_state(1, (300,), 1, True, seed=13, amp=0.02), (1, 1)), {}),
    ("sphere_3d_36x20x18_walls",
     lambda: with_walls(W.random_state(3, (36, 20, 18), 1, False, seed=15), (1, 0, 0, 1, 1, 0)), {}),
]


@pytest.mark.parametrize("name,make,var", ONE_STEP, ids=[c[0] for c in ONE_STEP])
def test_fp64_one_step(name, make, var):
    wl = make()
    o, g = run_both(wl, 1, B.DFV_FP64, **var)
    err = rel_l1(g.cons(), o.cons(), wl)
    assert np.all(err <= 1e-12), err


HUNDRED = [
    ("wedge_120x80_elvira", lambda: W.wedge_2d(120), EL),
    ("cylinder_64_elvira_fixed", lambda: W.cylinder_2d(64), ELFX),
    ("reflection_1d_wall", lambda: with_walls(W.shock_reflection_1d(400), (0, 1)), {}),
]


@pytest.mark.parametrize("name,make,var", HUNDRED, ids=[c[0] for c in HUNDRED])
def test_fp64_100_steps(name, make, var):
    wl = make()
    o, g = run_both(wl, 100, B.DFV_FP64, **var)
    err = rel_l1(g.cons(), o.cons(), wl)
    assert np.all(err <= 1e-8), err


FP32 = [
    ("wedge_120x80_elvira", lambda: W.wedge_2d(120), 40, EL),
    ("cylinder_64_fixed", lambda: W.cylinder_2d(64), 50, FX),
    ("impact_96_elvira", lambda: W.impact_2d(96), 20, EL),
]


@pytest.mark.parametrize("name,make,steps,var", FP32, ids=[c[0] for c in FP32])
def test_fp32(name, make, steps, var):
    wl = make()
    o, g = run_both(wl, steps, B.DFV_FP32, **var)
    err = rel_l1(g.cons(), o.cons(), wl)
    assert np.all(err <= 1e-4), err


def test_wedge_full_size_one_step():
    """The 1200x800 Mach 10 wedge (the paper's finest resolution), one step
    with ELVIRA, against the oracle: FP64 to 1e-12, FP32 to 1e-4."""
    wl = W.wedge_2d(1200)
    from oracle import Oracle
    o = Oracle.from_workload(wl, normal_method=1)
    dt = o.compute_dt(wl.cfl)
    o.step(dt)
    ref = o.cons()
    for prec, tol in ((B.DFV_FP64, 1e-12), (B.DFV_FP32, 1e-4)):
        g = B.Grid.from_workload(wl, precision=prec, normal_method=1)
        g.step(dt)
        err = rel_l1(g.cons(), ref, wl)
        assert np.all(err <= tol), (prec, err)
        del g


def test_elvira_rejected_off_2d():
    wl = W.shock_reflection_1d(64)
    with pytest.raises(B.DfvError):
        B.Grid.from_workload(wl, precision=B.DFV_FP64, normal_method=1)


def test_fixed_probe_counts_its_extra_launch():
    wl = W.cylinder_2d(64)
    per_step = []
    for mode in (0, 1):
        g = B.Grid.from_workload(wl, precision=B.DFV_FP64, probe_mode=mode)
        n0 = g.launch_count()
        g.step(1e-7)
        per_step.append(g.launch_count() - n0)
    assert per_step[1] == per_step[0] + 1


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32"])
def test_batch_with_walls_and_options_equals_single_grids(precision):
    wls = [with_walls(W.ellipse_instance(i, n=n), (0, 0, 1, 1) if i % 2 else (1, 0, 0, 0))
           for i, n in enumerate([40, 64, 97])]
    b = B.Batch(wls, precision=precision, **ELFX)
    b.set_all_fields()
    b.run(4, 0.8)
    for i, wl in enumerate(wls):
        g = B.Grid.from_workload(wl, precision=precision, **ELFX)
        g.run(4, 0.8)
        same_kernel_bits(b.get_fields(i), g.cons(), wl, precision)
