"""GPU parity of the two method variants against the oracle: the HLLC-LM flux
option and the Riemann-problem-based seeding of Sec. 3.2 (step 5, second
option), alone and together, on the workloads of the plain parity tests.
Same bars: FP64 relative L1 per plane <= 1e-12 after one step and <= 1e-8
after 100 steps; FP32 <= 1e-4 on the workload-shaped cases."""
import numpy as np
import pytest

import workloads as W
from gpu_util import rel_l1, run_both, same_kernel_bits

pytestmark = pytest.mark.gpu

B = pytest.importorskip("paper_2111_11806_gb300.binding")

LM = dict(hllc_lm=True)
RS = dict(seed_variant=1)
BOTH = dict(hllc_lm=True, seed_variant=1)

ONE_STEP = [
    ("cylinder_64_lm", lambda: W.cylinder_2d(64), LM),
    ("cylinder_96x80_both", lambda: W.cylinder_2d(96, ny=80), BOTH),
    ("reflection_1d_400_rs", lambda: W.shock_reflection_1d(400), RS),
    ("two_fluid_body_70x45_both", lambda: W.random_state(2, (70, 45), 2, False, seed=11), BOTH),
    ("solid_two_mat_40x37_rs", lambda: W.random_state(2, (40, 37), 2, True, seed=12, amp=0.02), RS),
    # the solid branch of HLLC-LM (normal traction in the star states) on the impact; the random-noise
    # solid state sits at Ma ~ 1e-3, where the option removes nearly all acoustic dissipation and the
    # oracle itself goes non-physical within one step
    ("impact_96_lm", lambda: W.impact_2d(96), LM),
    ("sphere_3d_36x20x18_both", lambda: W.random_state(3, (36, 20, 18), 1, False, seed=15), BOTH),
    ("periodic_two_fluid_33x40_both",
     lambda: W.random_state(2, (33, 40), 2, False, seed=16, periodic=(1, 1)), BOTH),
    ("dynamic_body_128x64_rs", lambda: W.dynamic_body_2d(128, 64), RS),
    ("impact_96_rs", lambda: W.impact_2d(96), RS),
]


@pytest.mark.parametrize("name,make,var", ONE_STEP, ids=[c[0] for c in ONE_STEP])
def test_variant_fp64_one_step(name, make, var):
    wl = make()
    o, g = run_both(wl, 1, B.DFV_FP64, **var)
    err = rel_l1(g.cons(), o.cons(), wl)
    assert np.all(err <= 1e-12), err


HUNDRED = [
    ("cylinder_64_lm", lambda: W.cylinder_2d(64), LM),
    ("cylinder_96x80_both", lambda: W.cylinder_2d(96, ny=80), BOTH),
    ("dynamic_body_128x64_rs", lambda: W.dynamic_body_2d(128, 64), RS),
    ("reflection_1d_400_rs", lambda: W.shock_reflection_1d(400), RS),
]


@pytest.mark.parametrize("name,make,var", HUNDRED, ids=[c[0] for c in HUNDRED])
def test_variant_fp64_100_steps(name, make, var):
    wl = make()
    o, g = run_both(wl, 100, B.DFV_FP64, **var)
    err = rel_l1(g.cons(), o.cons(), wl)
    assert np.all(err <= 1e-8), err


FP32 = [
    ("cylinder_64_lm", lambda: W.cylinder_2d(64), 50, LM),
    ("impact_96_rs", lambda: W.impact_2d(96), 20, RS),
    ("dynamic_body_128x64_rs", lambda: W.dynamic_body_2d(128, 64), 30, RS),
    ("cylinder_96x80_both", lambda: W.cylinder_2d(96, ny=80), 40, BOTH),
]


@pytest.mark.parametrize("name,make,steps,var", FP32, ids=[c[0] for c in FP32])
def test_variant_fp32(name, make, steps, var):
    wl = make()
    o, g = run_both(wl, steps, B.DFV_FP32, **var)
    err = rel_l1(g.cons(), o.cons(), wl)
    assert np.all(err <= 1e-4), err


def test_variants_change_the_result():
    """The options reach the kernels: each variant gives a different state
    than the plain scheme on the cylinder after a few steps."""
    wl = W.cylinder_2d(64)
    ref = B.Grid.from_workload(wl, precision=B.DFV_FP64)
    ref.run(5, wl.cfl)
    for var in (LM, RS):
        g = B.Grid.from_workload(wl, precision=B.DFV_FP64, **var)
        g.run(5, wl.cfl)
        assert np.max(np.abs(g.cons() - ref.cons())) > 0.0, var


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32"])
def test_batch_with_variants_equals_single_grids(precision):
    wls = [W.ellipse_instance(i, n=n) for i, n in enumerate([40, 64, 97])]
    b = B.Batch(wls, precision=precision, **BOTH)
    b.set_all_fields()
    b.run(4, 0.8)
    for i, wl in enumerate(wls):
        g = B.Grid.from_workload(wl, precision=precision, **BOTH)
        g.run(4, 0.8)
        same_kernel_bits(b.get_fields(i), g.cons(), wl, precision)


# ---- seeding of every stage input (dfv_options.seed_stages; oracle pins in
# tests/test_oracle_seed_stages.py)

SS = dict(seed_stages=True)

SEED_STAGES_ONE = [
    ("two_fluid_body_70x45_ss", lambda: W.random_state(2, (70, 45), 2, False, seed=11), SS),
    ("one_fluid_body_70x45_fixed_probe_ss", lambda: W.random_state(2, (70, 45), 1, False, seed=11),
     dict(seed_stages=True, probe_mode=1)),
    ("dynamic_body_128x64_ss", lambda: W.dynamic_body_2d(128, 64), SS),
    ("solid_two_mat_40x37_ss", lambda: W.random_state(2, (40, 37), 2, True, seed=12, amp=0.02), SS),
    ("sphere_3d_36x20x18_ss", lambda: W.random_state(3, (36, 20, 18), 1, False, seed=15), SS),
]


@pytest.mark.parametrize("name,make,var", SEED_STAGES_ONE, ids=[c[0] for c in SEED_STAGES_ONE])
def test_seed_stages_fp64_one_step(name, make, var):
    wl = make()
    o, g = run_both(wl, 1, B.DFV_FP64, **var)
    err = rel_l1(g.cons(), o.cons(), wl)
    assert np.all(err <= 1e-12), err


@pytest.mark.parametrize("name,make,var", [SEED_STAGES_ONE[0], SEED_STAGES_ONE[2]],
                         ids=[SEED_STAGES_ONE[i][0] for i in (0, 2)])
def test_seed_stages_fp64_100_steps(name, make, var):
    wl = make()
    o, g = run_both(wl, 100, B.DFV_FP64, **var)
    err = rel_l1(g.cons(), o.cons(), wl)
    assert np.all(err <= 1e-8), err


@pytest.mark.parametrize("name,make,steps", [
    ("cylinder_64", lambda: W.cylinder_2d(64), 30),                       # the 2-D gas kernel path
    ("one_fluid_body_70x45", lambda: W.random_state(2, (70, 45), 1, False, seed=11), 20),
    ("sphere_3d_36x20x18", lambda: W.random_state(3, (36, 20, 18), 1, False, seed=15), 10),
])
def test_seed_stages_fp32(name, make, steps):
    wl = make()
    o, g = run_both(wl, steps, B.DFV_FP32, seed_stages=True)
    err = rel_l1(g.cons(), o.cons(), wl)
    assert np.all(err <= 1e-4), err


def test_seed_stages_device_run_equals_host_steps():
    """dfv_run (graph replay; the extra seeding launches captured) against
    host-driven steps, bit for bit."""
    wl = W.random_state(2, (70, 45), 1, False, seed=11)
    g1 = B.Grid.from_workload(wl, precision=B.DFV_FP64, seed_stages=True)
    g2 = B.Grid.from_workload(wl, precision=B.DFV_FP64, seed_stages=True)
    t1 = 0.0
    for _ in range(8):
        dt = g1.compute_dt(0.8)
        g1.step(dt)
        t1 += dt
    assert g2.run(8, 0.8) == pytest.approx(t1, rel=1e-15)
    np.testing.assert_array_equal(g1.cons(), g2.cons())


def test_batch_refuses_seed_stages():
    with pytest.raises(B.DfvError, match="UNSUPPORTED"):
        B.Batch([W.ellipse_instance(0, n=64)], precision=B.DFV_FP32, seed_stages=True)
