"""GPU parity of the three-material form against the oracle (water, helium
and air; aluminium, water and air for the solid), same bars as the plain
parity tests: FP64 1e-12 after one step and 1e-8 after 100 steps, FP32 1e-4
on a smooth case."""
import numpy as np
import pytest

import workloads as W
from gpu_util import rel_l1, run_both

pytestmark = pytest.mark.gpu

B = pytest.importorskip("paper_2111_11806_gb300.binding")

ONE = [
    ("fluid_2d_70x45", lambda: W.random_state(2, (70, 45), 3, False, seed=81)),
    ("fluid_1d_257", lambda: W.random_state(1, (257,), 3, False, seed=82)),
    ("solid_2d_40x37", lambda: W.random_state(2, (40, 37), 3, True, seed=84, amp=0.02)),
    ("solid_1d_300", lambda: W.random_state(1, (300,), 3, True, seed=85, amp=0.02)),
    ("solid_2d_history_40x37", lambda: W.with_history(W.random_state(2, (40, 37), 3, True, seed=86, amp=0.02),
                                                      seed=8, amp=0.01)),
]


@pytest.mark.parametrize("name,make", ONE, ids=[c[0] for c in ONE])
def test_three_materials_fp64_one_step(name, make):
    wl = make()
    o, g = run_both(wl, 1, B.DFV_FP64)
    err = rel_l1(g.cons(), o.cons(), wl)
    assert np.all(err <= 1e-12), err


def test_three_materials_fp64_100_steps():
    wl = W.random_state(2, (70, 45), 3, False, seed=81, amp=0.05)
    o, g = run_both(wl, 100, B.DFV_FP64, cfl=0.6)
    err = rel_l1(g.cons(), o.cons(), wl)
    assert np.all(err <= 1e-8), err


def test_three_materials_fp32_smooth():
    """A smooth three-fluid state (no per-cell noise) in FP32."""
    wl = W.random_state(2, (64, 48), 3, False, seed=87, amp=0.02)
    L = W.layout(2, 3, False)
    X, Y, _ = W.cell_centres(wl.n, wl.lo, wl.hi)
    for a in range(2):
        wl.prim[L["iu"] + a] = 40.0 * np.sin(2 * np.pi * (X + 0.2 * a))
    wl.prim[L["ip"]] = 1e5 * (1.0 + 0.05 * np.cos(2 * np.pi * Y))
    o, g = run_both(wl, 20, B.DFV_FP32, cfl=0.6)
    err = rel_l1(g.cons(), o.cons(), wl)
    assert np.all(err <= 1e-4), err


def test_three_materials_3d_fp32_and_fp64_refused():
    """3-D three-material fluid: FP32 against the oracle (per-cell noise on
    every primitive); the FP64 form's tile exceeds a CTA's shared memory and
    is refused."""
    wl = W.random_state(3, (36, 20, 18), 3, False, seed=83)
    o, g = run_both(wl, 5, B.DFV_FP32)
    err = rel_l1(g.cons(), o.cons(), wl)
    assert np.all(err <= 1e-4), err
    with pytest.raises(B.DfvError, match="UNSUPPORTED"):
        B.Grid.from_workload(wl, precision=B.DFV_FP64)
