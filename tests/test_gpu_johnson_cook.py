"""GPU parity of the Johnson-Cook flow stress in the plastic update (FP64
polar decomposition and return in both forms) against the FP64 oracle:
relative L1 per conserved plane <= 1e-12 after one step and <= 1e-8 after 30
steps in FP64, <= 1e-4 after 20 steps in FP32.  Cases: a copper block with
plastic-strain planes striking the wedge (rate and hardening active where it
yields), and a random two-material state strained beyond yield everywhere."""
import numpy as np
import pytest

import workloads as W
from gpu_util import rel_l1, run_both

pytestmark = pytest.mark.gpu

B = pytest.importorskip("paper_2111_11806_gb300.binding")


def copper_impact(n=96):
    return W.with_history(W.impact_2d(n, solid_material=W.COPPER))


def copper_random():
    wl = W.random_state(2, (40, 37), 2, True, seed=401, amp=0.02)
    L = W.layout(2, 2, True)
    wl.materials = [W.COPPER, W.AIR]
    wl.prim[L["irho"]] = W.COPPER["rho0"] * wl.prim[L["irho"]] / W.ALUMINIUM["rho0"]
    return W.with_history(wl, seed=402, amp=0.5)


CASES = [("copper_impact_96", copper_impact), ("copper_random_40x37", copper_random)]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_fp64_matches_oracle(name, make):
    wl = make()
    o, g = run_both(wl, 1, B.DFV_FP64)
    err = rel_l1(g.cons(), o.cons(), wl)
    assert np.all(err <= 1e-12), err
    o, g = run_both(wl, 30, B.DFV_FP64)
    err = rel_l1(g.cons(), o.cons(), wl)
    assert np.all(err <= 1e-8), err


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_fp32_matches_oracle(name, make):
    wl = make()
    o, g = run_both(wl, 20, B.DFV_FP32)
    err = rel_l1(g.cons(), o.cons(), wl)
    assert np.all(err <= 1e-4), err


def test_johnson_cook_yields_differently_from_perfect_plasticity():
    """The flow stress matters: the same case with a constant yield stress of
    c1 ends with different plastic strain planes (on the GPU and the oracle
    alike)."""
    wl = copper_random()
    o, g = run_both(wl, 5, B.DFV_FP64)
    pp = dict({k: v for k, v in W.COPPER.items() if not k.startswith("jc_")}, sigY=W.COPPER["jc_c1"])
    wl2 = copper_random()
    wl2.materials = [pp, W.AIR]
    o2, g2 = run_both(wl2, 5, B.DFV_FP64)
    L = W.layout(2, 2, True, history=True)
    a, b = g.cons()[L["ih"]], g2.cons()[L["ih"]]
    assert np.abs(a - b).sum() > 1e-3 * np.abs(b).sum()
