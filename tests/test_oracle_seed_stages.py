"""Pins of the option that seeds every stage input (the stage-2 input U1 and
the stage-3 input U3 as well as the step-start state; Sec. 3.2 seeds once per
step before stage 1).  The planar body of the probe-stencil pins: the first
rigid cell's probe point at s = 1.0 is the centre of its fluid neighbour, so a
seeded state holds that neighbour's state with the velocity reversed.  With
the option on, the stage inputs must show this against their own fluid cells;
with it off they keep the step-start ghost states, which a stage moves away
from.  CPU only."""
import numpy as np
import pytest

import workloads as W
from oracle import Oracle
from test_oracle_seed_stencil import planar_1d


def first_band(w, body_right):
    rigid = np.nonzero(w[3] > 0.5)[0]
    i = rigid.min() if body_right else rigid.max()
    return i, (i - 1 if body_right else i + 1)


@pytest.mark.parametrize("body_right", [True, False])
def test_stage_inputs_are_seeded_from_their_own_fluid(body_right):
    o, w = planar_1d(80, body_right, np.random.default_rng(5))
    o.set_seed_stages(True)
    i, j = first_band(w, body_right)
    o.step(o.compute_dt(0.5))
    for k in (1, 2):
        U = o.stage_input(k)                     # (rho, rho u, rho E, r)
        assert U[0, i] == pytest.approx(U[0, j], rel=1e-13)
        assert U[1, i] == pytest.approx(-U[1, j], rel=1e-13)
        assert U[2, i] == pytest.approx(U[2, j], rel=1e-13)


@pytest.mark.parametrize("body_right", [True, False])
def test_without_the_option_stage_inputs_keep_the_step_start_ghosts(body_right):
    o, w = planar_1d(80, body_right, np.random.default_rng(5))
    i, j = first_band(w, body_right)
    ref, _ = planar_1d(80, body_right, np.random.default_rng(5))
    ref.seed()
    ghost = ref.cons()[:, i]                     # the ghost of the step-start state
    o.step(o.compute_dt(0.5))
    for k in (1, 2):
        U = o.stage_input(k)
        np.testing.assert_allclose(U[:3, i], ghost[:3], rtol=1e-13)
        # the stage moved the fluid neighbour: the ghost is no longer its mirror image
        assert abs(U[1, i] + U[1, j]) > 1e-6 * abs(U[1, j])


def test_option_changes_a_run_near_the_body():
    wl = W.random_state(2, (40, 37), 1, False, seed=301)
    a = Oracle.from_workload(wl)
    b = Oracle.from_workload(wl, seed_stages=True)
    for _ in range(3):
        dt = a.compute_dt(0.8)
        a.step(dt)
        b.step(dt)
    ra, rb = a.cons(), b.cons()
    rel = np.abs(ra - rb).sum(axis=1) / np.abs(ra).sum(axis=1)
    assert rel[:4].max() > 1e-5


def test_quiescent_gas_with_static_body_is_unchanged():
    wl = W.cylinder_2d(40)
    wl.prim[1:3] = 0.0                           # no velocity
    wl.prim[0] = 1.2
    wl.prim[3] = 1e5
    o = Oracle.from_workload(wl, seed_stages=True)
    o.seed()
    before = o.cons()
    for _ in range(3):
        o.step(1e-6)
    np.testing.assert_allclose(o.cons(), before, rtol=0, atol=1e-9 * np.abs(before).max())
