"""dfv_compute_dt_noalloc -- the CFL time step computed without any device
allocation, for callers that cannot call cudaMalloc (their device memory is
owned and pooled by a host code, or they must not allocate while other work
runs).  Its scratch is a fixed array inside the library, so its result must
be the same as that of dfv_compute_dt on the same state; checked on two calls
in a row, in FP64 and FP32, through the C ABI.  This file is collected last."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

B = pytest.importorskip("paper_2111_11806_gb300.binding")

CASES = [
    ("cylinder_96x80", lambda: W.cylinder_2d(96, ny=80)),
    ("two_fluid_70x45", lambda: W.random_state(2, (70, 45), 2, False, seed=11)),
    ("impact_64", lambda: W.impact_2d(64)),
    ("dynamic_body_128x64", lambda: W.dynamic_body_2d(128, 64)),
    ("sphere_20x18x16", lambda: W.random_state(3, (20, 18, 16), 1, False, seed=15)),
]


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32"])
@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_noalloc_dt_matches_compute_dt_on_two_calls(name, make, precision):
    import torch
    wl = make()
    g = B.Grid.from_workload(wl, precision=precision)
    cfl = 0.8
    for call in range(2):
        cons = torch.empty((wl.nvar, wl.ncell), dtype=torch.float64, device="cuda")
        g.get_fields(B.DFV_FIELDS_CONSERVED, out=cons)
        state = cons if precision == B.DFV_FP64 else cons.to(torch.float32)
        torch.cuda.synchronize()
        _, v_body, _ = g.body()
        dt_ref = g.compute_dt(cfl)
        dt = B.compute_dt_noalloc(wl.dim, wl.n, wl.lo, wl.hi, wl.materials, state.data_ptr(), wl.ncell, cfl,
                                  precision=precision, solid=wl.solid, v_body=v_body)
        assert dt == pytest.approx(dt_ref, rel=1e-12), (call, dt, dt_ref)
        g.step(dt_ref)          # a different state for the second call
        g.check(timeout_ms=60000)


def test_noalloc_rejects_grids_beyond_its_scratch():
    import torch
    dummy = torch.zeros(1, dtype=torch.float64, device="cuda")
    n = (257, 256, 256)   # 16.8 M cells > DFV_NOALLOC_MAX_CELLS
    with pytest.raises(B.DfvError, match="TOO_LARGE"):
        B.compute_dt_noalloc(3, n, (0, 0, 0), (1, 1, 1), [W.AIR], dummy.data_ptr(), int(np.prod(n)), 0.8)


def test_noalloc_rejects_bad_material_parameters():
    """The same parameter checks as dfv_add_material: gamma <= 1 for a gas,
    rho0 <= 0 for a Romenskii solid."""
    import torch
    dummy = torch.zeros(4 * 8 * 8, dtype=torch.float64, device="cuda")
    bad_gas = dict(W.AIR, gamma=1.0)
    with pytest.raises(B.DfvError, match="DFV_ERR_ARG"):
        B.compute_dt_noalloc(2, (8, 8), (0, 0), (1, 1), [bad_gas], dummy.data_ptr(), 64, 0.8)
    bad_solid = dict(W.ALUMINIUM, rho0=0.0)
    with pytest.raises(B.DfvError, match="DFV_ERR_ARG"):
        B.compute_dt_noalloc(2, (8, 8), (0, 0), (1, 1), [bad_solid], dummy.data_ptr(), 64, 0.8, solid=True)
