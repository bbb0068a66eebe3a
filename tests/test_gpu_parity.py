"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle on
the same seeded inputs.  Plain FP64: relative L1 per conserved plane <= 1e-12
after one step and <= 1e-8 after 100 steps.  FP32 bulk form: <= 1e-4.
Sizes span several tiles with ragged edges; the full-size 2-D workloads are
compared after one step."""
import math

import numpy as np
import pytest

import workloads as W
from gpu_util import rel_l1, run_both

pytestmark = pytest.mark.gpu

B = pytest.importorskip("paper_2111_11806_gb300.binding")


def cases_fp64():
    return [
        ("1d_reflection_400", lambda: W.shock_reflection_1d(400)),
        ("2d_cylinder_64", lambda: W.cylinder_2d(64)),
        ("2d_cylinder_96x80", lambda: W.cylinder_2d(96, ny=80)),
        ("2d_two_fluid_body_70x45", lambda: W.random_state(2, (70, 45), 2, False, seed=11)),
        ("2d_solid_two_mat_40x37", lambda: W.random_state(2, (40, 37), 2, True, seed=12, amp=0.02)),
        ("1d_solid_300", lambda: W.random_state(1, (300,), 1, True, seed=13, amp=0.02)),
        ("1d_two_fluid_257", lambda: W.random_state(1, (257,), 2, False, seed=14)),
        ("3d_sphere_36x20x18", lambda: W.random_state(3, (36, 20, 18), 1, False, seed=15)),
        ("2d_periodic_two_fluid_33x40", lambda: W.random_state(2, (33, 40), 2, False, seed=16, periodic=(1, 1))),
        ("2d_dynamic_body_128x64", lambda: W.dynamic_body_2d(128, 64)),
        ("2d_impact_96", lambda: W.impact_2d(96)),
    ]


@pytest.mark.parametrize("name,make", cases_fp64(), ids=[c[0] for c in cases_fp64()])
def test_fp64_one_step(name, make):
    wl = make()
    o, g = run_both(wl, 1, B.DFV_FP64)
    err = rel_l1(g.cons(), o.cons(), wl)
    assert np.all(err <= 1e-12), err


@pytest.mark.parametrize("name,make", cases_fp64()[:4] + cases_fp64()[9:11],
                         ids=[c[0] for c in cases_fp64()[:4] + cases_fp64()[9:11]])
def test_fp64_100_steps(name, make):
    wl = make()
    o, g = run_both(wl, 100, B.DFV_FP64)
    err = rel_l1(g.cons(), o.cons(), wl)
    assert np.all(err <= 1e-8), err


def test_fp64_dt_matches_oracle():
    wl = W.random_state(2, (50, 41), 2, True, seed=21, amp=0.02)
    from oracle import Oracle
    o = Oracle.from_workload(wl)
    g = B.Grid.from_workload(wl, precision=B.DFV_FP64)
    for _ in range(3):
        dt_o, dt_g = o.compute_dt(0.6), g.compute_dt(0.6)
        assert dt_g == pytest.approx(dt_o, rel=1e-13)
        o.step(dt_o)
        g.step(dt_o)


def test_dynamic_body_force_and_motion():
    wl = W.dynamic_body_2d(128, 64)
    o, g = run_both(wl, 20, B.DFV_FP64)
    fo, vo, xo = o.body()
    fg, vg, xg = g.body()
    scale = np.abs(fo).max()
    assert scale > 0
    # 20 nonlinear steps: the same 1e-8 bound as the fields after many steps
    np.testing.assert_allclose(fg, fo, rtol=0, atol=1e-8 * scale)
    np.testing.assert_allclose(vg, vo, rtol=1e-8, atol=1e-12)
    np.testing.assert_allclose(xg, xo, rtol=1e-8, atol=1e-15)
    assert vg[0] > 0   # the shock pushes the body in +x


def test_device_driven_run_matches_host_dt_loop():
    """dfv_run (dt on the device, graph replay) gives bit-identical fields to
    compute_dt + step issued from the host."""
    wl = W.cylinder_2d(80, ny=72)
    g1 = B.Grid.from_workload(wl, precision=B.DFV_FP64)
    g2 = B.Grid.from_workload(wl, precision=B.DFV_FP64)
    t1 = 0.0
    for _ in range(12):
        dt = g1.compute_dt(0.8)
        g1.step(dt)
        t1 += dt
    t2 = g2.run(12, 0.8)
    assert t2 == pytest.approx(t1, rel=1e-15)
    np.testing.assert_array_equal(g1.cons(), g2.cons())


def test_run_lands_on_t_end():
    wl = W.shock_reflection_1d(400)
    g = B.Grid.from_workload(wl, precision=B.DFV_FP64)
    t = g.run(1000, 0.8, t_end=8.874e-4)
    assert t == pytest.approx(8.874e-4, rel=1e-14)


@pytest.mark.parametrize("name,make,steps,tol", [
    ("2d_cylinder_64", lambda: W.cylinder_2d(64), 50, 1e-4),
    ("2d_impact_96", lambda: W.impact_2d(96), 20, 1e-4),
    ("2d_dynamic_body_128x64", lambda: W.dynamic_body_2d(128, 64), 30, 1e-4),
    ("2d_cylinder_96x80", lambda: W.cylinder_2d(96, ny=80), 40, 1e-4),
    # random per-cell noise on every primitive, two fluids, a body whose axis lies on a row of cell
    # centres (probe points on cell-centre lines: the probe-stencil reading of the seeding)
    ("2d_two_fluid_body_70x45", lambda: W.random_state(2, (70, 45), 2, False, seed=11), 20, 1e-4),
    ("3d_sphere_36x20x18", lambda: W.random_state(3, (36, 20, 18), 1, False, seed=15), 10, 1e-4),
    ("2d_one_fluid_body_70x45", lambda: W.random_state(2, (70, 45), 1, False, seed=11), 20, 1e-4),
])
def test_fp32_matches_oracle(name, make, steps, tol):
    wl = make()
    o, g = run_both(wl, steps, B.DFV_FP32)
    err = rel_l1(g.cons(), o.cons(), wl)
    assert np.all(err <= tol), err


def shock_x(prim_rho, n, row):
    r = prim_rho.reshape(-1, n)[row]
    return np.argmax(np.abs(np.diff(r)))


def test_fp32_shock_position_within_one_cell():
    wl = W.cylinder_2d(128)
    o, g = run_both(wl, 60, B.DFV_FP32)
    po, pg = o.prim(), g.prim()
    for row in (10, 64, 120):
        assert abs(shock_x(pg[0], 128, row) - shock_x(po[0], 128, row)) <= 1


@pytest.mark.parametrize("name,make", [
    ("cylinder_512", lambda: W.cylinder_2d(512)),
    ("dynamic_body_1024x512", lambda: W.dynamic_body_2d()),
    ("impact_1024", lambda: W.impact_2d(1024)),
])
def test_full_size_one_step(name, make):
    """The full-size 2-D workloads, one step, in the launch configuration the
    benchmark uses (FP64 against the oracle to 1e-12, FP32 to 1e-4)."""
    wl = make()
    from oracle import Oracle
    o = Oracle.from_workload(wl)
    dt = o.compute_dt(wl.cfl)
    o.step(dt)
    ref = o.cons()
    for prec, tol in ((B.DFV_FP64, 1e-12), (B.DFV_FP32, 1e-4)):
        g = B.Grid.from_workload(wl, precision=prec)
        g.step(dt)
        err = rel_l1(g.cons(), ref, wl)
        assert np.all(err <= tol), (prec, err)
        del g


def test_sphere_3d_full_size_symmetry():
    """256^3 sphere, FP32, 3 steps: the solution stays mirror-symmetric in y
    and z (a property of the exact update at any size)."""
    wl = W.sphere_3d(256)
    g = B.Grid.from_workload(wl, precision=B.DFV_FP32)
    g.run(3, wl.cfl)
    rho = g.prim()[0].reshape(256, 256, 256)       # [z, y, x]
    scale = np.abs(rho).max()
    assert np.max(np.abs(rho - rho[:, ::-1, :])) <= 1e-5 * scale
    assert np.max(np.abs(rho - rho[::-1, :, :])) <= 1e-5 * scale
    assert np.max(np.abs(rho - rho.transpose(1, 0, 2))) <= 1e-5 * scale


def test_nonphysical_state_is_reported_without_fault():
    """A negative pressure planted in the host fields makes the kernels raise
    the error word; the host sees DFV_ERR_NONPHYSICAL and the context stays usable."""
    wl = W.cylinder_2d(64)
    wl.prim[3, 100] = -5e5        # p < 0: c^2 < 0 there
    g = B.Grid.from_workload(wl, precision=B.DFV_FP64)
    with pytest.raises(B.DfvError, match="NONPHYSICAL"):
        dt = g.compute_dt(0.8)
        g.step(1e-7)
        g.check(timeout_ms=60000)
    g2 = B.Grid.from_workload(W.cylinder_2d(64), precision=B.DFV_FP64)
    g2.step(g2.compute_dt(0.8))
    g2.check(timeout_ms=60000)


def test_tiny_and_degenerate_grids():
    for n in [(1,), (5,), (3, 2), (1, 7), (2, 3, 1)]:
        dim = len(n)
        wl = W.random_state(dim, n, 1, False, seed=31, body=False)
        o, g = run_both(wl, 3, B.DFV_FP64)
        err = rel_l1(g.cons(), o.cons(), wl)
        assert np.all(err <= 1e-12), (n, err)


def test_invalid_arguments_raise():
    with pytest.raises(B.DfvError):
        B.Grid(2, (0, 4), (0, 0), (1, 1), [W.AIR])
    with pytest.raises(B.DfvError, match="UNSUPPORTED"):
        B.Grid(3, (8, 8, 8), (0, 0, 0), (1, 1, 1), [W.ALUMINIUM], solid=True)


def test_pitched_field_io_matches_packed():
    """dfv_set_fields_pitched / dfv_get_fields_pitched with padded planes give
    the packed calls' bits; the padding is neither read nor written; a pitch
    below the cell count is refused."""
    wl = W.random_state(2, (37, 23), 2, False, seed=41)
    a = B.Grid.from_workload(wl, precision=B.DFV_FP64)
    b = B.Grid.from_workload(wl, precision=B.DFV_FP64)
    pitch = wl.ncell + 13
    padded = np.full((wl.prim.shape[0], pitch), np.nan)
    padded[:, :wl.ncell] = wl.prim
    b.set_fields_pitched(padded)
    for g in (a, b):
        g.step(2e-7)
    for which in (B.DFV_FIELDS_CONSERVED, B.DFV_FIELDS_PRIMITIVE):
        out = np.full((wl.prim.shape[0], pitch), -7.0)
        b.get_fields_pitched(out, which)
        np.testing.assert_array_equal(out[:, :wl.ncell], a.get_fields(which))
        assert np.all(out[:, wl.ncell:] == -7.0)
    with pytest.raises(B.DfvError):
        b.set_fields_pitched(padded[:, : wl.ncell - 1].copy())


@pytest.mark.parametrize("pitched", [False, True])
def test_page_locked_and_device_fields_match_pageable(pitched):
    """Fields in page-locked host memory or on the device are converted in
    place (no staging copy): the same bits in and out as pageable host
    memory, packed or with padded planes (the padding untouched)."""
    import torch
    wl = W.random_state(2, (37, 23), 2, False, seed=42)
    nv = wl.prim.shape[0]
    pitch = wl.ncell + (13 if pitched else 0)

    def padded(fill, **kw):
        return torch.full((nv, pitch), fill, dtype=torch.float64, **kw)

    L = B.load()
    ref = B.Grid.from_workload(wl, precision=B.DFV_FP32)
    ref.step(2e-7)
    grids = []
    for kind in ("pinned", "device"):
        buf = padded(float("nan"), pin_memory=True) if kind == "pinned" else padded(float("nan"), device="cuda")
        buf[:, :wl.ncell] = torch.from_numpy(wl.prim)
        g = B.Grid.from_workload(wl, precision=B.DFV_FP32)
        ptr = B._vp(buf.data_ptr())
        if pitched:
            B._check(L.dfv_set_fields_pitched(g._h, ptr, pitch, int(kind == "device")), g._h, "set pitched")
        else:
            B._check(L.dfv_set_fields(g._h, ptr, int(kind == "device")), g._h, "set")
        g.step(2e-7)
        grids.append((kind, g))
    for which in (B.DFV_FIELDS_CONSERVED, B.DFV_FIELDS_PRIMITIVE):
        want = ref.get_fields(which)
        for kind, g in grids:
            out = padded(-7.0, pin_memory=True) if kind == "pinned" else padded(-7.0, device="cuda")
            ptr = B._vp(out.data_ptr())
            if pitched:
                B._check(L.dfv_get_fields_pitched(g._h, ptr, pitch, which, int(kind == "device")), g._h, "get")
            else:
                B._check(L.dfv_get_fields(g._h, ptr, which, int(kind == "device")), g._h, "get")
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            np.testing.assert_array_equal(got[:, :wl.ncell], want, err_msg=kind)
            assert np.all(got[:, wl.ncell:] == -7.0), kind
