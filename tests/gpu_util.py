"""Helpers of the GPU parity tests: running the oracle and the CUDA library on
the same seeded workload and measuring per-plane relative L1 differences."""
import numpy as np

import workloads as W


def plane_scales(ref, wl):
    """Denominator of the relative L1 per conserved plane: sum |ref|, with
    momentum planes floored at sum(rho) * 10 m/s and stretch-tensor planes at
    ncell (|V| ~ 1), so that near-zero momenta and off-diagonal stretches are
    measured against a physical scale rather than round-off."""
    L = W.layout(wl.dim, wl.nmat, wl.solid)
    rho = ref[L["irho"]: L["irho"] + wl.nmat].sum(axis=0)
    s = np.abs(ref).sum(axis=1)
    for a in range(wl.dim):
        s[L["iu"] + a] = max(s[L["iu"] + a], 10.0 * np.abs(rho).sum())
    s[L["ir"]] = max(s[L["ir"]], 1e-3 * ref.shape[1])
    for c in range(L["nv"]):          # stretch components are O(1): measure against |V| ~ 1
        s[L["iv"] + c] = max(s[L["iv"] + c], 1.0 * ref.shape[1])
    for l in range(wl.nmat - 1):
        s[L["iphi"] + l] = max(s[L["iphi"] + l], 1e-3 * ref.shape[1])
    return np.where(s > 0, s, 1.0)


def rel_l1(got, ref, wl):
    return np.abs(got - ref).sum(axis=1) / plane_scales(ref, wl)


def run_both(wl, steps, precision, cfl=None, use_run=False, **variants):
    """Advance the oracle and the GPU grid `steps` steps with the oracle's dt
    (dfv_step) or the device-computed dt (dfv_run); returns (oracle, grid).
    variants: hllc_lm, seed_variant, given to both sides."""
    from oracle import Oracle
    from paper_2111_11806_gb300 import binding as B
    cfl = wl.cfl if cfl is None else cfl
    o = Oracle.from_workload(wl, **variants)
    g = B.Grid.from_workload(wl, precision=precision, **variants)
    if use_run:
        g.run(steps, cfl)
        for _ in range(steps):
            o.step(o.compute_dt(cfl))
    else:
        for _ in range(steps):
            dt = o.compute_dt(cfl)
            o.step(dt)
            g.step(dt)
    return o, g


def same_kernel_bits(got, ref, wl, precision):
    """Batch instance against the single-grid run of the same instance.  The
    batch and single-grid kernels are separate compilations of the same tile
    and seeding code, and the compiler may contract a product and a sum into
    one FMA in one and not the other, so they agree to rounding: relative L1
    per plane <= 1e-13 (FP64) or 1e-6 (FP32) after a few steps."""
    err = rel_l1(got, ref, wl)
    assert np.all(err <= (1e-13 if precision == 0 else 1e-6)), err
