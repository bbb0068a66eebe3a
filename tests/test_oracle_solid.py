"""Pins of the oracle's elastoplastic path (Sec. 2.1): the longitudinal
elastic wave speed sqrt((K + 4G/3)/rho) of a small-amplitude wave, and the
Hugoniot elastic limit (K/(2G) + 2/3) sigma_Y of the elastic precursor in a
symmetric impact with perfect plasticity.  CPU only (1-D, 800 cells)."""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from oracle import Oracle

AL = W.ALUMINIUM
N = 800


def impact(uL, uR, t_end):
    o = Oracle(1, (N,), (0.0,), (1.0,), [AL], solid=True)
    x = (np.arange(N) + 0.5) / N
    w = np.zeros((7, N))
    w[0] = AL["rho0"]
    w[1] = np.where(x < 0.5, uL, uR)
    w[2] = 1e5
    w[3:6] = 1.0
    o.set_prim(w)
    t = 0.0
    while t < t_end * (1 - 1e-13):
        dt = min(o.compute_dt(0.6), t_end - t)
        o.step(dt)
        t += dt
    return x, o


def sigma_xx(o):
    wp, q = o.prim(), o.cons()
    out = np.zeros(N)
    for c in range(N):
        dH, _ = oracle.vbar_log(np.diag(wp[3:6, c]))
        cl = o.closure(q[:, c])
        out[c] = -cl["p"] + 2 * cl["G"] * dH[0, 0]   # tension positive
    return out


def test_elastic_wave_speed():
    t_end = 5e-5
    x, o = impact(1.0, 0.0, t_end)
    u = o.prim()[1]
    right = x > 0.5
    # front: where u falls through half of the 0.5 m/s particle-velocity jump
    i = np.where(right & (u < 0.25))[0][0]
    j = i - 1
    xf = x[j] + (x[i] - x[j]) * (u[j] - 0.25) / (u[j] - u[i])
    cL = math.sqrt((AL["K0"] + 4.0 / 3.0 * AL["G0"]) / AL["rho0"])
    assert (xf - 0.5) / t_end == pytest.approx(cL, rel=0.01)
    # particle velocity behind the front is half the jump (symmetric split)
    assert np.mean(u[(x > 0.55) & (x < 0.75)]) == pytest.approx(0.5, rel=0.01)


def test_hugoniot_elastic_limit_of_precursor():
    x, o = impact(100.0, -100.0, 6e-5)
    s = sigma_xx(o)
    hel = (AL["K0"] / (2 * AL["G0"]) + 2.0 / 3.0) * AL["sigY"]
    # the precursor plateau lies between the plastic and elastic fronts
    plateau = (x > 0.835) & (x < 0.855)
    assert np.ptp(s[plateau]) < 1e-3 * hel
    assert -np.mean(s[plateau]) == pytest.approx(hel, rel=0.03)
    # behind the plastic wave the stress is well above the HEL
    assert -np.mean(s[(x > 0.55) & (x < 0.75)]) > 2 * hel
