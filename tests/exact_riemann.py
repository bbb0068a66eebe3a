"""Exact solution of the 1-D Riemann problem for stiffened gases (ideal gas:
p_inf = 0), written for the tests from the textbook construction: with
pbar = p + p_inf each side behaves like an ideal gas in pbar, the star
pressure solves f_L(p) + f_R(p) + u_R - u_L = 0 with the shock / rarefaction
branches of f_K, and the self-similar solution is sampled at x/t.

Independent of the oracle: no import from oracle/ or from the library."""
import math

import numpy as np


class Side:
    def __init__(self, rho, u, p, gamma, pinf=0.0):
        self.rho, self.u, self.p, self.g, self.pinf = rho, u, p, gamma, pinf
        self.c = math.sqrt(gamma * (p + pinf) / rho)

    def f(self, p):
        g, pb, pK = self.g, p + self.pinf, self.p + self.pinf
        if p > self.p:  # shock
            A = 2.0 / ((g + 1.0) * self.rho)
            B = (g - 1.0) / (g + 1.0) * pK
            return (pb - pK) * math.sqrt(A / (pb + B))
        return 2.0 * self.c / (g - 1.0) * ((pb / pK) ** ((g - 1.0) / (2.0 * g)) - 1.0)


def star_state(L: Side, R: Side):
    def F(p):
        return L.f(p) + R.f(p) + R.u - L.u
    lo = max(-L.pinf, -R.pinf) + 1e-12 * max(L.p + L.pinf, R.p + R.pinf)
    hi = 10.0 * max(L.p + L.pinf, R.p + R.pinf)
    while F(hi) < 0.0:
        hi *= 10.0
    for _ in range(400):
        mid = 0.5 * (lo + hi)
        if F(mid) > 0.0:
            hi = mid
        else:
            lo = mid
    ps = 0.5 * (lo + hi)
    us = 0.5 * (L.u + R.u) + 0.5 * (R.f(ps) - L.f(ps))
    return ps, us


def sample(L: Side, R: Side, xi: np.ndarray):
    """(rho, u, p, side) at similarity coordinates xi = (x - x0)/t; side is 0
    for material of the left state, 1 for the right."""
    ps, us = star_state(L, R)
    rho = np.zeros_like(xi)
    u = np.zeros_like(xi)
    p = np.zeros_like(xi)
    side = np.zeros_like(xi)
    for i, s in enumerate(xi):
        if s <= us:
            K, sgn = L, -1.0
        else:
            K, sgn = R, 1.0
        side[i] = 0.0 if s <= us else 1.0
        g, pinf = K.g, K.pinf
        pb, pK = ps + pinf, K.p + pinf
        if ps > K.p:  # shock on this side
            ratio = pb / pK
            rs = K.rho * (ratio + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ratio + 1)
            S = K.u + sgn * K.c * math.sqrt((g + 1) / (2 * g) * ratio + (g - 1) / (2 * g))
            if (sgn < 0 and s <= S) or (sgn > 0 and s >= S):
                rho[i], u[i], p[i] = K.rho, K.u, K.p
            else:
                rho[i], u[i], p[i] = rs, us, ps
        else:  # rarefaction
            rs = K.rho * (pb / pK) ** (1.0 / g)
            cs = K.c * (pb / pK) ** ((g - 1) / (2 * g))
            head = K.u + sgn * K.c
            tail = us + sgn * cs
            if (sgn < 0 and s <= head) or (sgn > 0 and s >= head):
                rho[i], u[i], p[i] = K.rho, K.u, K.p
            elif (sgn < 0 and s >= tail) or (sgn > 0 and s <= tail):
                rho[i], u[i], p[i] = rs, us, ps
            else:
                uf = 2.0 / (g + 1) * (-sgn * K.c + (g - 1) / 2 * K.u + s)
                cf = -sgn * (uf - s) if sgn < 0 else (s - uf)
                cf = abs(uf - s)
                pf = pK * (cf / K.c) ** (2 * g / (g - 1)) - pinf
                rf = K.rho * (cf / K.c) ** (2.0 / (g - 1))
                rho[i], u[i], p[i] = rf, uf, pf
    return rho, u, p, side
