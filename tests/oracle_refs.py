"""Independent closed-form references used to pin the oracle (test code only):
the exact isothermal Riemann solution and the elliptical-drop ODE."""
from __future__ import annotations

import math

import numpy as np


def isothermal_riemann(rho_l, u_l, rho_r, u_r, c, xi):
    """Exact solution of isothermal gas dynamics (p = c^2 rho + const) at x/t = xi.

    Shock branch: u* = u_K -/+ c (rho* - rho_K) / sqrt(rho* rho_K);
    rarefaction branch: u* = u_K -/+ c ln(rho*/rho_K)."""
    def f(rho, rk):
        if rho > rk:
            return c * (rho - rk) / math.sqrt(rho * rk)
        return c * math.log(rho / rk)

    lo, hi = 1e-12, 1e12
    for _ in range(300):
        mid = math.sqrt(lo * hi)
        if f(mid, rho_l) + f(mid, rho_r) + (u_r - u_l) > 0:
            hi = mid
        else:
            lo = mid
    rs = math.sqrt(lo * hi)
    us = u_l - f(rs, rho_l)
    xi = np.asarray(xi, dtype=np.float64)
    rho = np.empty_like(xi)
    u = np.empty_like(xi)
    for k, x in enumerate(xi):
        if x <= us:   # left of the contact
            if rs > rho_l:
                s = u_l - c * math.sqrt(rs / rho_l)
                rho[k], u[k] = (rho_l, u_l) if x < s else (rs, us)
            else:
                head, tail = u_l - c, us - c
                if x < head:
                    rho[k], u[k] = rho_l, u_l
                elif x > tail:
                    rho[k], u[k] = rs, us
                else:
                    u[k] = x + c
                    rho[k] = rho_l * math.exp((u_l - u[k]) / c)
        else:
            if rs > rho_r:
                s = u_r + c * math.sqrt(rs / rho_r)
                rho[k], u[k] = (rho_r, u_r) if x > s else (rs, us)
            else:
                head, tail = u_r + c, us + c
                if x > head:
                    rho[k], u[k] = rho_r, u_r
                elif x < tail:
                    rho[k], u[k] = rs, us
                else:
                    u[k] = x - c
                    rho[k] = rho_r * math.exp((u[k] - u_r) / c)
    return rho, u


def drop_semi_axes(t_end: float, a0: float = 100.0, nsub: int = 20000):
    """Free incompressible elliptical drop with velocity (-A x, A y): the pressure
    p0(t)(1 - x^2/a^2 - y^2/b^2) in Euler's equations gives
    A' = A^2 (a^2 - b^2)/(a^2 + b^2), a' = -A a, b' = A b (classical RK4)."""
    def rhs(y):
        A, a, b = y
        return np.array([A * A * (a * a - b * b) / (a * a + b * b), -A * a, A * b])

    y = np.array([a0, 1.0, 1.0])
    h = t_end / nsub
    for _ in range(nsub):
        k1 = rhs(y)
        k2 = rhs(y + 0.5 * h * k1)
        k3 = rhs(y + 0.5 * h * k2)
        k4 = rhs(y + h * k3)
        y = y + h / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
    return y[1], y[2]


def read_golden(name):
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", name)
    rows = []
    with open(path) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append(line.split())
    return rows
