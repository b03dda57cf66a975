"""Closed-form solutions the flow and transport validations compare with,
checked on the CPU against finite-difference solutions of the same
equations (tests/test_analytic.py)."""

import math

import numpy as np
import pytest


def series(z, t, f, d, nu, terms=60):
    """Mean flow u_x(z, t) of the double Poiseuille start-up (body force +f
    below z = d, -f above, period 2d, fluid at rest at t = 0): in each half
    the Stokes start-up of a channel with no-slip walls at 0 and d."""
    zz = np.mod(z, 2 * d)
    sign = np.where(zz < d, 1.0, -1.0)
    zz = np.where(zz < d, zz, zz - d)
    u = f * zz * (d - zz) / (2 * nu)
    for k in range(terms):
        n = 2 * k + 1
        u -= 4 * f * d * d / (nu * math.pi ** 3) * np.sin(n * math.pi * zz / d) * \
            math.exp(-n * n * math.pi ** 2 * nu * t / (d * d)) / n ** 3
    return sign * u


def bessel_series(r, t, D, R, terms=80):
    """(C - C0)/(CD - C0) of Eq. 17 for a cylinder of radius R started at C0
    with the surface held at CD."""
    sp = pytest.importorskip('scipy.special')
    lam = sp.jn_zeros(0, terms) / R
    out = np.ones_like(r, dtype=np.float64)
    for l in lam:
        out -= 2.0 / R * sp.j0(l * r) / (l * sp.j1(l * R)) * math.exp(-D * l * l * t)
    return out
