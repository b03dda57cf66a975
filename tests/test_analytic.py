"""The closed forms of the validations (tests/analytic.py) against
Crank-Nicolson solutions of the equations they solve (CPU)."""

import numpy as np
import pytest

from analytic import series, bessel_series

sla = pytest.importorskip('scipy.linalg')


def _crank_nicolson(A, b, u0, dt, nsteps):
    """u' = A u + b with A tridiagonal (dense here, the grids are small)."""
    n = len(u0)
    I = np.eye(n)
    M1, M2 = I - 0.5 * dt * A, I + 0.5 * dt * A
    lu = sla.lu_factor(M1)
    u = u0.copy()
    for _ in range(nsteps):
        u = sla.lu_solve(lu, M2 @ u + dt * b)
    return u


def test_stokes_startup_series_matches_finite_differences():
    """u_t = nu u_zz + f on (0, d), u = 0 at both walls, u(z, 0) = 0."""
    d, nu, f = 10.0, 6.0, 0.2
    n = 399
    h = d / (n + 1)
    z = h * np.arange(1, n + 1)
    A = (np.diag(-2.0 * np.ones(n)) + np.diag(np.ones(n - 1), 1) + np.diag(np.ones(n - 1), -1)) * nu / h ** 2
    b = np.full(n, f)
    u = np.zeros(n)
    t, dt = 0.0, 1e-3
    umax = f * d * d / (8 * nu)
    for t_next in (0.5, 2.0, 8.0):
        k = int(round((t_next - t) / dt))
        u = _crank_nicolson(A, b, u, dt, k)
        t = t_next
        assert np.max(np.abs(u - series(z, t, f, d, nu))) < 1e-3 * umax, t
    # the other half carries the opposite flow
    assert np.allclose(series(z + d, t, f, d, nu), -series(z, t, f, d, nu))


def test_bessel_series_matches_radial_diffusion():
    """C_t = D (C_rr + C_r / r) on [0, R), C(R) = 1, C(r, 0) = 0, C_r(0) = 0:
    the series of Eq. 17 (C0 = 0, CD = 1)."""
    R, D = 5.0, 2.0
    n = 400
    h = R / n
    r = h * np.arange(n)                      # nodes 0 .. R - h; C(R) = 1 is the boundary
    A = np.zeros((n, n))
    b = np.zeros(n)
    A[0, 0], A[0, 1] = -4.0 * D / h ** 2, 4.0 * D / h ** 2   # symmetric node at the axis
    for i in range(1, n):
        lo = D / h ** 2 * (1.0 - h / (2 * r[i]))
        hi = D / h ** 2 * (1.0 + h / (2 * r[i]))
        A[i, i] = -2.0 * D / h ** 2
        A[i, i - 1] = lo
        if i + 1 < n:
            A[i, i + 1] = hi
        else:
            b[i] = hi * 1.0
    u = np.zeros(n)
    t, dt = 0.0, 2e-4
    for t_next in (0.2, 1.0, 3.0):
        k = int(round((t_next - t) / dt))
        u = _crank_nicolson(A, b, u, dt, k)
        t = t_next
        ref = bessel_series(r, t, D, R)
        assert np.max(np.abs(u - ref)) < 2e-3, (t, np.max(np.abs(u - ref)))
