"""Closed triangulated membrane meshes (inputs only).

A Fibonacci lattice of n points on the unit sphere is triangulated by its
convex hull (2n-4 triangles, 3n-6 edges for a closed genus-0 surface), with
every triangle ordered counter-clockwise seen from outside. The biconcave
cell is that triangulation mapped onto the Evans-Fung red-cell profile
(Evans & Fung 1972): z(rho) = +-D sqrt(1-rho^2) (a0 + a1 rho^2/4 + a2 rho^4/16)
with rho the normalised radius, a0=0.0518, a1=2.0026, a2=-4.491.
"""

from __future__ import annotations

import numpy as np


def fibonacci_sphere(n: int) -> np.ndarray:
    i = np.arange(n, dtype=np.float64) + 0.5
    z = 1.0 - 2.0 * i / n
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = np.pi * (3.0 - np.sqrt(5.0)) * i
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)


def _orient_outward(p: np.ndarray, tri: np.ndarray) -> np.ndarray:
    a, b, c = p[tri[:, 0]], p[tri[:, 1]], p[tri[:, 2]]
    nrm = np.cross(b - a, c - a)
    flip = np.einsum('ij,ij->i', nrm, a + b + c) < 0
    tri = tri.copy()
    tri[flip] = tri[flip][:, [0, 2, 1]]
    return tri


def sphere_mesh(n: int, radius: float = 1.0):
    from scipy.spatial import ConvexHull
    p = fibonacci_sphere(n)
    tri = ConvexHull(p).simplices.astype(np.int32)
    tri = _orient_outward(p, tri)
    return p * radius, tri.astype(np.int32)


def biconcave_mesh(n: int, diameter: float):
    """Vertices (n, 3) float64 centred at the origin, disc normal along z, and
    outward triangles (2n-4, 3) int32."""
    p, tri = sphere_mesh(n)
    rho2 = np.minimum(1.0, p[:, 0] ** 2 + p[:, 1] ** 2)
    a0, a1, a2 = 0.0518, 2.0026, -4.491
    half = diameter * np.sqrt(np.maximum(0.0, 1.0 - rho2)) * (
        a0 + a1 * rho2 / 4.0 + a2 * rho2 * rho2 / 16.0)
    out = np.empty_like(p)
    out[:, 0] = 0.5 * diameter * p[:, 0]
    out[:, 1] = 0.5 * diameter * p[:, 1]
    out[:, 2] = np.sign(p[:, 2]) * half
    return out, tri


def icosahedron(edge: float = 1.0):
    """Regular icosahedron with the given edge, outward triangles."""
    t = (1.0 + np.sqrt(5.0)) / 2.0
    v = np.array([[-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
                  [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
                  [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]], np.float64)
    v *= edge / 2.0
    from scipy.spatial import ConvexHull
    tri = ConvexHull(v).simplices.astype(np.int32)
    return v, _orient_outward(v, tri).astype(np.int32)


def edges_of(tri: np.ndarray) -> np.ndarray:
    e = np.concatenate([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [2, 0]]])
    e.sort(axis=1)
    return np.unique(e, axis=0)
