"""Small hand-built workloads for tests (inputs only, no method arithmetic)."""

import math
import os

import numpy as np

import workloads as W
from workloads.mesh import sphere_mesh, icosahedron

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), 'golden')


def read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith('#'):
                rows.append(line.split())
    return rows


def custom(pos, vel=None, conc=None, L=(10.0, 10.0, 10.0), periodic=(1, 1, 1), ns=1,
           a=25.0, gamma=4.5, sigma=3.0, rc=1.0, s_f=2.0, rcc=1.58, s_c=2.0, kappa=1.0,
           dt=0.01, seed=7, types=None, n_types=1, body_force=(0, 0, 0), frozen_types=0,
           reaction=None):
    pos = np.asarray(pos, np.float32).reshape(-1, 3)
    n = pos.shape[0]
    d = W._base('custom', L, periodic, n_types, ns, seed, 3.0, dt=dt, rc=rc, s_f=s_f,
                rcc=rcc, s_c=s_c, gamma=gamma)
    d['a'][:] = a
    d['gamma'][:] = gamma
    d['sigma'][:] = sigma
    d['kappa'][:] = kappa
    d['body_force'] = np.asarray(body_force, np.float32)
    d['frozen_types'] = frozen_types
    d['reaction'] = reaction
    d['particles'] = dict(
        pos=pos,
        vel=np.zeros((n, 3), np.float32) if vel is None else np.asarray(vel, np.float32).reshape(n, 3),
        conc=np.zeros((n, ns), np.float32) if conc is None else np.asarray(conc, np.float32).reshape(n, ns),
        type=np.zeros(n, np.int32) if types is None else np.asarray(types, np.int32))
    return d


def membrane_only(verts, tri, L=60.0, rest=None, vel=None, **mem):
    """A single membrane centred in a large periodic box, no free particles."""
    d = custom(np.zeros((0, 3)), L=(L, L, L), n_types=2)
    c = np.full(3, 0.5 * L)
    v = (np.asarray(verts, np.float64) + c).astype(np.float32)
    nv = v.shape[0]
    d['rbcs'] = [dict(pos=v, vel=np.zeros((nv, 3), np.float32) if vel is None else np.asarray(vel, np.float32),
                      conc=np.ones((nv, 1), np.float32), type=W.MEMBRANE,
                      tri=np.ascontiguousarray(tri, np.int32),
                      rest=None if rest is None else (np.asarray(rest, np.float64) + c).astype(np.float32))]
    p = W.membrane_defaults()
    p.update(mem)
    d['membrane'] = p
    return d


def small_sphere(n=42, radius=2.0):
    return sphere_mesh(n, radius)


def relerr(x, ref):
    x = np.asarray(x, np.float64)
    ref = np.asarray(ref, np.float64)
    den = np.linalg.norm(ref)
    return np.linalg.norm(x - ref) / (den if den > 0 else 1.0)


__all__ = ['custom', 'membrane_only', 'small_sphere', 'icosahedron', 'relerr', 'read_golden', 'math']
