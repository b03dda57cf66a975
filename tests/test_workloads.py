"""The seeded input generators (CPU): each workload has the geometry, counts
and parameter values its description states, and is reproducible from its
seed."""

import math

import numpy as np
import pytest

import workloads as W


def test_cylinder_diffusion_layout():
    """Fluid uniform inside R at C0 with Maxwell velocities, frozen wall
    particles at rest in the shell R..R + r_cc at C_D, both at rho; the
    paper's size holds about 402,000 fluid particles."""
    R, Lx, rho = 5.0, 10.0, 4.0
    d = W.cylinder_diffusion(R=R, Lx=Lx, rho=rho, c0=0.25, cd=0.75, seed=5)
    p = d['particles']
    c = 0.5 * d['L'].astype(np.float64)
    rad = np.hypot(p['pos'][:, 1] - c[1], p['pos'][:, 2] - c[2])
    wall = p['type'] == W.WALL
    assert d['frozen_types'] == 1 << W.WALL
    assert float(d['cylinder_radius']) == R
    assert rad[~wall].max() < R and rad[wall].min() >= R * (1 - 1e-6) and rad[wall].max() < R + 1.58
    assert (~wall).sum() == round(rho * math.pi * R * R * Lx)
    assert wall.sum() == round(rho * math.pi * ((R + 1.58) ** 2 - R * R) * Lx)
    assert np.all(p['conc'][~wall] == np.float32(0.25)) and np.all(p['conc'][wall] == np.float32(0.75))
    assert np.all(p['vel'][wall] == 0.0)
    v = p['vel'][~wall].astype(np.float64)
    assert np.abs(v.mean(0)).max() < 1e-6
    assert v.var() == pytest.approx(1.0, rel=0.1)
    # x uniform along the cylinder, inside the box
    assert p['pos'][:, 0].min() >= 0.0 and p['pos'][:, 0].max() < Lx
    assert 2 * (R + 1.58) < d['L'][1] and 2 * (R + 1.58) < d['L'][2]
    # the paper's setup: R = 20, length 80, rho = 4
    assert round(4.0 * math.pi * 400.0 * 80.0) == 402124
    # reproducible
    e = W.cylinder_diffusion(R=R, Lx=Lx, rho=rho, c0=0.25, cd=0.75, seed=5)
    assert np.array_equal(e['particles']['pos'], p['pos'])


def test_double_poiseuille_and_fluid_box():
    d = W.double_poiseuille(L=10.0, rho=4.0, f=0.1, seed=3, Lxy=12.0)
    assert tuple(d['L']) == (12.0, 12.0, 10.0)
    assert d['body_force_flip'] == 1 and d['body_force'][0] == np.float32(0.1)
    assert float(d['rc']) == pytest.approx(1.58) and float(d['s_f']) == pytest.approx(0.41)
    assert d['particles']['pos'].shape[0] == round(4.0 * 12 * 12 * 10)
    f = W.fluid_box(L=10.0, rho=4.0, seed=1)
    assert f['particles']['pos'].shape[0] == 4000
    assert float(f['a'][0, 0]) == pytest.approx(75.0 / 4.0)
    assert float(f['sigma'][0, 0]) ** 2 == pytest.approx(2.0 * 4.5, rel=1e-6)


def test_replica_ensemble_sizes():
    """Cubic boxes of integer side in [8, 16] at rho = 3, at most four cells
    each, permeability in [0.01, 1], body force in [0, 0.1]."""
    reps = W.replica_ensemble(n_rep=32, seed=9)
    for d in reps:
        L = d['L']
        assert L[0] == L[1] == L[2] and 8 <= L[0] <= 16 and float(L[0]).is_integer()
        assert len(d['rbcs']) <= 4
        assert 0.0 <= float(d['body_force'][0]) <= 0.1
        n_free = d['particles']['pos'].shape[0]
        assert n_free == round(3.0 * float(L[0]) ** 3)
