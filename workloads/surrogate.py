"""Seeded inputs of the surrogate network: initial weights and the parameter
points whose simulated outcomes form its data set (inputs only)."""

from __future__ import annotations

import math

import numpy as np

IN, HID, OUT = 4, 64, 2
SHAPES = [(HID, IN), (HID,), (HID, HID), (HID,), (OUT, HID), (OUT,)]
FAN_IN = [IN, IN, HID, HID, HID, HID]
NPARAM = sum(int(np.prod(s)) for s in SHAPES)


def init_params(seed, n_members=1):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights and biases, float32,
    one row per ensemble member."""
    rng = np.random.default_rng(np.random.SeedSequence(int(seed)))
    out = []
    for _ in range(n_members):
        parts = [rng.uniform(-1.0 / math.sqrt(f), 1.0 / math.sqrt(f), int(np.prod(s)))
                 for s, f in zip(SHAPES, FAN_IN)]
        out.append(np.concatenate(parts).astype(np.float32))
    return np.stack(out)


def sample_points(n, seed):
    """Parameter points: permeability log-uniform in [0.01, 1], body force
    U[0, 0.1], membranes per box 1..4, kappa log-uniform in [0.3, 3]."""
    rng = np.random.default_rng(np.random.SeedSequence(int(seed)))
    return dict(permeability=10.0 ** rng.uniform(-2.0, 0.0, n),
                body_force=rng.uniform(0.0, 0.1, n),
                n_rbc=rng.integers(1, 5, n),
                kappa=10.0 ** rng.uniform(math.log10(0.3), math.log10(3.0), n),
                seeds=rng.integers(1, 2**62, n))


def ensemble_points(n, seed, side_lo=8, side_hi=16, max_rbc=4):
    """Parameter points of the batched-ensemble configuration: cubic box side
    an integer in [side_lo, side_hi], 0..max_rbc membranes (clamped later to
    the box's non-overlapping slots), permeability log-uniform in [0.01, 1],
    body force U[0, 0.1], solvent kappa log-uniform in [0.3, 3]."""
    rng = np.random.default_rng(np.random.SeedSequence(int(seed)))
    return dict(L=rng.integers(side_lo, side_hi + 1, n).astype(np.float64),
                permeability=10.0 ** rng.uniform(-2.0, 0.0, n),
                body_force=rng.uniform(0.0, 0.1, n),
                n_rbc=rng.integers(0, max_rbc + 1, n),
                kappa=10.0 ** rng.uniform(math.log10(0.3), math.log10(3.0), n),
                seeds=rng.integers(1, 2**62, n))
