"""Parameter sweeps steered by the surrogate network.

The simulator (the batched tDPD + RBC step through the C ABI) produces the
outcomes a sweep asks for; the network (tdpd_mlp_*) learns them from
simulated points and predicts new ones; a prediction whose ensemble spread
exceeds the threshold falls back to the plain simulation, which stays the
judge of the network's error.

Point -> features: permeability (membrane-solvent kappa), body force,
haematocrit (membrane volume fraction), solvent diffusivity (solvent kappa,
to which the Fickian diffusivity of Eq. 9 is proportional).
Point -> outcomes: mean release rate of species 0 from the membranes
(fraction of the initial membrane amount per unit time, 0 without
membranes) and the final mean concentration of the solvent.

A point set carries its box side per point ('L', the batched ensemble's
cubic boxes of side 8..16) or, without it, the 10^3 box of the quick sweep.
"""

from __future__ import annotations

import functools

import numpy as np

import workloads as W
from workloads.surrogate import ensemble_points, init_params, sample_points

from . import binding as bd

BOX = 10.0
RBC_DIAMETER = 5.0


@functools.lru_cache(maxsize=4)
def _mesh(diameter):
    return W.biconcave_mesh(500, diameter)


def _side(point, k):
    return float(point['L'][k]) if 'L' in point else BOX


def replica(point, k):
    """Workload of point k: a periodic box of the point's side at density 3
    with its number of membranes (clamped to the box's slots), permeability,
    body force and solvent kappa."""
    L = _side(point, k)
    rng = np.random.default_rng(np.random.SeedSequence(int(point['seeds'][k])))
    d = W._base('sweep', (L, L, L), (1, 1, 1), 2, 1, int(point['seeds'][k]), 3.0, dt=W.MEMBRANE_DT)
    d['particles'] = W.fluid_particles(rng, d['L'], 3.0, 1)
    d['particles']['conc'][:] = 0.0
    verts, tri = _mesh(RBC_DIAMETER)
    thick = float(verts[:, 2].max() - verts[:, 2].min())
    sxy = int(L // (RBC_DIAMETER + 1.0))
    sz = int(L // (thick + 1.0))
    slots = [(i, j, kk) for kk in range(sz) for j in range(sxy) for i in range(sxy)]
    for s in slots[:min(int(point['n_rbc'][k]), len(slots))]:
        c = ((s[0] + 0.5) * L / sxy, (s[1] + 0.5) * L / sxy, (s[2] + 0.5) * L / sz)
        d['rbcs'].append(W.place_rbc(verts, tri, c, d['L'], rng))
    kap = d['kappa']
    kap[W.SOLVENT, W.SOLVENT, 0] = point['kappa'][k]
    kap[W.SOLVENT, W.MEMBRANE, 0] = kap[W.MEMBRANE, W.SOLVENT, 0] = point['permeability'][k]
    d['body_force'] = np.asarray([point['body_force'][k], 0.0, 0.0], np.float32)
    d['membrane'] = W.membrane_defaults()
    return d


def rbc_volume():
    v, t = _mesh(RBC_DIAMETER)
    a, b, c = v[t[:, 0]], v[t[:, 1]], v[t[:, 2]]
    return float(np.einsum('ij,ij->i', a, np.cross(b, c)).sum() / 6.0)


def features(point, idx=None):
    idx = np.arange(len(point['permeability'])) if idx is None else np.asarray(idx)
    L = np.array([_side(point, int(k)) for k in idx])
    n_rbc = np.minimum(point['n_rbc'][idx], [_slots(x) for x in L])
    hct = n_rbc * rbc_volume() / L ** 3
    return np.stack([point['permeability'][idx], point['body_force'][idx], hct, point['kappa'][idx]],
                    1).astype(np.float32)


def _slots(L=BOX):
    verts, _ = _mesh(RBC_DIAMETER)
    thick = float(verts[:, 2].max() - verts[:, 2].min())
    return int(L // (RBC_DIAMETER + 1.0)) ** 2 * int(L // (thick + 1.0))


def simulate(point, idx, steps, stream_ptr=None):
    """Run the points idx as one batch for `steps` steps; returns outcomes
    (n, 2): release rate, final solvent concentration (NaN for a replica whose
    status reports a fault: it was quarantined and its outcome is not kept)."""
    idx = np.asarray(idx)
    descs = [replica(point, int(k)) for k in idx]
    hs = [bd.create_from(d) for d in descs]
    batch = bd.tdpd_batch_create(hs)
    for h in hs:
        bd.tdpd_destroy(h)
    try:
        if stream_ptr:
            bd.tdpd_set_stream(batch, stream_ptr)
        # one lane per particle and the half shell, pinned: a replica then gives
        # the same bits in any batch, so a point simulated again (a fallback)
        # reproduces its recorded outcome exactly
        bd.tdpd_set_lanes(batch, 1)
        bd.tdpd_set_pair_mode(batch, 2)
        bd.tdpd_commit(batch)
        before = [bd.tdpd_read_observables(batch, r) for r in range(len(descs))]
        bd.tdpd_step(batch, steps)
        status = bd.tdpd_replica_status(batch)
        after = [bd.tdpd_read_observables(batch, r) for r in range(len(descs))]
    finally:
        bd.tdpd_destroy(batch)
    t = steps * float(np.float32(descs[0]['dt']))
    out = np.zeros((len(idx), 2))
    for r, (a, b) in enumerate(zip(before, after)):
        if status[r] != 0:                 # the replica went non-finite
            out[r] = np.nan
            continue
        m0 = a['mass_membrane'][0]
        out[r, 0] = (m0 - b['mass_membrane'][0]) / (m0 * t) if m0 > 0 else 0.0
        out[r, 1] = (b['mass'][0] - b['mass_membrane'][0]) / (b['n_particles'] - b['n_membrane'])
    return out


class Surrogate:
    """An ensemble network trained on simulated outcomes."""

    def __init__(self, members=5, seed=0):
        self.members = members
        self.h = bd.tdpd_mlp_create(members)
        bd.tdpd_mlp_set_params(self.h, init_params(seed, members))

    def fit(self, X, Y, steps=2000, lr=3e-3):
        bd.tdpd_mlp_set_data(self.h, X, Y)
        return bd.tdpd_mlp_train(self.h, steps, lr, self.members)

    def predict(self, X):
        mean, spread, _ = bd.tdpd_mlp_predict(self.h, X, self.members)
        return mean, spread

    def close(self):
        bd.tdpd_mlp_destroy(self.h)
        self.h = None


def predict_with_fallback(model, point, idx, steps, threshold=0.05):
    """Network prediction for points idx; a point whose relative ensemble
    spread exceeds `threshold` on either output is simulated instead.
    Returns (values, fell_back mask)."""
    X = features(point, idx)
    mean, spread = model.predict(X)
    fell = (spread > threshold).any(axis=1)
    vals = mean.astype(np.float64)
    if fell.any():
        vals[fell] = simulate(point, np.asarray(idx)[fell], steps)
    return vals, fell


__all__ = ['sample_points', 'ensemble_points', 'replica', 'features', 'simulate', 'Surrogate',
           'predict_with_fallback']
