"""Shared helpers of the GPU parity tests: load a workload into libtdpd and
into the oracle, and compare the two with the tolerances of the tests."""

import numpy as np

import oracle
import workloads as W

# per-step force and flux: normwise relative
TOL_FORCE = 1e-5
# trajectories after 10 steps: normwise relative (positions: relative to the
# displacement over the run)
TOL_TRAJ = 1e-4


def B():
    from paper_1611_06163_gb300 import binding
    return binding


def make(desc):
    bd = B()
    h = bd.create_from(desc)
    bd.tdpd_commit(h)
    return h


def normwise(x, ref):
    x = np.asarray(x, np.float64)
    ref = np.asarray(ref, np.float64)
    d = np.linalg.norm(ref)
    return float(np.linalg.norm(x - ref) / (d if d > 0 else 1.0))


def elementwise(x, ref):
    """max_i |x_i - ref_i| / (|ref_i| + rms(ref))"""
    x = np.asarray(x, np.float64)
    ref = np.asarray(ref, np.float64)
    rms = np.sqrt(np.mean(ref ** 2)) if ref.size else 1.0
    return float(np.max(np.abs(x - ref) / (np.abs(ref) + rms))) if ref.size else 0.0


def wrap_diff(a, b, L):
    d = np.asarray(a, np.float64) - np.asarray(b, np.float64)
    L = np.asarray(L, np.float64)
    return d - L * np.round(d / L)


def forces_vs_oracle(desc, h=None, mode=1):
    bd = B()
    own = h is None
    if own:
        h = make(desc)
    try:
        ns = int(desc['n_species'])
        F, Q = bd.tdpd_read_forces(h, 0, ns)
    finally:
        if own:
            bd.tdpd_destroy(h)
    o = oracle.Oracle(desc, mode=mode)
    return F, Q, o.F, o.Q


def run_vs_oracle(desc, nsteps, mode=1):
    bd = B()
    h = make(desc)
    try:
        ns = int(desc['n_species'])
        pos0, _, _ = bd.tdpd_read_state(h, 0, ns)
        bd.tdpd_step(h, nsteps)
        bd.tdpd_sync(h)
        pos, vel, conc = bd.tdpd_read_state(h, 0, ns)
        F, Q = bd.tdpd_read_forces(h, 0, ns)
        obs = bd.tdpd_read_observables(h, 0)
        A, V = bd.tdpd_read_rbc(h, 0, len(desc['rbcs']))
    finally:
        bd.tdpd_destroy(h)
    o = oracle.Oracle(desc, mode=mode)
    o.run(nsteps)
    L = desc['L']
    disp = wrap_diff(o.pos, pos0, L)
    err = dict(
        pos=float(np.linalg.norm(wrap_diff(pos, o.pos, L)) / np.linalg.norm(disp)),
        vel=normwise(vel, o.vel),
        conc=normwise(conc, o.conc),
        force=normwise(F, o.F),
        flux=normwise(Q, o.Q),
    )
    return err, obs, o, (A, V)


__all__ = ['B', 'make', 'normwise', 'elementwise', 'wrap_diff', 'forces_vs_oracle', 'run_vs_oracle',
           'TOL_FORCE', 'TOL_TRAJ', 'W', 'oracle']
