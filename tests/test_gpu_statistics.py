"""Statistical agreement of long runs, GPU against the FP64 oracle.

Beyond ten steps the two trajectories drift apart (the dynamics amplify
rounding differences), so they are compared through the statistics they
sample: the temperature, the self-diffusion coefficient and the decay of a
concentration profile, each within 1 %. Both start from the same state with
the same random streams, on a fluid large enough (about 88,000 particles)
that each statistic is sampled to a few tenths of a per cent.
"""

import numpy as np
import pytest

import oracle
import workloads as W
from gpu_common import B, wrap_diff

pytestmark = pytest.mark.gpu

SNAP = 20           # steps between snapshots
NSNAP = 30          # 600 steps, t = 6


def _stats(pos_series, vel_series, conc_series, L):
    """Unwrapped displacements from successive snapshots (each well under half
    a box), temperature per snapshot, and the amplitude of the sin(2 pi x/L)
    mode of the concentration per snapshot."""
    L = np.asarray(L, np.float64)
    unwrapped = [np.asarray(pos_series[0], np.float64)]
    for a, b in zip(pos_series[:-1], pos_series[1:]):
        unwrapped.append(unwrapped[-1] + wrap_diff(b, a, L))
    kT = []
    for v in vel_series:
        v = np.asarray(v, np.float64)
        dv = v - v.mean(axis=0)
        kT.append(float((dv * dv).sum() / (3 * (len(v) - 1))))
    amp = []
    for p, c in zip(pos_series, conc_series):
        s = np.sin(2 * np.pi * np.asarray(p, np.float64)[:, 0] / L[0])
        amp.append(float(2.0 * np.mean(np.asarray(c, np.float64)[:, 0] * s)))
    return unwrapped, np.array(kT), np.array(amp)


def _msd_coefficient(unwrapped, dt_snap, t0s, lag):
    out = []
    for t0 in t0s:
        i0 = int(round(t0 / dt_snap))
        i1 = i0 + int(round(lag / dt_snap))
        d = unwrapped[i1] - unwrapped[i0]
        out.append(np.mean(np.sum(d * d, axis=1)) / (6.0 * lag))
    return float(np.mean(out))


def test_long_run_temperature_diffusion_and_concentration_profile():
    bd = B()
    L = 28.0
    d = W.fluid_box(L=L, rho=4.0, seed=81)                    # 87,808 particles, dt = 0.01
    p = d['particles']
    p['conc'][:, 0] = (0.5 + 0.4 * np.sin(2 * np.pi * p['pos'][:, 0].astype(np.float64) / L)).astype(np.float32)
    h = bd.create_from(d)
    bd.tdpd_commit(h)
    g_pos, g_vel, g_conc = [], [], []
    for k in range(NSNAP + 1):
        if k:
            bd.tdpd_step(h, SNAP)
        x, v, c = bd.tdpd_read_state(h, 0, 1)
        g_pos.append(x); g_vel.append(v); g_conc.append(c)
    st = bd.tdpd_replica_status(h)
    bd.tdpd_destroy(h)
    assert (st == 0).all()

    o = oracle.Oracle(d, mode=1)
    o_pos, o_vel, o_conc = [o.pos.copy()], [o.vel.copy()], [o.conc.copy()]
    for _ in range(NSNAP):
        o.run(SNAP)
        o_pos.append(o.pos.copy()); o_vel.append(o.vel.copy()); o_conc.append(o.conc.copy())

    dts = SNAP * float(np.float32(d['dt']))
    gu, gkT, gamp = _stats(g_pos, g_vel, g_conc, d['L'])
    ou, okT, oamp = _stats(o_pos, o_vel, o_conc, d['L'])
    # temperature over t in [2, 6] (after the random start has relaxed)
    i2 = int(round(2.0 / dts))
    assert gkT[i2:].mean() == pytest.approx(okT[i2:].mean(), rel=0.01)
    assert gkT[i2:].mean() == pytest.approx(1.0, rel=0.03)
    # self-diffusion from the mean squared displacement over a lag of 4
    Dg = _msd_coefficient(gu, dts, (1.6, 2.0), 4.0)
    Do = _msd_coefficient(ou, dts, (1.6, 2.0), 4.0)
    assert Dg == pytest.approx(Do, rel=0.01), (Dg, Do)
    # concentration profile: the sine mode decays; its amplitude at t = 2, 4, 6
    for t in (2.0, 4.0, 6.0):
        i = int(round(t / dts))
        assert gamp[i] == pytest.approx(oamp[i], rel=0.01), (t, gamp[i], oamp[i])
    assert gamp[-1] < 0.9 * gamp[0]


def test_rbc_area_and_volume_hold_at_targets_in_solvent():
    """The single-RBC workload on the device: over t = 5 to 10 the cell's
    FP64 area and volume stay within 1 % of the targets A0 and V0 of the
    oracle's membrane model (the cell starts 1.2 % above V0). The penalty of
    Eq. 14-15 is finite, so thermal undulations and the solvent hold the
    mean area about 0.5 % below A0."""
    bd = B()
    d = W.single_rbc(seed=91)
    o = oracle.Oracle(d, mode=1)
    _, _, A0, V0 = o.membrane_rest()
    h = bd.create_from(d)
    bd.tdpd_commit(h)
    bd.tdpd_step(h, 1000)                       # t = 5 at dt = 0.005
    A, V = [], []
    for _ in range(20):
        bd.tdpd_step(h, 50)
        a, v = bd.tdpd_read_rbc(h, 0, 1)
        A.append(a[0]); V.append(v[0])
    st = bd.tdpd_replica_status(h)
    bd.tdpd_destroy(h)
    assert (st == 0).all()
    assert abs(np.mean(A) - A0[0]) / A0[0] < 1e-2
    assert abs(np.mean(V) - V0[0]) / V0[0] < 1e-2
    assert np.max(np.abs(np.array(A) - A0[0])) / A0[0] < 2e-2
    assert np.max(np.abs(np.array(V) - V0[0])) / V0[0] < 2e-2


def test_benchmark_workloads_run_their_full_length():
    """The 512-replica ensemble and the RBC channel run 2000 steps (t = 10, the
    configured run length): every replica stays finite, each replica's
    temperature (relative to its mean flow) stays within 10 % of kT, solute is
    conserved (Fickian flux is pairwise antisymmetric; the channel's reaction
    A -> B keeps A + B), and every membrane keeps its area and volume within
    5 % of the targets."""
    bd = B()
    reps = W.replica_ensemble(n_rep=512, seed=1004)
    hs = [bd.create_from(r) for r in reps]
    h = bd.tdpd_batch_create(hs)
    bd.tdpd_commit(h)
    m0 = [bd.tdpd_read_observables(h, r)['mass'].sum() for r in range(len(reps))]
    bd.tdpd_step(h, 2000)
    st = bd.tdpd_replica_status(h)
    assert (st == 0).all()
    worst_a = worst_v = 0.0
    for r, d in enumerate(reps):
        ob = bd.tdpd_read_observables(h, r)
        assert ob['step'] == 2000
        assert abs(ob['kT'] - 1.0) < 0.1, (r, ob['kT'])
        assert abs(ob['mass'].sum() - m0[r]) <= 1e-4 * max(1.0, abs(m0[r])), r
        nb = len(d['rbcs'])
        if nb:
            o = oracle.Oracle(d, mode=1)
            _, _, A0, V0 = o.membrane_rest()
            A, V = bd.tdpd_read_rbc(h, r, nb)
            worst_a = max(worst_a, float(np.max(np.abs(A - A0) / A0)))
            worst_v = max(worst_v, float(np.max(np.abs(V - V0) / V0)))
    print('ensemble after 2000 steps: worst area %.4f, worst volume %.4f' % (worst_a, worst_v))
    assert worst_a < 0.05 and worst_v < 0.05
    bd.tdpd_destroy(h)
    for x in hs:
        bd.tdpd_destroy(x)

    d = W.rbc_channel()
    h = bd.create_from(d)
    bd.tdpd_commit(h)
    m0 = bd.tdpd_read_observables(h, 0)['mass'].sum()
    bd.tdpd_step(h, 2000)
    assert (bd.tdpd_replica_status(h) == 0).all()
    ob = bd.tdpd_read_observables(h, 0)
    assert abs(ob['kT'] - 1.0) < 0.1, ob['kT']
    assert abs(ob['mass'].sum() - m0) <= 1e-4 * max(1.0, abs(m0))
    o = oracle.Oracle(d, mode=1)
    _, _, A0, V0 = o.membrane_rest()
    A, V = bd.tdpd_read_rbc(h, 0, len(d['rbcs']))
    print('channel after 2000 steps: worst area %.4f, worst volume %.4f'
          % (np.max(np.abs(A - A0) / A0), np.max(np.abs(V - V0) / V0)))
    assert np.max(np.abs(A - A0) / A0) < 0.05 and np.max(np.abs(V - V0) / V0) < 0.05
    bd.tdpd_destroy(h)
