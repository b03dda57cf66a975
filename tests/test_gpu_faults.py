"""Failure detection on the device, with every fault made on the host: a
replica whose pair coefficients overflow binary32 (non-finite forces) and a
replica whose loaded state overflows its neighbour lists. Each is reported in
its own status word, the faulted replica is quarantined (not moved, not
re-evaluated), and the other replicas of the batch step on with the same bits
as when they run alone. Nothing here faults, traps or hangs the GPU: the
kernels bound every list write by the capacity and only set status bits."""

import numpy as np
import pytest

import workloads as W
from gpu_common import B

pytestmark = pytest.mark.gpu

ENONFINITE, EOVERFLOW = 5, 4


def _alone(bd, desc, lanes, steps):
    h = bd.create_from(dict(desc, lanes=lanes))
    try:
        bd.tdpd_commit(h)
        bd.tdpd_step(h, steps)
        return bd.tdpd_read_state(h, 0, 1) + bd.tdpd_read_forces(h, 0, 1)
    finally:
        bd.tdpd_destroy(h)


def _same(a, b):
    return all(np.array_equal(x, y) for x, y in zip(a, b))


@pytest.mark.parametrize('sort_mode', [1, 2])
def test_non_finite_replica_is_reported_and_quarantined(sort_mode):
    """(With the list-mode sort as the kernel chain and as one cluster.)"""
    bd = B()
    reps = W.replica_ensemble(n_rep=4, seed=301, side_lo=8, side_hi=10)
    bad = 2
    reps[bad]['a'][:] = np.float32(3e38)            # one pair term is already near binary32's maximum
    hs = [bd.create_from(r) for r in reps]
    batch = bd.tdpd_batch_create(hs)
    try:
        bd.tdpd_set_lanes(batch, 4)
        bd.tdpd_set_sort_mode(batch, sort_mode)
        bd.tdpd_commit(batch)
        st = bd.tdpd_replica_status(batch)
        assert list(st) == [0, 0, ENONFINITE, 0]
        with pytest.raises(bd.TdpdError) as e:
            bd.tdpd_sync(batch)
        assert e.value.status == ENONFINITE and 'replica 2' in str(e.value)
        held = bd.tdpd_read_state(batch, bad, 1)
        bd.tdpd_step(batch, 6)
        assert list(bd.tdpd_replica_status(batch)) == [0, 0, ENONFINITE, 0]
        # quarantined: the faulted replica did not move
        assert _same(bd.tdpd_read_state(batch, bad, 1), held)
        # the others are unaffected, bit for bit
        for k in (0, 1, 3):
            got = bd.tdpd_read_state(batch, k, 1) + bd.tdpd_read_forces(batch, k, 1)
            assert _same(got, _alone(bd, reps[k], 4, 6)), k
            assert np.isfinite(got[0]).all()
    finally:
        bd.tdpd_destroy(batch)
        for h in hs:
            bd.tdpd_destroy(h)


@pytest.mark.parametrize('sort_mode', [1, 2])
def test_list_overflow_is_reported_not_silent(sort_mode):
    """The lists are sized at commit (1.5 x the longest, plus 16). A state
    loaded into one replica with every particle squeezed into one eighth of
    its box (eight times the density) needs longer lists: the build stops at
    the capacity, the replica reports TDPD_EOVERFLOW and is quarantined, and
    the other replicas continue exactly as alone."""
    bd = B()
    reps = W.replica_ensemble(n_rep=3, seed=303, side_lo=9, side_hi=11, max_rbc=0)
    hs = [bd.create_from(r) for r in reps]
    batch = bd.tdpd_batch_create(hs)
    try:
        bd.tdpd_set_lanes(batch, 4)
        bd.tdpd_set_sort_mode(batch, sort_mode)
        bd.tdpd_commit(batch)
        assert (bd.tdpd_replica_status(batch) == 0).all()
        x, v, c = bd.tdpd_read_state(batch, 1, 1)
        squeezed = (x * np.float32(0.5)).astype(np.float32)
        bd.tdpd_set_state(batch, 1, squeezed, v, c)
        assert list(bd.tdpd_replica_status(batch)) == [0, EOVERFLOW, 0]
        with pytest.raises(bd.TdpdError) as e:
            bd.tdpd_sync(batch)
        assert e.value.status == EOVERFLOW
        held = bd.tdpd_read_state(batch, 1, 1)
        assert np.array_equal(held[0], squeezed)
        bd.tdpd_step(batch, 5)
        assert list(bd.tdpd_replica_status(batch)) == [0, EOVERFLOW, 0]
        assert _same(bd.tdpd_read_state(batch, 1, 1), held)
        for k in (0, 2):
            assert _same(bd.tdpd_read_state(batch, k, 1) + bd.tdpd_read_forces(batch, k, 1),
                         _alone(bd, reps[k], 4, 5)), k
        # loading a sound state clears the status and the replica steps again
        bd.tdpd_set_state(batch, 1, x, v, c)
        assert (bd.tdpd_replica_status(batch) == 0).all()
        bd.tdpd_step(batch, 2)
        assert not np.array_equal(bd.tdpd_read_state(batch, 1, 1)[0], x)
        assert (bd.tdpd_replica_status(batch) == 0).all()
    finally:
        bd.tdpd_destroy(batch)
        for h in hs:
            bd.tdpd_destroy(h)


def test_quarantine_in_cell_mode():
    """Cell mode (no lists, every particle re-binned each step): a faulted
    replica is binned where it stands and keeps its state; the others match
    their runs alone."""
    bd = B()
    reps = W.replica_ensemble(n_rep=3, seed=305, side_lo=8, side_hi=9, max_rbc=0)
    reps[0]['a'][:] = np.float32(3e38)
    hs = [bd.create_from(dict(r, skin=0.0)) for r in reps]
    batch = bd.tdpd_batch_create(hs)
    try:
        bd.tdpd_set_skin(batch, 0.0)
        bd.tdpd_set_lanes(batch, 2)
        bd.tdpd_commit(batch)
        assert list(bd.tdpd_replica_status(batch)) == [ENONFINITE, 0, 0]
        held = bd.tdpd_read_state(batch, 0, 1)
        bd.tdpd_step(batch, 4)
        assert _same(bd.tdpd_read_state(batch, 0, 1), held)
        for k in (1, 2):
            got = bd.tdpd_read_state(batch, k, 1) + bd.tdpd_read_forces(batch, k, 1)
            assert _same(got, _alone(bd, dict(reps[k], skin=0.0), 2, 4)), k
    finally:
        bd.tdpd_destroy(batch)
        for h in hs:
            bd.tdpd_destroy(h)


def test_commit_checks_eq4_fluctuation_dissipation():
    """Eq. 4 fixes sigma^2 = 2 kT gamma with one kT: a type pair with a
    different ratio, or with gamma > 0 and sigma = 0, is refused at commit."""
    bd = B()
    d = W.fluid_box(L=6.0, rho=3.0, seed=307)
    d2 = dict(d, n_types=2)
    for k in ('a', 'gamma', 'sigma'):
        d2[k] = np.full((2, 2), d[k][0, 0], np.float32)
    d2['kappa'] = np.ones((2, 2, 1), np.float32)
    d2['sigma'][0, 1] = d2['sigma'][1, 0] = np.float32(4.0)      # kT 16/9 instead of 1
    for bad in (d2, dict(d, sigma=np.zeros((1, 1), np.float32))):
        h = bd.create_from(bad)
        try:
            with pytest.raises(bd.TdpdError) as e:
                bd.tdpd_commit(h)
            assert e.value.status == 1 and 'Eq. 4' in str(e.value)
        finally:
            bd.tdpd_destroy(h)
