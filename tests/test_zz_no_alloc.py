"""The allocation-free entry point tdpd_pair_forces_noalloc.

Some callers cannot allocate device memory themselves -- a program whose pool
allocator owns the GPU, or a callback inside another engine's time step where
cudaMalloc would synchronise or is forbidden. This entry point serves them
with a fixed scratch array inside the library; here its forces and fluxes are
checked against the ordinary path (tdpd_commit + tdpd_read_forces) on calls
in a row, which also exercises the reuse of the scratch between calls, and at
a nonzero step against both the ordinary path and the FP64 oracle. The file
is named so that pytest collects it last.
"""

import numpy as np
import pytest

import oracle
import workloads as W
from gpu_common import B, make, normwise, TOL_FORCE

pytestmark = pytest.mark.gpu


def _pair_table(desc):
    T = int(desc['n_types'])
    return np.stack([desc['a'], desc['gamma'], desc['sigma']], axis=-1).reshape(T * T * 3)


def _noalloc_forces(desc, step=0, state=None, types=None):
    import torch
    bd = B()
    pos, vel, conc, typ, _ = W.flat_state(desc)
    if state is not None:
        pos, vel, conc = state
    if types is not None:
        typ = np.asarray(types, np.int32)
    n, ns = pos.shape[0], int(desc['n_species'])
    dev = torch.device('cuda', torch.cuda.current_device())
    tp = torch.from_numpy(np.ascontiguousarray(pos, np.float32)).to(dev)
    tv = torch.from_numpy(np.ascontiguousarray(vel, np.float32)).to(dev)
    tc = torch.from_numpy(np.ascontiguousarray(conc, np.float32)).to(dev)
    tt = torch.from_numpy(typ).to(dev)
    tf = torch.full((n, 3), float('nan'), device=dev)
    tq = torch.full((n, ns), float('nan'), device=dev)
    stream = torch.cuda.current_stream()
    bd.tdpd_pair_forces_noalloc(bd.config_from(desc), _pair_table(desc), desc['kappa'].reshape(-1), n,
                                tp.data_ptr(), tv.data_ptr(), tc.data_ptr(), tt.data_ptr(), step,
                                tf.data_ptr(), tq.data_ptr(), stream.cuda_stream)
    stream.synchronize()
    return tf.cpu().numpy(), tq.cpu().numpy()


def _reference_forces(desc):
    bd = B()
    h = make(desc)
    try:
        return bd.tdpd_read_forces(h, 0, int(desc['n_species']))
    finally:
        bd.tdpd_destroy(h)


def test_noalloc_matches_forces_of_the_ordinary_path_twice():
    # different systems in a row (two, then three species: the latter runs the
    # pair kernel's general form): no call may see the previous call's
    # leftovers in the shared scratch
    first = W.fluid_box(L=8.0, rho=3.0, n_species=2, seed=31)
    second = W.fluid_box(L=9.0, rho=4.0, n_species=1, seed=32)
    second['body_force'][:] = [0.05, 0.0, 0.0]
    third = W.fluid_box(L=7.0, rho=3.0, n_species=3, seed=34)
    third['kappa'][...] = np.array([0.5, 1.0, 2.0], np.float32)
    for desc in (first, second, third):
        F, Q = _noalloc_forces(desc)
        Fr, Qr = _reference_forces(desc)
        assert np.isfinite(F).all() and np.isfinite(Q).all()
        assert normwise(F, Fr) < TOL_FORCE
        assert normwise(Q, Qr) < TOL_FORCE


def test_noalloc_at_a_nonzero_step_matches_ordinary_path_and_oracle():
    """The step number keys the pair random numbers: after 9 steps of the
    ordinary path, its state reloaded there (tdpd_set_state: forces at step 9
    with v~ = v) and the same state through this entry point with step 9 give
    the same forces, both within tolerance of the FP64 oracle at step 9; the
    same call with step 0 does not."""
    bd = B()
    desc = W.fluid_box(L=8.0, rho=3.0, n_species=2, seed=35)
    h = make(desc)
    try:
        bd.tdpd_step(h, 9)
        x, v, c = bd.tdpd_read_state(h, 0, 2)
        bd.tdpd_set_state(h, 0, x, v, c)
        Fr, Qr = bd.tdpd_read_forces(h, 0, 2)
    finally:
        bd.tdpd_destroy(h)
    F, Q = _noalloc_forces(desc, step=9, state=(x, v, c))
    o = oracle.Oracle(desc, mode=1)
    o.set_state(x, v, c, step=9)
    assert normwise(F, Fr) < TOL_FORCE and normwise(Q, Qr) < TOL_FORCE
    assert normwise(F, o.F) < TOL_FORCE and normwise(Q, o.Q) < TOL_FORCE
    F0, _ = _noalloc_forces(desc, step=0, state=(x, v, c))
    assert normwise(F0, o.F) > 1e-2


def test_noalloc_marks_bad_types_in_its_outputs():
    """A type outside [0, n_types) makes every output NaN (the call returns
    no device status); the next valid call is clean again."""
    desc = W.fluid_box(L=7.0, rho=3.0, n_species=1, seed=36)
    n = W.n_particles(desc)
    typ = np.zeros(n, np.int32)
    typ[17] = 3
    F, Q = _noalloc_forces(desc, types=typ)
    assert np.isnan(F).all() and np.isnan(Q).all()
    F, Q = _noalloc_forces(desc)
    Fr, Qr = _reference_forces(desc)
    assert normwise(F, Fr) < TOL_FORCE and normwise(Q, Qr) < TOL_FORCE


def test_noalloc_rejects_sizes_beyond_its_limits():
    bd = B()
    big = W.fluid_box(L=20.0, rho=3.0, seed=33)          # 24,000 particles > 16,384
    cfg = bd.config_from(big)
    pair = np.zeros(3, np.float32)
    kap = np.ones(1, np.float32)
    with pytest.raises(bd.TdpdError) as e:
        bd.tdpd_pair_forces_noalloc(cfg, pair, kap, 24000, 1, 1, 1, 1, 0, 1, 1)
    assert e.value.status == 1
    # a 30^3 box needs 37^3 > 16,384 cells of edge >= 1.58/2
    cfg = bd.config_from(W.fluid_box(L=30.0, rho=0.1, seed=33))
    with pytest.raises(bd.TdpdError) as e:
        bd.tdpd_pair_forces_noalloc(cfg, pair, kap, 100, 1, 1, 1, 1, 0, 1, 1)
    assert e.value.status == 1 and 'cells' in str(e.value)
    # five species exceed the limit of four
    d5 = W.fluid_box(L=7.0, rho=1.0, n_species=5, seed=33)
    with pytest.raises(bd.TdpdError) as e:
        bd.tdpd_pair_forces_noalloc(bd.config_from(d5), pair, np.ones(5, np.float32), 100, 1, 1, 1, 1, 0, 1, 1)
    assert e.value.status == 1 and 'species' in str(e.value)
    # the checks of tdpd_create: a non-finite box edge
    bad = W.fluid_box(L=7.0, rho=1.0, seed=33)
    cfg = bd.config_from(bad)
    cfg.L[1] = float('inf')
    with pytest.raises(bd.TdpdError) as e:
        bd.tdpd_pair_forces_noalloc(cfg, pair, kap, 100, 1, 1, 1, 1, 0, 1, 1)
    assert e.value.status == 1
