"""The allocation-free entry point tdpd_pair_forces_noalloc.

Some callers cannot allocate device memory themselves -- a program whose pool
allocator owns the GPU, or a callback inside another engine's time step where
cudaMalloc would synchronise or is forbidden. This entry point serves them
with a fixed scratch array inside the library; here its forces and fluxes are
checked against the ordinary path (tdpd_commit + tdpd_read_forces) on two
calls in a row, which also exercises the reuse of the scratch between calls.
The file is named so that pytest collects it last.
"""

import numpy as np
import pytest

import workloads as W
from gpu_common import B, make, normwise, TOL_FORCE

pytestmark = pytest.mark.gpu


def _noalloc_forces(desc, step=0):
    import torch
    bd = B()
    pos, vel, conc, typ, _ = W.flat_state(desc)
    n, ns, T = pos.shape[0], int(desc['n_species']), int(desc['n_types'])
    dev = torch.device('cuda', torch.cuda.current_device())
    tp = torch.from_numpy(pos).to(dev)
    tv = torch.from_numpy(vel).to(dev)
    tc = torch.from_numpy(conc).to(dev)
    tt = torch.from_numpy(typ).to(dev)
    tf = torch.full((n, 3), float('nan'), device=dev)
    tq = torch.full((n, ns), float('nan'), device=dev)
    pair = np.stack([desc['a'], desc['gamma'], desc['sigma']], axis=-1).reshape(T * T * 3)
    stream = torch.cuda.current_stream()
    bd.tdpd_pair_forces_noalloc(bd.config_from(desc), pair, desc['kappa'].reshape(-1), n,
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
    # two different systems in a row: the second call must not see the first
    # call's leftovers in the shared scratch
    first = W.fluid_box(L=8.0, rho=3.0, n_species=2, seed=31)
    second = W.fluid_box(L=9.0, rho=4.0, n_species=1, seed=32)
    second['body_force'][:] = [0.05, 0.0, 0.0]
    for desc in (first, second):
        F, Q = _noalloc_forces(desc)
        Fr, Qr = _reference_forces(desc)
        assert np.isfinite(F).all() and np.isfinite(Q).all()
        assert normwise(F, Fr) < TOL_FORCE
        assert normwise(Q, Qr) < TOL_FORCE


def test_noalloc_rejects_sizes_beyond_its_limits():
    bd = B()
    big = W.fluid_box(L=20.0, rho=3.0, seed=33)          # 24,000 particles > 16,384
    cfg = bd.config_from(big)
    pair = np.zeros(3, np.float32)
    kap = np.ones(1, np.float32)
    with pytest.raises(bd.TdpdError) as e:
        bd.tdpd_pair_forces_noalloc(cfg, pair, kap, 24000, 1, 1, 1, 1, 0, 1, 1)
    assert e.value.status == 1
