"""The FP64 reductions of the step, each against the FP64 oracle on the same
state: the device's totals of the device state (read back, binary32 values
exact in binary64) against the oracle's plain binary64 sums of that state.
Kinetic temperature, momentum and species totals come from k_observables
(binary32 terms, float-float sums, one binary64 combine); membrane area and
volume from the K-Gather (binary32 triangle terms relative to a reference
point, float-float sums). Each test prints its measured errors."""

import numpy as np
import pytest

import oracle
import workloads as W
from gpu_common import B, make

pytestmark = pytest.mark.gpu


def _errors(desc, steps):
    bd = B()
    ns = int(desc['n_species'])
    h = make(desc)
    try:
        bd.tdpd_step(h, steps)
        bd.tdpd_sync(h)
        x, v, c = bd.tdpd_read_state(h, 0, ns)
        obs = bd.tdpd_read_observables(h, 0)
        A, V = bd.tdpd_read_rbc(h, 0, len(desc['rbcs']))
    finally:
        bd.tdpd_destroy(h)
    o = oracle.Oracle(desc, mode=1)
    o.pos = np.ascontiguousarray(x, np.float64)
    o.vel = np.ascontiguousarray(v, np.float64)
    o.conc = np.ascontiguousarray(c, np.float64).reshape(o.n, o.ns)
    ob = o.observables()
    frozen = np.array([(desc['frozen_types'] >> int(t)) & 1 for t in W.flat_state(desc)[3]], bool)
    scale_p = np.abs(v[~frozen].astype(np.float64)).sum(axis=0)
    err = {
        'kT': abs(obs['kT'] - ob['kT']) / ob['kT'],
        'momentum': float(np.max(np.abs(obs['momentum'] - ob['momentum']) / scale_p)),
        'mass': float(np.max(np.abs(obs['mass'] - ob['mass']) / np.abs(ob['mass']).clip(1e-300))),
    }
    if len(desc['rbcs']):
        err['area'] = float(np.max(np.abs(A - ob['area']) / ob['area']))
        err['volume'] = float(np.max(np.abs(V - ob['volume']) / ob['volume']))
    return err


# Bounds: the temperature, momentum and species sums add binary32 values (or
# their exact squares) in float-float (about 2^-44 relative per addition) and
# combine once in binary64: 1e-11. Area and volume add binary32 triangle
# terms, each rounded at about 2^-24 of its size: 2e-7 of the total.
BOUND = {'kT': 1e-11, 'momentum': 1e-11, 'mass': 1e-11, 'area': 2e-7, 'volume': 2e-7}


@pytest.mark.parametrize('name,steps', [('single_rbc', 0), ('single_rbc', 10), ('channel', 10)])
def test_fp64_reductions_against_oracle(name, steps):
    desc = W.single_rbc() if name == 'single_rbc' else W.rbc_channel()
    err = _errors(desc, steps)
    print('\nFP64 reductions, %s after %d steps: %s' % (name, steps,
          ', '.join('%s %.2e' % kv for kv in err.items())))
    for k, e in err.items():
        assert e < BOUND[k], (k, e, err)
