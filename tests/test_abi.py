"""The C ABI: libtdpd.so builds, loads without a GPU, and exports every
function include/tdpd.h declares; struct layouts agree between C and the
binding; host-side argument checks reject bad input before any device work."""

import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, 'include', 'tdpd.h')


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r'/\*.*?\*/', '', text, flags=re.S)
    return sorted(set(re.findall(r'\b(tdpd_[a-z0-9_]+)\s*\(', text)))


def test_library_exports_every_declared_function():
    import paper_1611_06163_gb300 as pkg
    path = pkg.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 25
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_struct_layouts_match_c():
    from paper_1611_06163_gb300 import binding as bd
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "tdpd.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(tdpd_config), sizeof(tdpd_obs), sizeof(tdpd_membrane),
         offsetof(tdpd_config, seed), offsetof(tdpd_config, cells_per_cutoff), offsetof(tdpd_obs, mass));
  return 0;
}
'''
    tmp = os.path.join(ROOT, 'paper_1611_06163_gb300', '_build')
    os.makedirs(tmp, exist_ok=True)
    c = os.path.join(tmp, 'abi_sizes.c')
    exe = os.path.join(tmp, 'abi_sizes')
    open(c, 'w').write(src)
    subprocess.run(['gcc', '-I', os.path.join(ROOT, 'include'), c, '-o', exe], check=True)
    out = [int(x) for x in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()]
    assert out == [ctypes.sizeof(bd.tdpd_config), ctypes.sizeof(bd.tdpd_obs), ctypes.sizeof(bd.tdpd_membrane),
                   bd.tdpd_config.seed.offset, bd.tdpd_config.cells_per_cutoff.offset, bd.tdpd_obs.mass.offset]


def test_host_validation_without_gpu():
    """Configuration errors are reported by the host before any CUDA call."""
    from paper_1611_06163_gb300 import binding as bd
    import workloads as W
    d = W.fluid_box(L=10.0)
    cfg = bd.config_from(d)
    cfg.n_species = 0
    with pytest.raises(bd.TdpdError) as e:
        bd.tdpd_create(cfg)
    assert e.value.status == 1 and 'n_species' in str(e.value)
    cfg = bd.config_from(d)
    cfg.periodic[0] = 0
    with pytest.raises(bd.TdpdError):
        bd.tdpd_create(cfg)
    cfg = bd.config_from(d)
    cfg.dt = -1.0
    with pytest.raises(bd.TdpdError):
        bd.tdpd_create(cfg)

