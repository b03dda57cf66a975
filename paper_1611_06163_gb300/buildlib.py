"""Build libtdpd.so in-tree with nvcc for sm_103a (GB300).

Each .cu translation unit is compiled in parallel to an object under
``_build/``, then linked into ``libtdpd.so`` next to this file.
"""

from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, 'csrc')
INC = os.path.join(ROOT, 'include')
OUT = os.path.join(HERE, '_build')
LIB = os.path.join(HERE, 'libtdpd.so')
SOURCES = ['engine.cu', 'k_sort.cu', 'k_pair.cu', 'k_pair_std.cu', 'k_list.cu', 'k_membrane.cu', 'k_misc.cu', 'noalloc.cu', 'mlp.cu']

NVCC_FLAGS = ['-gencode', 'arch=compute_103a,code=sm_103a', '-lineinfo', '-O3', '-std=c++17',
              '-Xcompiler', '-fPIC', '-Xcompiler', '-O2', '-I' + INC, '-I' + CSRC]


def _nvcc():
    for c in (os.environ.get('NVCC'), '/usr/local/cuda/bin/nvcc', 'nvcc'):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return 'nvcc'


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INC, 'tdpd.h')]
    return max(os.path.getmtime(f) for f in files)


def _compile(src, extra):
    obj = os.path.join(OUT, os.path.splitext(src)[0] + '.o')
    cmd = [_nvcc(), *NVCC_FLAGS, *extra, '-c', os.path.join(CSRC, src), '-o', obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError('nvcc failed for %s:\n%s\n%s' % (src, ' '.join(cmd), r.stderr))
    return obj, r.stderr


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        res = list(ex.map(lambda s: _compile(s, list(extra)), SOURCES))
    if verbose:
        for _, err in res:
            if err:
                sys.stderr.write(err)
    tmp = LIB + '.%d.tmp' % os.getpid()
    cmd = [_nvcc(), '-gencode', 'arch=compute_103a,code=sm_103a', '-shared', '-o', tmp] + [o for o, _ in res]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError('link failed:\n%s\n%s' % (' '.join(cmd), r.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == '__main__':
    v = '-v' in sys.argv
    extra = ['-Xptxas', '-v'] if v else []
    print(build(force=True, verbose=v, extra=extra))
