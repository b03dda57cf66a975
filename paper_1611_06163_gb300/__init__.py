"""GB300-native tDPD + RBC step (arXiv:1611.06163): CUDA kernels behind the C
ABI of include/tdpd.h, with a thin ctypes binding in the ``binding`` module
(importing it loads libtdpd.so and fails if the library is not built)."""

import os as _os

LIB_PATH = _os.path.join(_os.path.dirname(_os.path.abspath(__file__)), 'libtdpd.so')


def build(force: bool = False) -> str:
    """Compile libtdpd.so in-tree for sm_103a (no-op when up to date)."""
    from . import buildlib as _b
    return _b.build(force=force)
