"""FP64 CPU oracle for the tDPD + RBC step (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package. It shares no code with the CUDA library:
the arithmetic lives in ``tdpd_oracle.c`` (plain C, double precision), built
here with gcc on first use. Inputs come from the ``workloads`` module, rounded
to float32 exactly as the library stores them, so a comparison measures only
the arithmetic.
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

import workloads

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, 'tdpd_oracle.c')
_HDR = os.path.join(_HERE, 'tdpd_oracle.h')
_LIB = os.path.join(_HERE, 'liboracle.so')
_lock = threading.Lock()
_lib = None

# fixed, machine-independent floating point: no FMA contraction, no fast-math
CFLAGS = ['-O2', '-std=c11', '-fPIC', '-shared', '-fopenmp', '-ffp-contract=off',
          '-fno-fast-math', '-Wall']


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (gcc, OpenMP)."""
    with _lock:
        stale = (not os.path.exists(_LIB) or
                 os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
        if force or stale:
            tmp = _LIB + '.%d.tmp' % os.getpid()
            subprocess.run(['gcc', *CFLAGS, '-o', tmp, _SRC, '-lm'], check=True)
            os.replace(tmp, _LIB)
    return _LIB


class _Sys(C.Structure):
    _fields_ = [
        ('n', C.c_int), ('ns', C.c_int), ('ntypes', C.c_int),
        ('L', C.c_double * 3), ('periodic', C.c_int * 3),
        ('wall_lo', C.c_double), ('wall_hi', C.c_double),
        ('a', C.c_void_p), ('gamma', C.c_void_p), ('sigma', C.c_void_p),
        ('rc', C.c_double), ('s_f', C.c_double),
        ('kappa', C.c_void_p), ('rcc', C.c_double), ('s_c', C.c_double),
        ('seed', C.c_uint64), ('exclude_same_body', C.c_int),
        ('dt', C.c_double), ('lam', C.c_double), ('fbody', C.c_double * 3),
        ('frozen_types', C.c_uint32),
        ('k_react', C.c_double), ('r_src', C.c_int), ('r_dst', C.c_int),
        ('react_types', C.c_uint32),
        ('type', C.c_void_p), ('body', C.c_void_p), ('id', C.c_void_p),
        ('qr_ms', C.c_double), ('qr_rho', C.c_double), ('fbody_flip', C.c_int),
        ('cyl_R', C.c_double),
    ]


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        P = C.c_void_p
        L.orc_tea.argtypes = [P, P, C.c_int]
        L.orc_normal_pair.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32, P]
        L.orc_uniform_pair.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32, P, P]
        L.orc_pair_forces.argtypes = [P, P, P, P, C.c_uint32, C.c_int, P, P]
        L.orc_pair_forces.restype = C.c_int
        L.orc_mem_create.argtypes = [C.c_int, C.c_int, C.c_int, P, P, P, P, P, P]
        L.orc_mem_create.restype = P
        L.orc_mem_destroy.argtypes = [P]
        L.orc_mem_nedges.argtypes = [P]
        L.orc_mem_reset_lag.argtypes = [P]
        L.orc_mem_reset_lag.restype = None
        L.orc_mem_nedges.restype = C.c_int
        L.orc_mem_rest.argtypes = [P, P, P, P, P]
        L.orc_mem_forces.argtypes = [P, P, P, P, C.c_uint64, C.c_uint32, C.c_double, C.c_int, P, P]
        L.orc_mem_energy.argtypes = [P, P, C.c_int]
        L.orc_mem_energy.restype = C.c_double
        L.orc_mem_angles.argtypes = [P, P, C.c_int, P]
        L.orc_forces.argtypes = [P, P, P, P, P, C.c_uint32, C.c_int, P, P]
        L.orc_forces.restype = C.c_int
        L.orc_run.argtypes = [P, P, P, P, P, P, P, C.c_uint32, C.c_int, C.c_int]
        L.orc_run.restype = C.c_int
        L.orc_observables.argtypes = [P, P, P, P]
        L.orc_num_threads.restype = C.c_int
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def tea(v0, v1, key, rounds):
    v = np.array([v0, v1], np.uint32)
    k = np.asarray(key, np.uint32)
    lib().orc_tea(_p(v), _p(k), int(rounds))
    return int(v[0]), int(v[1])


def normal_pair(seed, i, j, step, stream):
    g = np.zeros(2)
    lib().orc_normal_pair(seed, i, j, step, stream, _p(g))
    return g


def uniform_pair(seed, i, j, step, stream):
    b = np.zeros(2, np.uint32)
    u = np.zeros(2)
    lib().orc_uniform_pair(seed, i, j, step, stream, _p(b), _p(u))
    return b, u


def _f64(x):
    """Value as the library stores it (binary32), widened to double."""
    return np.asarray(x, np.float32).astype(np.float64)


MEM_KEYS = ('kT', 'p', 'x0', 'm', 'kg', 'kl', 'kv', 'kb', 'theta0', 'gammaT', 'gammaC', 'v_ratio', 'lagged_av')


class Oracle:
    """One workload held in FP64: state, forces at the current step, step count."""

    def __init__(self, desc, mode: int = 1):
        self.desc = desc
        self.mode = mode
        pos, vel, conc, typ, body = workloads.flat_state(desc)
        self.n = pos.shape[0]
        self.ns = int(desc['n_species'])
        self.T = int(desc['n_types'])
        self.pos = pos.astype(np.float64)
        self.vel = vel.astype(np.float64)
        self.conc = conc.astype(np.float64).reshape(self.n, self.ns)
        self.type = typ.astype(np.int32)
        self.body = body.astype(np.int32)
        self.id = np.arange(self.n, dtype=np.uint32)
        self.a = _f64(desc['a']).ravel().copy()
        self.gamma = _f64(desc['gamma']).ravel().copy()
        self.sigma = _f64(desc['sigma']).ravel().copy()
        self.kappa = _f64(desc['kappa']).ravel().copy()
        s = _Sys()
        s.n, s.ns, s.ntypes = self.n, self.ns, self.T
        s.L[:] = _f64(desc['L']).tolist()
        s.periodic[:] = [int(x) for x in desc['periodic']]
        s.wall_lo, s.wall_hi = float(_f64(desc['wall_lo'])), float(_f64(desc['wall_hi']))
        s.a, s.gamma, s.sigma = _p(self.a), _p(self.gamma), _p(self.sigma)
        s.rc, s.s_f = float(_f64(desc['rc'])), float(_f64(desc['s_f']))
        s.kappa = _p(self.kappa)
        s.rcc, s.s_c = float(_f64(desc['rcc'])), float(_f64(desc['s_c']))
        s.seed = int(desc['seed']) & (2**64 - 1)
        s.exclude_same_body = int(desc['exclude_same_body'])
        s.dt, s.lam = float(_f64(desc['dt'])), float(_f64(desc['lam']))
        s.fbody[:] = _f64(desc['body_force']).tolist()
        s.frozen_types = int(desc['frozen_types'])
        s.fbody_flip = int(desc.get('body_force_flip', 0))
        s.cyl_R = float(_f64(desc.get('cylinder_radius', 0.0)))
        r = desc.get('reaction')
        if r:
            s.k_react, s.r_src, s.r_dst, s.react_types = float(_f64(r['k'])), r['src'], r['dst'], r['types']
        s.type, s.body, s.id = _p(self.type), _p(self.body), _p(self.id)
        q = desc.get('random_flux')
        if q:
            s.qr_ms, s.qr_rho = float(_f64(q['m_s'])), float(_f64(q['rho']))
        self.sys = s
        self.mem = None
        self.nrbc = len(desc['rbcs'])
        if self.nrbc:
            tri = desc['rbcs'][0]['tri']
            for rb in desc['rbcs']:
                assert np.array_equal(rb['tri'], tri), 'oracle: one membrane topology per workload'
            self.nv = desc['rbcs'][0]['pos'].shape[0]
            self.tri = np.ascontiguousarray(tri, np.int32)
            self.ntri = self.tri.shape[0]
            first = []
            off = desc['particles']['pos'].shape[0]
            for rb in desc['rbcs']:
                first.append(off)
                off += rb['pos'].shape[0]
            self.first = np.asarray(first, np.int32)
            rest = np.concatenate([(rb['rest'] if rb['rest'] is not None else rb['pos'])
                                   for rb in desc['rbcs']]).astype(np.float32).astype(np.float64)
            mp = desc['membrane']
            self.mparams = np.array([float(_f64(mp.get(k, 0))) for k in MEM_KEYS])
            Lp = np.array(s.L[:], np.float64)
            per = np.array(s.periodic[:], np.int32)
            self.mem = lib().orc_mem_create(self.nrbc, self.nv, self.ntri, _p(self.tri), _p(self.first),
                                            _p(rest), _p(Lp), _p(per), _p(self.mparams))
            if not self.mem:
                raise ValueError('oracle: membrane mesh is not a closed oriented surface')
            self.ne = lib().orc_mem_nedges(self.mem)
        self.step = 0
        self.F = np.zeros((self.n, 3))
        self.Q = np.zeros((self.n, self.ns))
        self.init_forces()

    def __del__(self):
        if getattr(self, 'mem', None):
            lib().orc_mem_destroy(self.mem)
            self.mem = None

    # ---------------------------------------------------------------- forces
    def pair_forces(self, pos=None, vel=None, conc=None, step=None, mode=None):
        pos = self.pos if pos is None else np.ascontiguousarray(pos, np.float64)
        vel = self.vel if vel is None else np.ascontiguousarray(vel, np.float64)
        conc = self.conc if conc is None else np.ascontiguousarray(conc, np.float64)
        F = np.zeros((self.n, 3))
        Q = np.zeros((self.n, self.ns))
        rc = lib().orc_pair_forces(C.byref(self.sys), _p(pos), _p(vel), _p(conc),
                                   self.step if step is None else step,
                                   self.mode if mode is None else mode, _p(F), _p(Q))
        if rc:
            raise ValueError('oracle: box smaller than three cells')
        return F, Q

    def membrane_forces(self, pos=None, vel=None, step=None, parts=15):
        pos = self.pos if pos is None else np.ascontiguousarray(pos, np.float64)
        vel = self.vel if vel is None else np.ascontiguousarray(vel, np.float64)
        F = np.zeros((self.n, 3))
        AV = np.zeros((max(self.nrbc, 1), 2))
        if self.mem:
            lib().orc_mem_forces(self.mem, _p(pos), _p(vel), _p(self.id), self.sys.seed,
                                 self.step if step is None else step, self.sys.dt, parts, _p(F), _p(AV))
        return F, AV[:self.nrbc]

    def membrane_energy(self, pos=None, parts=13):
        pos = self.pos if pos is None else np.ascontiguousarray(pos, np.float64)
        return lib().orc_mem_energy(self.mem, _p(pos), parts)

    def membrane_angles(self, b=0, pos=None):
        pos = self.pos if pos is None else np.ascontiguousarray(pos, np.float64)
        th = np.zeros(self.ne)
        lib().orc_mem_angles(self.mem, _p(pos), b, _p(th))
        return th

    def membrane_rest(self):
        A0j = np.zeros((self.nrbc, self.ntri))
        l0 = np.zeros((self.nrbc, self.ne))
        A0 = np.zeros(self.nrbc)
        V0 = np.zeros(self.nrbc)
        lib().orc_mem_rest(self.mem, _p(A0j), _p(l0), _p(A0), _p(V0))
        return A0j, l0, A0, V0

    def forces(self, pos=None, vel=None, conc=None, step=None, mode=None):
        pos = self.pos if pos is None else np.ascontiguousarray(pos, np.float64)
        vel = self.vel if vel is None else np.ascontiguousarray(vel, np.float64)
        conc = self.conc if conc is None else np.ascontiguousarray(conc, np.float64)
        F = np.zeros((self.n, 3))
        Q = np.zeros((self.n, self.ns))
        rc = lib().orc_forces(C.byref(self.sys), self.mem, _p(pos), _p(vel), _p(conc),
                              self.step if step is None else step,
                              self.mode if mode is None else mode, _p(F), _p(Q))
        if rc:
            raise ValueError('oracle: box smaller than three cells')
        return F, Q

    def init_forces(self):
        if getattr(self, 'mem', None):
            lib().orc_mem_reset_lag(self.mem)
        self.F, self.Q = self.forces()

    def set_state(self, pos, vel, conc, step=0):
        self.pos = np.ascontiguousarray(pos, np.float32).astype(np.float64)
        self.vel = np.ascontiguousarray(vel, np.float32).astype(np.float64)
        self.conc = np.ascontiguousarray(conc, np.float32).astype(np.float64).reshape(self.n, self.ns)
        self.step = step
        self.init_forces()

    def run(self, nsteps: int, mode=None):
        rc = lib().orc_run(C.byref(self.sys), self.mem, _p(self.pos), _p(self.vel), _p(self.conc),
                           _p(self.F), _p(self.Q), self.step, int(nsteps),
                           self.mode if mode is None else mode)
        if rc:
            raise ValueError('oracle: box smaller than three cells')
        self.step += int(nsteps)

    def observables(self):
        out = np.zeros(5 + self.ns)
        lib().orc_observables(C.byref(self.sys), _p(self.vel), _p(self.conc), _p(out))
        _, AV = self.membrane_forces(parts=0) if self.nrbc else (None, np.zeros((0, 2)))
        return dict(kT=out[0], momentum=out[1:4].copy(), mass=out[4:4 + self.ns].copy(),
                    n_mobile=int(out[4 + self.ns]), area=AV[:, 0].copy(), volume=AV[:, 1].copy())


def num_threads() -> int:
    return lib().orc_num_threads()
