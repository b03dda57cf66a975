"""Thin ctypes binding of libtdpd.so (tdpd.h). Argument marshalling only:
every step of the simulation runs in the library's CUDA kernels.

Functions carry the C names. Arrays are numpy (host) and are converted to
contiguous float32/int32 before the call. A non-zero status raises TdpdError
with the library's message. If libtdpd.so is missing this module raises at
import: there is no fallback path.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, 'libtdpd.so')

MAX_TYPES = 4
MAX_SPECIES = 16
STATUS = {0: 'OK', 1: 'EINVAL', 2: 'ENOMEM', 3: 'ECUDA', 4: 'EOVERFLOW', 5: 'ENONFINITE',
          6: 'ETIMEOUT', 7: 'ESTATE'}


class TdpdError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__('%s: %s' % (STATUS.get(status, status), msg))
        self.status = status


class tdpd_config(C.Structure):
    _fields_ = [('L', C.c_float * 3), ('periodic', C.c_int32 * 3),
                ('wall_lo', C.c_float), ('wall_hi', C.c_float),
                ('n_types', C.c_int32), ('n_species', C.c_int32), ('seed', C.c_uint64),
                ('dt', C.c_float), ('lam', C.c_float), ('rc', C.c_float), ('s_f', C.c_float),
                ('rcc', C.c_float), ('s_c', C.c_float), ('body_force', C.c_float * 3),
                ('frozen_types', C.c_uint32), ('exclude_same_body', C.c_int32),
                ('cells_per_cutoff', C.c_int32)]


class tdpd_membrane(C.Structure):
    _fields_ = [(k, C.c_float) for k in ('kT', 'p', 'x0', 'm', 'kg', 'kl', 'kv', 'kb', 'theta0',
                                          'gammaT', 'gammaC', 'v_ratio')] + [('lagged_av', C.c_int32)]


class tdpd_obs(C.Structure):
    _fields_ = [('step', C.c_int64), ('n_particles', C.c_int32), ('n_mobile', C.c_int32),
                ('n_species', C.c_int32), ('n_rbc', C.c_int32), ('kT', C.c_double),
                ('momentum', C.c_double * 3), ('mass', C.c_double * MAX_SPECIES),
                ('n_membrane', C.c_int32), ('pad_', C.c_int32),
                ('mass_membrane', C.c_double * MAX_SPECIES)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError('libtdpd.so not built (run python paper_1611_06163_gb300/buildlib.py or '
                          '__graft_entry__.build()); there is no fallback implementation')
    L = C.CDLL(LIB_PATH)
    P, I, F = C.c_void_p, C.c_int, C.c_float
    sig = {
        'tdpd_create': ([C.POINTER(P), C.POINTER(tdpd_config)], I),
        'tdpd_set_pair': ([P, I, I, F, F, F], I),
        'tdpd_set_kappa': ([P, I, I, I, F], I),
        'tdpd_set_reaction': ([P, F, I, I, C.c_uint32], I),
        'tdpd_set_membrane': ([P, C.POINTER(tdpd_membrane)], I),
        'tdpd_add_particles': ([P, I, P, P, P, P], I),
        'tdpd_add_rbc': ([P, I, P, P, P, I, I, P, P, C.POINTER(I)], I),
        'tdpd_batch_create': ([C.POINTER(P), P, I], I),
        'tdpd_set_stream': ([P, P], I),
        'tdpd_set_lanes': ([P, I], I),
        'tdpd_set_skin': ([P, C.c_float], I),
        'tdpd_lanes': ([P], I),
        'tdpd_set_pair_mode': ([P, I], I),
        'tdpd_list_shape': ([P, C.POINTER(C.c_float), C.POINTER(I), P, I, C.POINTER(I)], I),
        'tdpd_pair_mode': ([P], I),
        'tdpd_set_sort_mode': ([P, I], I),
        'tdpd_sort_mode': ([P, P], I),
        'tdpd_set_random_flux': ([P, C.c_float, C.c_float], I),
        'tdpd_set_body_force_profile': ([P, I], I),
        'tdpd_set_cylinder_wall': ([P, F], I),
        'tdpd_list_rebuilds': ([P, I, C.POINTER(C.c_int64)], I),
        'tdpd_commit': ([P], I),
        'tdpd_step': ([P, I], I),
        'tdpd_sync': ([P], I),
        'tdpd_set_state': ([P, I, P, P, P], I),
        'tdpd_set_states': ([P, P, P, P], I),
        'tdpd_set_states_device': ([P, P, P, P], I),
        'tdpd_read_state_device': ([P, I, P, P, P], I),
        'tdpd_save': ([P, C.c_char_p], I),
        'tdpd_load': ([P, C.c_char_p], I),
        'tdpd_read_state': ([P, I, P, P, P], I),
        'tdpd_read_forces': ([P, I, P, P], I),
        'tdpd_read_observables': ([P, I, C.POINTER(tdpd_obs)], I),
        'tdpd_read_rbc': ([P, I, P, P], I),
        'tdpd_replica_status': ([P, P], I),
        'tdpd_num_replicas': ([P], I),
        'tdpd_num_particles': ([P, I], I),
        'tdpd_current_step': ([P], C.c_int64),
        'tdpd_launches_per_step': ([P], I),
        'tdpd_last_error': ([P], C.c_char_p),
        'tdpd_destroy': ([P], None),
        'tdpd_debug_rng': ([C.c_uint64, I, P, P, P, P, P, P], I),
        'tdpd_step_timed': ([P, P, I, C.POINTER(I)], I),
        'tdpd_kernel_name': ([P, I], C.c_char_p),
        'tdpd_mlp_create': ([C.POINTER(P), I], I),
        'tdpd_mlp_set_params': ([P, P], I),
        'tdpd_mlp_get_params': ([P, P], I),
        'tdpd_mlp_set_data': ([P, I, P, P], I),
        'tdpd_mlp_loss_grad': ([P, P, P], I),
        'tdpd_mlp_train': ([P, I, F, P], I),
        'tdpd_mlp_predict': ([P, I, P, P, P, P], I),
        'tdpd_mlp_destroy': ([P], None),
        'tdpd_pair_forces_noalloc': ([C.POINTER(tdpd_config), P, P, I, P, P, P, P, C.c_uint32, P, P, P], I),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    return L


lib = _load()


def _chk(handle, status):
    if status != 0:
        msg = lib.tdpd_last_error(handle)
        raise TdpdError(status, msg.decode() if msg else '')


def _f32(a, shape=None):
    a = np.ascontiguousarray(a, np.float32)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


# ------------------------------------------------------------------ C names

def tdpd_create(cfg: tdpd_config):
    h = C.c_void_p()
    _chk(None, lib.tdpd_create(C.byref(h), C.byref(cfg)))
    return h


def tdpd_set_pair(h, ti, tj, a, gamma, sigma):
    _chk(h, lib.tdpd_set_pair(h, ti, tj, float(a), float(gamma), float(sigma)))


def tdpd_set_kappa(h, ti, tj, species, kappa):
    _chk(h, lib.tdpd_set_kappa(h, ti, tj, species, float(kappa)))


def tdpd_set_reaction(h, k, src, dst, types):
    _chk(h, lib.tdpd_set_reaction(h, float(k), src, dst, types))


def tdpd_set_membrane(h, m: tdpd_membrane):
    _chk(h, lib.tdpd_set_membrane(h, C.byref(m)))


def tdpd_add_particles(h, pos, vel, conc, typ):
    pos = _f32(pos)
    n = pos.size // 3
    vel = _f32(vel)
    conc = None if conc is None else _f32(conc)
    typ = np.ascontiguousarray(typ, np.int32)
    _chk(h, lib.tdpd_add_particles(h, n, _ptr(pos), _ptr(vel), _ptr(conc), _ptr(typ)))


def tdpd_add_rbc(h, pos, vel, conc, typ, tri, rest=None):
    pos = _f32(pos)
    vel = _f32(vel)
    conc = None if conc is None else _f32(conc)
    tri = np.ascontiguousarray(tri, np.int32)
    rest = None if rest is None else _f32(rest)
    idx = C.c_int(-1)
    _chk(h, lib.tdpd_add_rbc(h, pos.size // 3, _ptr(pos), _ptr(vel), _ptr(conc), int(typ),
                             tri.size // 3, _ptr(tri), _ptr(rest), C.byref(idx)))
    return idx.value


def tdpd_batch_create(handles):
    arr = (C.c_void_p * len(handles))(*[h.value for h in handles])
    out = C.c_void_p()
    _chk(None, lib.tdpd_batch_create(C.byref(out), arr, len(handles)))
    return out


def tdpd_set_stream(h, stream_ptr):
    _chk(h, lib.tdpd_set_stream(h, C.c_void_p(stream_ptr) if stream_ptr else None))


def tdpd_set_lanes(h, lanes):
    _chk(h, lib.tdpd_set_lanes(h, int(lanes)))


def tdpd_set_pair_mode(h, mode):
    _chk(h, lib.tdpd_set_pair_mode(h, int(mode)))


def tdpd_pair_mode(h):
    return int(lib.tdpd_pair_mode(h))


def tdpd_set_sort_mode(h, mode):
    _chk(h, lib.tdpd_set_sort_mode(h, int(mode)))


def tdpd_sort_mode(h):
    """(sort in use: 1 kernel chain, 2 one cluster; commit's times of 16 steps
    with the cluster and with the chain in ms, -1 when not timed)."""
    t = np.full(2, -1.0, np.float32)
    m = int(lib.tdpd_sort_mode(h, _ptr(t)))
    return m, t.copy()


def tdpd_list_shape(h):
    """(skin, cells_per_cutoff, commit's step times of the candidate shapes in ms)."""
    sk, m, n = C.c_float(0), C.c_int(0), C.c_int(0)
    t = np.zeros(16, np.float32)
    _chk(h, lib.tdpd_list_shape(h, C.byref(sk), C.byref(m), _ptr(t), 16, C.byref(n)))
    return float(sk.value), int(m.value), t[:min(n.value, 16)].copy()


def tdpd_set_skin(h, skin):
    _chk(h, lib.tdpd_set_skin(h, float(skin)))


def tdpd_list_rebuilds(h, replica=0):
    v = C.c_int64(0)
    _chk(h, lib.tdpd_list_rebuilds(h, int(replica), C.byref(v)))
    return v.value


def tdpd_set_random_flux(h, m_s, rho):
    _chk(h, lib.tdpd_set_random_flux(h, float(m_s), float(rho)))


def tdpd_set_body_force_profile(h, mode):
    _chk(h, lib.tdpd_set_body_force_profile(h, int(mode)))


def tdpd_set_cylinder_wall(h, radius):
    _chk(h, lib.tdpd_set_cylinder_wall(h, float(radius)))


def tdpd_lanes(h):
    return lib.tdpd_lanes(h)


def tdpd_commit(h):
    _chk(h, lib.tdpd_commit(h))


def tdpd_step(h, n):
    _chk(h, lib.tdpd_step(h, int(n)))


def tdpd_step_timed(h, max_kernels=16):
    ms = np.zeros(max_kernels, np.float32)
    nk = C.c_int(0)
    _chk(h, lib.tdpd_step_timed(h, _ptr(ms), max_kernels, C.byref(nk)))
    return ms[:nk.value].astype(np.float64)


def tdpd_kernel_name(h, k):
    r = lib.tdpd_kernel_name(h, k)
    return r.decode() if r else None


def tdpd_sync(h):
    _chk(h, lib.tdpd_sync(h))


def tdpd_set_state(h, replica, pos, vel, conc=None):
    pos, vel = _f32(pos), _f32(vel)
    conc = None if conc is None else _f32(conc)
    _chk(h, lib.tdpd_set_state(h, replica, _ptr(pos), _ptr(vel), _ptr(conc)))


def tdpd_set_states(h, pos, vel, conc):
    """Every replica's state at once: arrays of all replicas one after
    another in replica order, each in its load order."""
    pos, vel, conc = _f32(pos), _f32(vel), _f32(conc)
    _chk(h, lib.tdpd_set_states(h, _ptr(pos), _ptr(vel), _ptr(conc)))


def tdpd_set_states_device(h, pos_ptr, vel_ptr, conc_ptr):
    """tdpd_set_states with device pointers (integers, e.g. a CUDA
    tensor's data_ptr())."""
    _chk(h, lib.tdpd_set_states_device(h, C.c_void_p(pos_ptr), C.c_void_p(vel_ptr), C.c_void_p(conc_ptr)))


def tdpd_read_state_device(h, replica, pos_ptr, vel_ptr, conc_ptr):
    """Enqueue a load-order copy of the replica's state into device arrays
    (integer pointers; 0 skips one) on the library's stream."""
    _chk(h, lib.tdpd_read_state_device(h, int(replica), C.c_void_p(pos_ptr or None), C.c_void_p(vel_ptr or None),
                                       C.c_void_p(conc_ptr or None)))


def tdpd_save(h, path):
    _chk(h, lib.tdpd_save(h, os.fsencode(path)))


def tdpd_load(h, path):
    _chk(h, lib.tdpd_load(h, os.fsencode(path)))


def tdpd_num_particles(h, replica=0):
    return lib.tdpd_num_particles(h, replica)


def tdpd_num_replicas(h):
    return lib.tdpd_num_replicas(h)


def tdpd_current_step(h):
    return lib.tdpd_current_step(h)


def tdpd_launches_per_step(h):
    return lib.tdpd_launches_per_step(h)


def tdpd_read_state(h, replica=0, ns=1, out=None):
    n = tdpd_num_particles(h, replica)
    if out is None:
        out = (np.empty((n, 3), np.float32), np.empty((n, 3), np.float32), np.empty((n, ns), np.float32))
    pos, vel, conc = out
    _chk(h, lib.tdpd_read_state(h, replica, _ptr(pos), _ptr(vel), _ptr(conc)))
    return pos, vel, conc


def tdpd_read_forces(h, replica=0, ns=1):
    n = tdpd_num_particles(h, replica)
    F = np.empty((n, 3), np.float32)
    Q = np.empty((n, ns), np.float32)
    _chk(h, lib.tdpd_read_forces(h, replica, _ptr(F), _ptr(Q)))
    return F, Q


def tdpd_read_observables(h, replica=0):
    o = tdpd_obs()
    _chk(h, lib.tdpd_read_observables(h, replica, C.byref(o)))
    return dict(step=o.step, n_particles=o.n_particles, n_mobile=o.n_mobile, n_species=o.n_species,
                n_rbc=o.n_rbc, kT=o.kT, momentum=np.array(o.momentum[:]),
                mass=np.array(o.mass[:o.n_species]), n_membrane=o.n_membrane,
                mass_membrane=np.array(o.mass_membrane[:o.n_species]))


def tdpd_read_rbc(h, replica, n_rbc):
    A = np.zeros(n_rbc)
    V = np.zeros(n_rbc)
    if n_rbc:
        _chk(h, lib.tdpd_read_rbc(h, replica, _ptr(A), _ptr(V)))
    return A, V


def tdpd_replica_status(h):
    st = np.zeros(tdpd_num_replicas(h), np.int32)
    _chk(h, lib.tdpd_replica_status(h, _ptr(st)))
    return st


def tdpd_destroy(h):
    if h:
        lib.tdpd_destroy(h)


def tdpd_debug_rng(seed, i, j, step, stream):
    i, j, step, stream = (np.ascontiguousarray(x, np.uint32) for x in (i, j, step, stream))
    n = i.size
    bits = np.zeros(2 * n, np.uint32)
    normal = np.zeros(2 * n, np.float32)
    _chk(None, lib.tdpd_debug_rng(seed, n, _ptr(i), _ptr(j), _ptr(step), _ptr(stream),
                                  _ptr(bits), _ptr(normal)))
    return bits.reshape(n, 2), normal.reshape(n, 2)


def tdpd_pair_forces_noalloc(cfg, pair_coef, kappa, n, pos_ptr, vel_ptr, conc_ptr, type_ptr, step,
                             force_ptr, flux_ptr, stream_ptr=None):
    """Allocation-free pair force + flux; the array arguments are device
    pointers (integers), pair_coef/kappa host arrays (see tdpd.h)."""
    pc = np.ascontiguousarray(pair_coef, np.float32)
    kp = np.ascontiguousarray(kappa, np.float32)
    _chk(None, lib.tdpd_pair_forces_noalloc(C.byref(cfg), _ptr(pc), _ptr(kp), int(n),
                                            C.c_void_p(pos_ptr), C.c_void_p(vel_ptr),
                                            C.c_void_p(conc_ptr), C.c_void_p(type_ptr), int(step),
                                            C.c_void_p(force_ptr), C.c_void_p(flux_ptr),
                                            C.c_void_p(stream_ptr) if stream_ptr else None))


MLP_NPARAM = 4610


def tdpd_mlp_create(members):
    h = C.c_void_p()
    _chk(None, lib.tdpd_mlp_create(C.byref(h), int(members)))
    return h


def tdpd_mlp_set_params(h, params):
    p = _f32(params)
    _chk(None, lib.tdpd_mlp_set_params(h, _ptr(p)))


def tdpd_mlp_get_params(h, members):
    p = np.zeros((members, MLP_NPARAM), np.float32)
    _chk(None, lib.tdpd_mlp_get_params(h, _ptr(p)))
    return p


def tdpd_mlp_set_data(h, X, Y):
    X = _f32(X)
    Y = _f32(Y)
    _chk(None, lib.tdpd_mlp_set_data(h, X.shape[0], _ptr(X), _ptr(Y)))


def tdpd_mlp_loss_grad(h, members):
    loss = np.zeros(members)
    grad = np.zeros((members, MLP_NPARAM), np.float32)
    _chk(None, lib.tdpd_mlp_loss_grad(h, _ptr(loss), _ptr(grad)))
    return loss, grad


def tdpd_mlp_train(h, steps, lr, members):
    loss = np.zeros(members)
    _chk(None, lib.tdpd_mlp_train(h, int(steps), float(lr), _ptr(loss)))
    return loss


def tdpd_mlp_predict(h, X, members):
    X = _f32(X)
    n = X.shape[0]
    mean = np.zeros((n, 2), np.float32)
    spread = np.zeros((n, 2), np.float32)
    each = np.zeros((members, n, 2), np.float32)
    _chk(None, lib.tdpd_mlp_predict(h, n, _ptr(X), _ptr(mean), _ptr(spread), _ptr(each)))
    return mean, spread, each


def tdpd_mlp_destroy(h):
    if h:
        lib.tdpd_mlp_destroy(h)


# ------------------------------------------------------ workload marshalling

def config_from(desc) -> tdpd_config:
    c = tdpd_config()
    c.L[:] = [float(x) for x in desc['L']]
    c.periodic[:] = [int(x) for x in desc['periodic']]
    c.wall_lo, c.wall_hi = float(desc['wall_lo']), float(desc['wall_hi'])
    c.n_types, c.n_species = int(desc['n_types']), int(desc['n_species'])
    c.seed = int(desc['seed']) & (2**64 - 1)
    c.dt, c.lam = float(desc['dt']), float(desc['lam'])
    c.rc, c.s_f, c.rcc, c.s_c = float(desc['rc']), float(desc['s_f']), float(desc['rcc']), float(desc['s_c'])
    c.body_force[:] = [float(x) for x in desc['body_force']]
    c.frozen_types = int(desc['frozen_types'])
    c.exclude_same_body = int(desc['exclude_same_body'])
    c.cells_per_cutoff = int(desc.get('cells_per_cutoff', 0))
    return c


def create_from(desc, stream_ptr=None):
    """A handle loaded with a workload description (see the workloads module)."""
    h = tdpd_create(config_from(desc))
    try:
        T, S = int(desc['n_types']), int(desc['n_species'])
        for i in range(T):
            for j in range(i, T):
                tdpd_set_pair(h, i, j, desc['a'][i, j], desc['gamma'][i, j], desc['sigma'][i, j])
                for s in range(S):
                    tdpd_set_kappa(h, i, j, s, desc['kappa'][i, j, s])
        r = desc.get('reaction')
        if r:
            tdpd_set_reaction(h, r['k'], r['src'], r['dst'], r['types'])
        if desc.get('membrane'):
            m = tdpd_membrane(**{k: (int(v) if k == 'lagged_av' else float(v)) for k, v in desc['membrane'].items()})
            tdpd_set_membrane(h, m)
        p = desc['particles']
        if p['pos'].shape[0]:
            tdpd_add_particles(h, p['pos'], p['vel'], p['conc'], p['type'])
        for rb in desc['rbcs']:
            tdpd_add_rbc(h, rb['pos'], rb['vel'], rb['conc'], rb['type'], rb['tri'], rb['rest'])
        if desc.get('body_force_flip'):
            tdpd_set_body_force_profile(h, 1)
        if desc.get('cylinder_radius'):
            tdpd_set_cylinder_wall(h, desc['cylinder_radius'])
        q = desc.get('random_flux')
        if q:
            tdpd_set_random_flux(h, q['m_s'], q['rho'])
        if desc.get('skin') is not None:
            tdpd_set_skin(h, desc['skin'])
        if desc.get('lanes') is not None:
            tdpd_set_lanes(h, desc['lanes'])
        if desc.get('pair_mode') is not None:
            tdpd_set_pair_mode(h, desc['pair_mode'])
        if desc.get('sort_mode') is not None:
            tdpd_set_sort_mode(h, desc['sort_mode'])
        if stream_ptr:
            tdpd_set_stream(h, stream_ptr)
    except Exception:
        tdpd_destroy(h)
        raise
    return h
