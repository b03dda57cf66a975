"""Pins of the FP64 oracle to facts fixed outside itself: published test
vectors, closed forms, potentials whose gradient is the force, conservation
laws, fluctuation-dissipation statistics and exact solutions."""

import math

import numpy as np
import pytest
from scipy import integrate

import oracle
import workloads as W
from helpers import custom, membrane_only, small_sphere, icosahedron, relerr, read_golden


# ------------------------------------------------------------------ RNG

def test_tea_published_vector():
    for row in read_golden('tea_vectors.txt'):
        rounds = int(row[0])
        k = [int(x, 16) for x in row[1:5]]
        v = [int(x, 16) for x in row[5:7]]
        c = [int(x, 16) for x in row[7:9]]
        assert oracle.tea(v[0], v[1], k, rounds) == (c[0], c[1])


def test_uniforms_exact_in_binary32_and_open_interval():
    for i in range(2000):
        bits, u = oracle.uniform_pair(12345, i, 3 * i + 1, i % 7, i % 3)
        for b, x in zip(bits, u):
            assert 0.0 < x < 1.0
            assert float(np.float32(x)) == x
            assert x == ((int(b) >> 9) + 0.5) / 2.0 ** 23


def test_pair_normals_symmetric_and_standard():
    rng = np.random.default_rng(3)
    n = 60000
    ii = rng.integers(0, 2**24, n)
    jj = rng.integers(0, 2**24, n)
    g = np.array([oracle.normal_pair(99, int(a), int(b), 17, 0) for a, b in zip(ii, jj)])
    # symmetric key: xi_ij = xi_ji (Sec. 2.1: xi symmetric)
    for a, b in zip(ii[:200], jj[:200]):
        assert np.array_equal(oracle.normal_pair(99, int(a), int(b), 17, 0),
                              oracle.normal_pair(99, int(b), int(a), 17, 0))
    x = g.ravel()
    se = 1.0 / math.sqrt(x.size)
    assert abs(x.mean()) < 5 * se
    assert abs(x.var() - 1.0) < 5 * math.sqrt(2.0) * se
    assert abs(np.mean(x ** 4) - 3.0) < 5 * math.sqrt(96.0) * se
    assert abs(np.corrcoef(g[:, 0], g[:, 1])[0, 1]) < 5 * se * math.sqrt(2)
    # consecutive pairs, consecutive steps and streams are uncorrelated
    a = np.array([oracle.normal_pair(99, k, k + 1, 0, 0)[0] for k in range(20000)])
    b = np.array([oracle.normal_pair(99, k, k + 1, 1, 0)[0] for k in range(20000)])
    c = np.array([oracle.normal_pair(99, k, k + 1, 0, 1)[0] for k in range(20000)])
    lim = 5.0 / math.sqrt(20000)
    assert abs(np.corrcoef(a[:-1], a[1:])[0, 1]) < lim
    assert abs(np.corrcoef(a, b)[0, 1]) < lim
    assert abs(np.corrcoef(a, c)[0, 1]) < lim


# --------------------------------------------------------- pair forces

def _cloud(n, L, seed, periodic=(1, 1, 1), **kw):
    rng = np.random.default_rng(seed)
    pos = rng.random((n, 3)) * np.asarray(L)
    vel = rng.normal(0, 1, (n, 3))
    conc = rng.random((n, kw.pop('ns', 1)))
    return custom(pos, vel, conc, L=L, periodic=periodic, ns=conc.shape[1], **kw)


def test_pair_sums_vanish_momentum_and_species():
    """F_ij = -F_ji and Q_ij = -Q_ji, so sum F = 0, sum Q = 0; central
    forces in an open box also give zero total torque."""
    d = _cloud(700, (7.0, 7.0, 7.0), 1, ns=3)
    o = oracle.Oracle(d, mode=0)
    F, Q = o.pair_forces()
    scale = np.abs(F).max()
    assert np.abs(F.sum(0)).max() < 1e-11 * scale * len(F)
    assert np.abs(Q.sum(0)).max() < 1e-12 * np.abs(Q).max() * len(Q)
    d = _cloud(300, (6.0, 6.0, 6.0), 2, periodic=(0, 0, 0))
    o = oracle.Oracle(d, mode=0)
    F, _ = o.pair_forces()
    torque = np.cross(o.pos, F).sum(0)
    assert np.abs(torque).max() < 1e-10 * np.abs(F).max() * len(F)


def test_conservative_force_is_minus_gradient_of_soft_potential():
    """F^C = a w_C e_ij with w_C = 1 - r/rc is -grad of U = sum a rc/2 (1-r/rc)^2."""
    d = _cloud(60, (3.0, 3.0, 3.0), 3, periodic=(0, 0, 0), gamma=0.0, sigma=0.0, kappa=0.0, a=18.75)
    o = oracle.Oracle(d, mode=0)
    F, _ = o.pair_forces()

    def U(p):
        dd = p[:, None, :] - p[None, :, :]
        r = np.sqrt((dd ** 2).sum(-1))
        iu = np.triu_indices(len(p), 1)
        r = r[iu]
        r = r[r < 1.0]
        return (18.75 * 1.0 / 2.0 * (1.0 - r) ** 2).sum()

    h = 1e-6
    G = np.zeros_like(F)
    for i in range(len(F)):
        for c in range(3):
            p = o.pos.copy(); p[i, c] += h; up = U(p)
            p[i, c] -= 2 * h; um = U(p)
            G[i, c] = -(up - um) / (2 * h)
    assert relerr(F, G) < 1e-7


def test_dissipative_force_is_minus_velocity_gradient_of_rayleigh_function():
    """F^D_i = -dR/dv_i with R = 1/2 sum gamma w_D (e.v_ij)^2, w_D = w_R^2; its
    power sum_i F_i.v_i = -2R <= 0."""
    for s_f in (2.0, 0.41):
        d = _cloud(60, (3.0, 3.0, 3.0), 4, periodic=(0, 0, 0), a=0.0, sigma=0.0, kappa=0.0,
                   gamma=4.5, s_f=s_f)
        o = oracle.Oracle(d, mode=0)
        F, _ = o.pair_forces()
        sf = float(np.float32(s_f))   # the exponent as stored (binary32)

        def R(v):
            p = o.pos
            tot = 0.0
            for i in range(len(p)):
                for j in range(i + 1, len(p)):
                    dd = p[i] - p[j]
                    r = np.linalg.norm(dd)
                    if r < 1.0:
                        e = dd / r
                        tot += 0.5 * 4.5 * (1 - r) ** sf * np.dot(e, v[i] - v[j]) ** 2
            return tot

        h = 1e-5
        G = np.zeros_like(F)
        for i in range(len(F)):
            for c in range(3):
                v = o.vel.copy(); v[i, c] += h; rp = R(v)
                v[i, c] -= 2 * h; rm = R(v)
                G[i, c] = -(rp - rm) / (2 * h)
        assert relerr(F, G) < 1e-7
        assert (F * o.vel).sum() == pytest.approx(-2 * R(o.vel), rel=1e-10)


def test_random_force_variance_matches_sigma_wR():
    """F^R = sigma w_R xi dt^-1/2 e: over steps, <F.e> = 0 and
    <(F.e)^2> dt / (sigma w_R)^2 = 1 (Eq. 3, xi ~ N(0,1))."""
    for s_f in (2.0, 0.41):
        d = custom([[1.0, 1.0, 1.0], [1.5, 1.0, 1.0]], L=(5.0, 5.0, 5.0), a=0.0, gamma=0.0,
                   sigma=3.0, kappa=0.0, s_f=s_f, dt=0.01)
        o = oracle.Oracle(d, mode=0)
        wR = 0.5 ** (float(np.float32(s_f)) / 2)
        xs = np.array([o.pair_forces(step=k)[0][0, 0] for k in range(20000)]) * math.sqrt(0.01) / (3.0 * wR)
        # particle 0 sits at smaller x: e_01 = -x_hat
        assert abs(xs.mean()) < 5 / math.sqrt(len(xs))
        assert abs(xs.var() - 1.0) < 5 * math.sqrt(2.0 / len(xs))


def test_cell_list_equals_all_pairs():
    """The cell-list mode sums the same pairs as the O(n^2) mode."""
    for L, ns in (((6.0, 6.0, 6.0), 1), ((5.0, 7.0, 6.0), 3)):
        d = _cloud(int(4 * np.prod(L)), L, 5, ns=ns)
        o = oracle.Oracle(d, mode=0)
        F0, Q0 = o.pair_forces(mode=0)
        F1, Q1 = o.pair_forces(mode=1)
        assert np.abs(F0 - F1).max() < 1e-12 * np.abs(F0).max() * 10
        assert np.abs(Q0 - Q1).max() < 1e-12 * np.abs(Q0).max() * 10


def _mode_rate(k, kappa, rho, rcc, s_c):
    f = lambda r: (1 - r / rcc) ** s_c * (1 - math.sin(k * r) / (k * r)) * 4 * math.pi * r * r
    return kappa * rho * integrate.quad(f, 0, rcc, limit=200)[0]


def test_flux_sine_mode_decay_matches_continuum_integral_and_eq9():
    """For uniformly random particles (g = 1) and C = sin(k x), the Fickian
    flux of Eq. 6 projects on the mode with rate
    kappa rho int w_DC(r) (1 - sin(kr)/(kr)) 4 pi r^2 dr, which tends to
    D^F k^2 with D^F from Eq. 9 as k -> 0."""
    L, rho, kappa, rcc = 10.0, 4.0, 1.0, 1.58
    k = 2 * math.pi / L
    rates = []
    for seed in range(6):
        rng = np.random.default_rng(100 + seed)
        pos = rng.random((int(rho * L ** 3), 3)) * L
        conc = np.sin(k * pos[:, 0:1])
        d = custom(pos, conc=conc, L=(L, L, L), a=0.0, gamma=0.0, sigma=0.0, kappa=kappa, rcc=rcc)
        o = oracle.Oracle(d, mode=1)
        _, Q = o.pair_forces()
        s = np.sin(k * o.pos[:, 0])
        rates.append(-(Q[:, 0] * s).sum() / (s * s).sum())
    expect = _mode_rate(k, kappa, rho, rcc, 2.0)
    assert expect == pytest.approx(0.3039, abs=2e-4)
    assert np.mean(rates) == pytest.approx(expect, rel=0.03)
    # Eq. 9 with g = 1: D^F = (2 pi kappa rho / 3) int_0^rcc r^4 w_DC dr
    DF = 2 * math.pi * kappa * rho / 3 * integrate.quad(lambda r: r ** 4 * (1 - r / rcc) ** 2, 0, rcc)[0]
    assert DF == pytest.approx(2 * math.pi * kappa * rho / 3 * rcc ** 5 / 105, rel=1e-12)
    ks = 1e-3
    assert _mode_rate(ks, kappa, rho, rcc, 2.0) / ks ** 2 == pytest.approx(DF, rel=1e-5)


# ------------------------------------------------------------ integrator

def test_free_particle_under_body_force_is_exact_parabola():
    """GW-VV integrates a constant force exactly: r = r0 + v0 t + f t^2/2, v = v0 + f t."""
    r0 = np.array([[2.0, 3.0, 4.0]])
    v0 = np.array([[0.3, -0.2, 0.1]])
    f = np.array([0.05, 0.0, -0.02])
    d = custom(r0, v0, L=(10.0, 10.0, 10.0), body_force=f)
    o = oracle.Oracle(d, mode=0)
    n = 300
    o.run(n)
    t = n * float(np.float32(0.01))
    rf = (r0.astype(np.float32).astype(float) + v0.astype(np.float32).astype(float) * t
          + 0.5 * f.astype(np.float32).astype(float) * t * t)
    rf = rf - 10.0 * np.floor(rf / 10.0)
    assert np.abs(o.pos - rf).max() < 1e-12
    v32 = v0.astype(np.float32).astype(float)
    f32 = f.astype(np.float32).astype(float)
    assert np.abs(o.vel - (v32 + f32 * t)).max() < 1e-12


def test_body_force_momentum_grows_linearly():
    """Pair forces cancel, so sum p(t) = sum p(0) + N f t."""
    d = _cloud(500, (5.0, 5.0, 5.0), 6, body_force=(0.05, -0.01, 0.0))
    o = oracle.Oracle(d, mode=1)
    p0 = o.vel.sum(0)
    o.run(40)
    t = 40 * float(np.float32(0.01))
    f = np.array([0.05, -0.01, 0.0], np.float32).astype(float)
    assert np.abs(o.vel.sum(0) - (p0 + 500 * f * t)).max() < 1e-9


def test_reaction_total_follows_scalar_recurrence():
    """With A->B at rate k on all particles, the total of A obeys the
    scalar GW-VV recurrence and A + B is conserved; the diffusive flux cancels."""
    rng = np.random.default_rng(7)
    n, kr = 400, 0.5
    pos = rng.random((n, 3)) * 5.0
    conc = np.stack([rng.random(n), np.zeros(n)], 1)
    d = custom(pos, rng.normal(0, 1, (n, 3)), conc, L=(5.0, 5.0, 5.0), ns=2, kappa=1.0,
               reaction=dict(k=kr, src=0, dst=1, types=1))
    o = oracle.Oracle(d, mode=1)
    k = float(np.float32(kr))
    dt = float(np.float32(0.01))
    M = o.conc[:, 0].sum()
    tot = o.conc.sum()
    q = -k * M
    for _ in range(30):
        Mt = M + 0.5 * dt * q
        q2 = -k * Mt
        M = M + 0.5 * dt * (q + q2)
        q = q2
    o.run(30)
    assert o.conc[:, 0].sum() == pytest.approx(M, rel=1e-12)
    assert o.conc.sum() == pytest.approx(tot, rel=1e-12)


def test_conservative_dynamics_conserves_energy():
    """With gamma = sigma = 0 the soft-sphere system is Hamiltonian; velocity
    Verlet keeps E = K + U bounded to O(dt^2)."""
    rng = np.random.default_rng(8)
    L = 5.0
    n = int(3 * L ** 3)
    # start from a relaxed configuration: lattice with small noise
    g = np.stack(np.meshgrid(*[np.arange(5)] * 3, indexing='ij'), -1).reshape(-1, 3)
    pos = np.concatenate([g + 0.25, g + 0.6, g + [0.9, 0.2, 0.5]])[:n] + rng.uniform(-0.05, 0.05, (n, 3))
    pos = np.mod(pos, L)
    d = custom(pos, rng.normal(0, 1, (n, 3)), L=(L, L, L), gamma=0.0, sigma=0.0, kappa=0.0)
    o = oracle.Oracle(d, mode=1)

    def energy():
        p = o.pos
        dd = p[:, None, :] - p[None, :, :]
        dd -= L * np.round(dd / L)
        r = np.sqrt((dd ** 2).sum(-1))
        iu = np.triu_indices(n, 1)
        r = r[iu]
        r = r[r < 1.0]
        return 0.5 * (o.vel ** 2).sum() + (25.0 / 2 * (1 - r) ** 2).sum()

    E0 = energy()
    K0 = 0.5 * (o.vel ** 2).sum()
    es = []
    for _ in range(10):
        o.run(20)
        es.append(energy())
    assert np.max(np.abs(np.array(es) - E0)) < 2e-3 * K0


def test_observables_definitions():
    rng = np.random.default_rng(9)
    d = _cloud(300, (5.0, 5.0, 5.0), 9, ns=2)
    o = oracle.Oracle(d, mode=1)
    ob = o.observables()
    v = o.vel
    assert ob['kT'] == pytest.approx(np.mean([np.var(v[:, c], ddof=1) for c in range(3)]), rel=1e-12)
    assert np.allclose(ob['momentum'], v.sum(0), rtol=1e-12, atol=1e-12)
    assert np.allclose(ob['mass'], o.conc.sum(0), rtol=1e-12)
    assert ob['n_mobile'] == 300


@pytest.mark.slow
def test_equilibrium_temperature_fdt():
    """With sigma^2 = 2 kT gamma and w_D = w_R^2 (Eq. 4) the fluid
    equilibrates at kT = 1 within 1% (4000 particles, dt = 0.01)."""
    d = W.fluid_box(L=10.0, rho=4.0, seed=1001)
    o = oracle.Oracle(d, mode=1)
    o.run(400)
    ks = []
    for _ in range(60):
        o.run(10)
        ks.append(o.observables()['kT'])
    assert abs(np.mean(ks) - 1.0) < 0.01


# ------------------------------------------------------------- membrane

def _perturbed_sphere(n=42, radius=2.0, seed=0, dx=0.08, **mem):
    v, t = small_sphere(n, radius)
    rng = np.random.default_rng(seed)
    u = v * 1.04 + rng.uniform(-dx, dx, v.shape)
    return membrane_only(u, t, rest=v, **mem)


@pytest.mark.parametrize('parts', [1, 4, 8, 13])
@pytest.mark.parametrize('theta0', [0.0, 0.1])
def test_membrane_conservative_forces_are_minus_energy_gradient(parts, theta0):
    """Bond (Eq. 10-11), area/volume (Eq. 14-15) and bending (Eq. 16)
    forces equal -grad of their energies (central differences)."""
    d = _perturbed_sphere(theta0=theta0)
    o = oracle.Oracle(d, mode=1)
    F, _ = o.membrane_forces(parts=parts)
    h = 1e-6
    G = np.zeros_like(F)
    for i in range(o.n):
        for c in range(3):
            p = o.pos.copy(); p[i, c] += h; ep = o.membrane_energy(p, parts)
            p[i, c] -= 2 * h; em = o.membrane_energy(p, parts)
            G[i, c] = -(ep - em) / (2 * h)
    assert relerr(F, G) < 2e-6


def test_membrane_conservative_forces_free_of_net_force_and_torque():
    d = _perturbed_sphere(seed=1, theta0=0.1)
    o = oracle.Oracle(d, mode=1)
    F, _ = o.membrane_forces(parts=13)
    s = np.abs(F).max() * o.n
    assert np.abs(F.sum(0)).max() < 1e-12 * s
    c = o.pos.mean(0)
    assert np.abs(np.cross(o.pos - c, F).sum(0)).max() < 1e-12 * s * 3


def test_bonds_are_force_free_at_rest_length():
    v, t = small_sphere(42, 2.0)
    o = oracle.Oracle(membrane_only(v, t), mode=1)
    F, _ = o.membrane_forces(parts=1)
    assert np.abs(F).max() < 1e-9


@pytest.mark.parametrize('edge', [1.0, 2.0])
def test_icosahedron_area_volume_and_angles(edge):
    """The gather of Eq. 14-15 and the angle of Eq. 16 on a regular
    icosahedron equal the textbook values."""
    row = [r for r in read_golden('icosahedron.txt') if float(r[0]) == edge][0]
    A, V, cth = float(row[1]), float(row[2]), float(row[3])
    v, t = icosahedron(edge)
    o = oracle.Oracle(membrane_only(v, t), mode=1)
    ob = o.observables()
    assert ob['area'][0] == pytest.approx(A, rel=1e-6)
    assert ob['volume'][0] == pytest.approx(V, rel=1e-6)
    th = o.membrane_angles()
    assert np.allclose(np.cos(th), cth, atol=1e-6)
    assert (th > 0).all()
    # bending energy of the solid: 30 edges of k_b (1 - cos(theta - theta0))
    assert o.membrane_energy(parts=8) == pytest.approx(30 * 20.0 * (1 - cth), rel=1e-6)


def test_sphere_mesh_area_volume_converge():
    """The gather on inscribed triangulations of a sphere stays below
    4 pi R^2 and 4/3 pi R^3 and converges to them at first order in 1/n."""
    errs = []
    for n in (500, 2000):
        v, t = small_sphere(n, 3.0)
        o = oracle.Oracle(membrane_only(v, t), mode=1)
        ob = o.observables()
        eA = 1 - ob['area'][0] / (4 * math.pi * 9.0)
        eV = 1 - ob['volume'][0] / (4 / 3 * math.pi * 27.0)
        assert 0 < eA < 1e-2 and 0 < eV < 2e-2
        errs.append((eA, eV))
    assert errs[1][0] < errs[0][0] / 3 and errs[1][1] < errs[0][1] / 3


def test_bond_dissipation_is_minus_velocity_gradient():
    """Eq. 12: F^D = -gT v_ij - gC (v_ij.e) e is -dR/dv of
    R = 1/2 sum_bonds [gT |v_ij|^2 + gC (v_ij.e)^2] (random part off: kT = 0)."""
    v, t = small_sphere(42, 2.0)
    rng = np.random.default_rng(11)
    vel = rng.normal(0, 1, v.shape)
    o = oracle.Oracle(membrane_only(v, t, vel=vel, kT=0.0), mode=1)
    F, _ = o.membrane_forces(parts=2)
    from workloads.mesh import edges_of
    E = edges_of(t)

    def R(vv):
        d = o.pos[E[:, 0]] - o.pos[E[:, 1]]
        e = d / np.linalg.norm(d, axis=1)[:, None]
        vij = vv[E[:, 0]] - vv[E[:, 1]]
        return 0.5 * (6.0 * (vij ** 2).sum(1) + 3.0 * (vij * e).sum(1) ** 2).sum()

    h = 1e-5
    G = np.zeros_like(F)
    for i in range(o.n):
        for c in range(3):
            vv = o.vel.copy(); vv[i, c] += h; rp = R(vv)
            vv[i, c] -= 2 * h; rm = R(vv)
            G[i, c] = -(rp - rm) / (2 * h)
    assert relerr(F, G) < 1e-8


def test_bond_random_force_covariance_satisfies_fdt():
    """Eq. 13: the random bond force has covariance (2kT/dt)(gT I + gC e e^T)
    per bond, the fluctuation partner of Eq. 12."""
    v, t = icosahedron(1.0)
    o = oracle.Oracle(membrane_only(v, t, kT=1.0), mode=1)
    samples = np.array([o.membrane_forces(parts=2, step=k)[0][0] for k in range(20000)])
    from workloads.mesh import edges_of
    E = edges_of(t)
    C = np.zeros((3, 3))
    dt = float(np.float32(0.01))
    for a, b in E:
        if 0 in (a, b):
            d = o.pos[a] - o.pos[b]
            e = d / np.linalg.norm(d)
            C += 2.0 / dt * (6.0 * np.eye(3) + 3.0 * np.outer(e, e))
    S = np.cov(samples.T)
    assert np.abs(samples.mean(0)).max() < 5 * math.sqrt(C.max() / len(samples))
    assert np.abs(S - C).max() < 0.05 * C.max()


def test_lagged_area_volume_uses_previous_totals():
    """Sec. 3.3 concurrent variant: an evaluation with lagged area and volume
    differs from the sequential one only by the constraint coefficients,
    taken at the previous evaluation's totals (A', V') instead of the current
    ones (A, V): F_lag - F_seq = -(k_g (A' - A)/A0) grad A - (k_v (V' - V)/V0)
    grad V, with grad A and grad V by central differences of the totals; an
    unmoved state gives the sequential forces; the first evaluation after a
    state is loaded is the sequential one."""
    d = _perturbed_sphere(seed=3, kT=0.0)
    seq = oracle.Oracle(d, mode=1)
    d_lag = _perturbed_sphere(seed=3, kT=0.0, lagged_av=1)
    lag = oracle.Oracle(d_lag, mode=1)
    assert np.array_equal(lag.F, seq.F)                      # first evaluation
    x0 = seq.pos.copy()
    _, AV0 = seq.membrane_forces(parts=0)
    # a second evaluation of the unmoved state: previous totals = current
    F1, _ = lag.forces()
    assert relerr(F1, seq.F) < 1e-14
    # move the vertices, evaluate lagged (previous totals: those at x0)
    rng = np.random.default_rng(4)
    x1 = x0 + rng.uniform(-0.03, 0.03, x0.shape)
    lag.forces(pos=x0)                                        # totals at x0 carried
    F_lag, _ = lag.forces(pos=x1)
    F_seq, _ = seq.forces(pos=x1)
    _, AV1 = seq.membrane_forces(pos=x1, parts=0)
    h = 1e-6
    gA = np.zeros_like(x1)
    gV = np.zeros_like(x1)
    for i in range(seq.n):
        for c in range(3):
            p = x1.copy(); p[i, c] += h; _, ap = seq.membrane_forces(pos=p, parts=0)
            p[i, c] -= 2 * h; _, am = seq.membrane_forces(pos=p, parts=0)
            gA[i, c] = (ap[0, 0] - am[0, 0]) / (2 * h)
            gV[i, c] = (ap[0, 1] - am[0, 1]) / (2 * h)
    _, _, A0, V0 = seq.membrane_rest()
    mp = d['membrane']
    expect = -(mp['kg'] * (AV0[0, 0] - AV1[0, 0]) / A0[0]) * gA - (mp['kv'] * (AV0[0, 1] - AV1[0, 1]) / V0[0]) * gV
    assert np.linalg.norm(F_lag - F_seq) > 1e-3 * np.linalg.norm(F_seq)
    assert relerr(F_lag - F_seq, expect) < 1e-5


def test_random_flux_exchanges_solute_and_scales_with_its_strength():
    """Eq. 7: each pair's random flux leaves i and enters j (zeta_ji =
    -zeta_ij), so every species total stays conserved to rounding with the
    random flux on; the random part is linear in m_s and vanishes at m_s = 0."""
    d = _cloud(300, (6.0, 6.0, 6.0), 21, ns=3)
    base = oracle.Oracle(d, mode=1)
    parts = []
    for ms in (0.05, 0.1):
        d['random_flux'] = dict(m_s=ms, rho=3.0)
        o = oracle.Oracle(d, mode=1)
        assert np.abs(o.Q.sum(axis=0)).max() < 1e-12 * np.abs(o.Q).sum()
        parts.append(o.Q - base.Q)
    assert np.linalg.norm(parts[0]) > 1e-3 * np.linalg.norm(base.Q)
    assert relerr(parts[1], 2.0 * parts[0]) < 1e-6
    d['random_flux'] = dict(m_s=0.0, rho=3.0)
    assert np.array_equal(oracle.Oracle(d, mode=1).Q, base.Q)


def test_random_flux_equilibrium_variance_matches_fdt():
    """Eq. 8 fluctuation-dissipation balance: with the Fickian and random
    fluxes on fixed particles around a uniform concentration C0, the
    linearised dynamics dC = -L C dt + B dW has B B^T = 2 m_s^2 rho C0 L
    (w_RC^2 = w_DC), so the stationary covariance is m_s^2 rho C0 times the
    projector off the uniform mode: the spread of C over the particles has
    mean square m_s^2 rho C0 (N - 1)/N, whatever the positions and kappa."""
    n, L = 400, 5.1
    rng = np.random.default_rng(5)
    pos = rng.random((n, 3)) * L
    ms, rho, c0 = 0.1, 3.0, 1.0
    d = custom(pos, None, np.full((n, 1), c0), L=(L, L, L), a=0.0, gamma=0.0, sigma=0.0, kappa=0.5,
               dt=0.01, seed=11)
    d['random_flux'] = dict(m_s=ms, rho=rho)
    o = oracle.Oracle(d, mode=1)
    o.run(1000)                                  # slowest mode relaxes in ~170 steps
    samples = []
    for _ in range(100):
        o.run(20)
        samples.append(np.var(o.conc[:, 0]))
    assert np.abs(o.pos - pos.astype(np.float32)).max() == 0.0     # nothing moved
    expect = ms * ms * rho * c0 * (n - 1) / n
    assert np.mean(samples) == pytest.approx(expect, rel=0.02)


def test_flipped_body_force_drives_each_half_oppositely():
    """Double Poiseuille forcing (Sec. 4.1): +f below z = L/2, -f above. Two
    free particles, one in each half and moving only along x, follow exact
    parabolas of opposite curvature; with the flip off both take +f."""
    r0 = np.array([[2.0, 3.0, 2.5], [2.0, 6.0, 7.5]])
    f = np.array([0.05, 0.0, 0.0])
    d = custom(r0, np.zeros((2, 3)), L=(10.0, 10.0, 10.0), body_force=f)
    d['body_force_flip'] = 1
    o = oracle.Oracle(d, mode=0)
    o.run(200)
    t = 200 * float(np.float32(0.01))
    f32 = float(np.float32(0.05))
    assert o.vel[0, 0] == pytest.approx(f32 * t, abs=1e-12)
    assert o.vel[1, 0] == pytest.approx(-f32 * t, abs=1e-12)
    x = np.array([2.0 + 0.5 * f32 * t * t, 2.0 - 0.5 * f32 * t * t]) % 10.0
    assert np.abs(o.pos[:, 0] - x).max() < 1e-12
    d['body_force_flip'] = 0
    o = oracle.Oracle(d, mode=0)
    o.run(200)
    assert np.abs(o.vel[:, 0] - f32 * t).max() < 1e-12


def test_membrane_relaxes_to_its_area_and_volume_targets():
    """Area and volume constraints (Eq. 14-15) hold a cell at its targets: a
    500-vertex biconcave membrane started 1.2 % above its target volume, with
    the bond viscosity of Eq. 12 and no thermal noise, settles within 1e-3 of
    A0 and V0 (the penalty balances the bond and bending forces a few 1e-4
    off the targets)."""
    verts, tri = W.biconcave_mesh(500, 8.0)
    d = membrane_only(verts, tri, L=30.0, kT=0.0)
    d['dt'] = np.float32(0.005)
    o = oracle.Oracle(d, mode=1)
    _, _, A0, V0 = o.membrane_rest()
    _, AV = o.membrane_forces(parts=0)
    assert abs(AV[0, 1] - V0[0]) / V0[0] > 0.01
    o.run(2000)
    _, AV = o.membrane_forces(parts=0)
    assert abs(AV[0, 0] - A0[0]) / A0[0] < 1e-3
    assert abs(AV[0, 1] - V0[0]) / V0[0] < 1e-3


def test_cylinder_wall_reflects_radially():
    """Bounce-back at the cylinder of the transport validation (Sec. 4.2,
    Eq. 17): a free particle whose predicted position lies outside radius R
    of the axis lands on the same radial line at distance 2R - d, with x
    untouched and its velocity reversed; one that stays inside moves freely."""
    L, R = 10.0, 3.0
    r0 = np.array([[2.0, 7.0, 7.0], [4.0, 5.0, 6.0]])        # radial 2.83 and 1.0
    v0 = np.array([[0.5, 20.0, 20.0], [1.0, 2.0, -3.0]])
    d = custom(r0, v0, L=(L, L, L), a=0.0, gamma=0.0, sigma=0.0, kappa=0.0)
    d['cylinder_radius'] = np.float32(R)
    o = oracle.Oracle(d, mode=0)
    p32 = d['particles']['pos'].astype(np.float64)
    v32 = d['particles']['vel'].astype(np.float64)
    dt = float(np.float32(0.01))
    o.run(1)
    pred = p32 + dt * v32
    c = np.array([L / 2, L / 2])
    # particle 0 crossed the surface
    u = pred[0, 1:] - c
    dist = math.hypot(*u)
    assert dist > R
    w = o.pos[0, 1:] - c
    assert math.hypot(*w) == pytest.approx(2 * R - dist, abs=1e-12)
    assert w[0] * u[1] - w[1] * u[0] == pytest.approx(0.0, abs=1e-12)   # same radial line
    assert np.dot(w, u) > 0
    assert o.pos[0, 0] == pytest.approx(pred[0, 0], abs=1e-12)
    assert np.allclose(o.vel[0], -v32[0], atol=1e-12)
    # particle 1 stayed inside
    assert np.allclose(o.pos[1], pred[1], atol=1e-12)
    assert np.allclose(o.vel[1], v32[1], atol=1e-12)


def test_cylinder_keeps_fluid_inside_and_reservoir_fixed():
    """The small cylinder workload on the oracle: after 20 steps every fluid
    particle is within R of the axis, the frozen shell has not moved and still
    holds the boundary concentration, and solute has entered the fluid."""
    d = W.cylinder_diffusion(R=3.0, Lx=6.0, seed=31)
    p = d['particles']
    wall = p['type'] == W.WALL
    o = oracle.Oracle(d, mode=1)
    o.run(20)
    c = 0.5 * d['L'].astype(np.float64)
    rad = np.hypot(o.pos[:, 1] - c[1], o.pos[:, 2] - c[2])
    assert rad[~wall].max() <= 3.0 + 1e-12
    assert np.array_equal(o.pos[wall], p['pos'][wall].astype(np.float64))
    assert np.all(o.conc[wall] == 1.0)
    assert o.conc[~wall].sum() > 0.0


def test_planar_walls_reflect_and_reverse():
    """Bounce-back at the planar walls of the channel workload (the reading
    of the wall treatment Sec. 4.2 cites but does not state): a particle
    whose predicted z passes wall_hi (wall_lo) lands at 2 wall_hi - z
    (2 wall_lo - z) with x, y as predicted and its velocity reversed before
    the corrector adds the force; a particle that stays between the walls
    moves freely. With no pair forces the force is the body force f, so the
    corrector gives v' = -v + dt f after a reflection and v + dt f without."""
    L, lo, hi = 10.0, 1.0, 9.0
    r0 = np.array([[2.0, 3.0, 8.9], [4.0, 5.0, 1.05], [6.0, 7.0, 5.0]])
    v0 = np.array([[0.5, -1.0, 30.0], [1.0, 2.0, -20.0], [0.3, 0.2, -0.4]])
    f = np.array([0.05, -0.02, 0.1])
    d = custom(r0, v0, L=(L, L, L), periodic=(1, 1, 0), a=0.0, gamma=0.0, sigma=0.0, kappa=0.0,
               body_force=f)
    d['wall_lo'], d['wall_hi'] = np.float32(lo), np.float32(hi)
    o = oracle.Oracle(d, mode=0)
    p32 = d['particles']['pos'].astype(np.float64)
    v32 = d['particles']['vel'].astype(np.float64)
    f32 = d['body_force'].astype(np.float64)
    dt = float(np.float32(0.01))
    o.run(1)
    pred = p32 + dt * v32 + 0.5 * dt * dt * f32
    assert pred[0, 2] > hi and pred[1, 2] < lo and lo < pred[2, 2] < hi
    assert o.pos[0, 2] == pytest.approx(2 * hi - pred[0, 2], abs=1e-12)
    assert o.pos[1, 2] == pytest.approx(2 * lo - pred[1, 2], abs=1e-12)
    assert np.allclose(o.pos[:2, :2], pred[:2, :2], atol=1e-12)
    assert np.allclose(o.vel[:2], -v32[:2] + dt * f32, atol=1e-12)
    assert np.allclose(o.pos[2], pred[2], atol=1e-12)
    assert np.allclose(o.vel[2], v32[2] + dt * f32, atol=1e-12)


def _two_icosahedra(exclude=1, only_first=False):
    """Two regular icosahedra (edge 0.8 < r_c, so the vertices of one cell
    are inside each other's force range) whose faces come within r_c of each
    other, with random velocities and concentrations."""
    v, t = icosahedron(0.8)
    rng = np.random.default_rng(17)
    d = membrane_only(v, t, L=12.0, vel=rng.normal(0, 1, v.shape))
    d['a'][:] = 25.0
    d['gamma'][:] = 4.5
    d['sigma'][:] = 3.0
    d['kappa'][:] = 1.0
    d['exclude_same_body'] = exclude
    r = d['rbcs'][0]
    r['conc'] = rng.random((12, 1)).astype(np.float32)
    if not only_first:
        r2 = dict(r)
        r2['pos'] = (r['pos'].astype(np.float64) + [1.3, 0.2, 0.1]).astype(np.float32)
        r2['vel'] = rng.normal(0, 1, v.shape).astype(np.float32)
        r2['conc'] = rng.random((12, 1)).astype(np.float32)
        d['rbcs'] = [r, r2]
    return d


def test_same_membrane_pairs_feel_no_force_but_exchange_flux():
    """The membrane-solvent reading of Sec. 2.2: vertices of one membrane
    exert no Eq. 3 force on each other, but exchange the Eq. 6 flux; vertices
    of two different membranes interact fully. One cell alone: every pair
    force is zero, the flux is not. Two cells: the force on a vertex of the
    first equals its force with the exclusion off minus its force from its
    own cell (the first cell alone, exclusion off, same ids and step), and
    the flux does not depend on the exclusion."""
    o1 = oracle.Oracle(_two_icosahedra(1, only_first=True), mode=0)
    F1, Q1 = o1.pair_forces()
    assert np.all(F1 == 0.0)
    assert np.abs(Q1).max() > 1e-2
    o1n = oracle.Oracle(_two_icosahedra(0, only_first=True), mode=0)
    Fself, Q1n = o1n.pair_forces()
    assert np.abs(Fself).max() > 1.0              # the same pairs do interact when not excluded
    assert np.array_equal(Q1, Q1n)
    oe = oracle.Oracle(_two_icosahedra(1), mode=0)
    on = oracle.Oracle(_two_icosahedra(0), mode=0)
    Fe, Qe = oe.pair_forces()
    Fn, Qn = on.pair_forces()
    assert np.abs(Fe[:12]).max() > 1.0            # cross-membrane pairs interact
    assert np.allclose(Fe[:12], Fn[:12] - Fself, rtol=0, atol=1e-12 * np.abs(Fn).max())
    assert np.allclose(Qe, Qn, rtol=0, atol=1e-15)
    # the second cell: its own-cell forces are the first cell's pattern moved
    assert np.allclose(Fe.sum(0), 0.0, atol=1e-10 * np.abs(Fe).max())


def test_unwrap_across_periodic_faces_is_translation_invariant():
    """Area, volume (Eq. 14-15) and every membrane force of a cell do not
    change when the cell is translated across a periodic corner of the box so
    that its vertices are wrapped to three faces: the oracle rebuilds the
    cell by minimum images along its edges before summing. Without the
    unwrap the wrapped coordinates would give a different area and volume
    (checked by summing the triangles of the raw wrapped positions)."""
    d = _perturbed_sphere(n=162, radius=3.0, seed=9, theta0=0.1)
    L = float(d['L'][0])
    rng = np.random.default_rng(2)
    vel = rng.normal(0, 1, (162, 3))
    o = oracle.Oracle(d, mode=1)
    p0 = o.pos.copy()
    F0, AV0 = o.membrane_forces(pos=p0, vel=vel, parts=15)
    shift = np.array([L / 2 - 0.4, L / 2 + 0.3, -L / 2 + 0.2])
    p1 = p0 + shift
    p1 -= np.floor(p1 / L) * L
    for c in range(3):
        assert p1[:, c].min() < 2.0 and p1[:, c].max() > L - 2.0   # split across every axis
    F1, AV1 = o.membrane_forces(pos=p1, vel=vel, parts=15)
    assert np.allclose(AV1, AV0, rtol=1e-11, atol=0)
    assert np.allclose(F1, F0, rtol=0, atol=1e-9 * np.abs(F0).max())
    tri = d['rbcs'][0]['tri']
    a, b, c = p1[tri[:, 0]], p1[tri[:, 1]], p1[tri[:, 2]]
    raw_area = 0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1).sum()
    assert abs(raw_area - AV0[0, 0]) > 0.1 * AV0[0, 0]
