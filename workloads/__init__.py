"""Seeded synthetic inputs for the tDPD + RBC step.

This module only draws inputs: particle positions, velocities and
concentrations, triangulated membrane meshes and their placement, and the
parameter values of each workload. It contains none of the method's
arithmetic (no forces, fluxes, energies or integration); both the CUDA path
and the CPU oracle consume what it returns.

A workload description is a plain dict (see ``fluid_box`` and ``single_rbc``)
holding numpy arrays in float32 / int32, the precision the library stores.

Particle identities follow the load order: free particles get ids 0..n-1 in
the order given, then the vertices of each membrane are appended, membrane
by membrane, in vertex order. The pairwise random numbers are keyed on these
ids, so both implementations see the same random stream.
"""

from __future__ import annotations

import math

import numpy as np

from .mesh import biconcave_mesh, sphere_mesh, fibonacci_sphere  # noqa: F401

SOLVENT, MEMBRANE, WALL = 0, 1, 2

# Evans-Fung reference cell: diameter 7.82 um, area ~135 um^2, volume ~94 um^3.
# Only the ratio V/A^1.5 of that reference enters (the area-volume scaling of
# the RBC model, Sec. 2.2); its value 94/135^1.5 = 0.0599.
RBC_V_RATIO = 94.0 / 135.0 ** 1.5


def _rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence(int(seed)))


def membrane_defaults(kT: float = 1.0) -> dict:
    """Membrane parameters used by the RBC workloads (DPD units).

    x0 = l0/l_m = 1/2.2 and m = 2 (stress-free WLC-POW bonds), persistence
    length p = 0.05, k_g = k_v = 5000, k_l = 500, k_b = 20 kT, theta0 = 0,
    gamma_T = 6, gamma_C = 3 (3*gamma_C >= gamma_T keeps the trace part of the
    random bond force real), reduced volume V0/A0^1.5 of the Evans-Fung cell.
    The local area stiffness k_l = 500 keeps the triangles of the small
    (diameter 5) cells from degenerating: with k_l = 100 a few replicas in a
    thousand blew up within t = 10 at dt = 0.005, none with 500. Area and
    volume constraints are evaluated at the current positions (lagged_av = 0).
    """
    return dict(kT=kT, p=0.05, x0=1.0 / 2.2, m=2.0, kg=5000.0, kl=500.0,
                kv=5000.0, kb=20.0 * kT, theta0=0.0, gammaT=6.0, gammaC=3.0,
                v_ratio=RBC_V_RATIO, lagged_av=0)


def _base(name, L, periodic, n_types, n_species, seed, rho, dt=0.01, kT=1.0,
          rc=1.0, s_f=2.0, rcc=1.58, s_c=2.0, gamma=4.5):
    a = 75.0 * kT / rho
    sigma = math.sqrt(2.0 * kT * gamma)
    T = n_types
    d = dict(
        name=name,
        L=np.asarray(L, np.float32),
        periodic=np.asarray(periodic, np.int32),
        wall_lo=np.float32(0.0), wall_hi=np.float32(0.0),
        n_types=T, n_species=n_species, seed=int(seed),
        dt=np.float32(dt), lam=np.float32(0.5), kT=np.float32(kT),
        rc=np.float32(rc), s_f=np.float32(s_f), rcc=np.float32(rcc), s_c=np.float32(s_c),
        a=np.full((T, T), a, np.float32),
        gamma=np.full((T, T), gamma, np.float32),
        sigma=np.full((T, T), sigma, np.float32),
        kappa=np.ones((T, T, n_species), np.float32),
        body_force=np.zeros(3, np.float32),
        frozen_types=0, exclude_same_body=1,
        reaction=None, membrane=None,
        particles=None, rbcs=[],
        rho=float(rho),
    )
    return d


def fluid_particles(rng, L, rho, n_species, kT=1.0, lo=None, hi=None, ptype=SOLVENT):
    """Uniform positions in the box (or slab [lo, hi) along z), Maxwell
    velocities at kT with the mean removed, concentrations U[0, 1)."""
    L = np.asarray(L, np.float64)
    zlo = 0.0 if lo is None else lo
    zhi = L[2] if hi is None else hi
    vol = L[0] * L[1] * (zhi - zlo)
    n = int(round(rho * vol))
    pos = rng.random((n, 3))
    pos[:, 0] *= L[0]
    pos[:, 1] *= L[1]
    pos[:, 2] = zlo + pos[:, 2] * (zhi - zlo)
    pos = np.minimum(pos.astype(np.float32), np.nextafter(L.astype(np.float32), 0))
    vel = rng.normal(0.0, math.sqrt(kT), (n, 3))
    if n > 1:
        vel -= vel.mean(axis=0)
    conc = rng.random((n, n_species))
    return dict(pos=pos, vel=vel.astype(np.float32), conc=conc.astype(np.float32),
                type=np.full(n, ptype, np.int32))


def fluid_box(L=10.0, rho=4.0, n_species=1, seed=1001, kT=1.0, **kw):
    """Plain tDPD fluid in a periodic cube (4000 particles at L=10, rho=4)."""
    d = _base('fluid', (L, L, L), (1, 1, 1), 1, n_species, seed, rho, kT=kT, **kw)
    d['particles'] = fluid_particles(_rng(seed), d['L'], rho, n_species, kT)
    return d


def double_poiseuille(L=40.0, rho=4.0, f=0.02, seed=1005, Lxy=None):
    """The flow validation setup of Sec. 4.1: a periodic cube of tDPD fluid
    (40^3 at rho = 4: 256,000 particles) with a = 18.75, gamma = 4.5,
    r_c = 1.58 and w_R exponent s = 0.41, driven along x by a body force f
    below z = L/2 and -f above it (double Poiseuille flow). The paper does
    not give f. Lxy (default L) sets the box edges along x and y."""
    Lxy = L if Lxy is None else Lxy
    d = _base('double_poiseuille', (Lxy, Lxy, L), (1, 1, 1), 1, 1, seed, rho, rc=1.58, s_f=0.41)
    d['a'][:] = 18.75
    d['particles'] = fluid_particles(_rng(seed), d['L'], rho, 1)
    d['body_force'] = np.asarray([f, 0.0, 0.0], np.float32)
    d['body_force_flip'] = 1
    return d


def _annulus(rng, n, r0, r1, L, cy, cz):
    """n points uniform in the shell r0 <= distance from the axis < r1 of a
    cylinder along x (length L)."""
    rad = np.sqrt(r0 * r0 + rng.random(n) * (r1 * r1 - r0 * r0))
    th = rng.random(n) * 2.0 * math.pi
    pos = np.empty((n, 3))
    pos[:, 0] = rng.random(n) * L
    pos[:, 1] = cy + rad * np.cos(th)
    pos[:, 2] = cz + rad * np.sin(th)
    return pos


def cylinder_diffusion(R=20.0, Lx=80.0, rho=4.0, kappa=5.0, c0=0.0, cd=1.0, seed=1006):
    """The transport validation setup of Sec. 4.2 (Eq. 17): tDPD fluid filling
    a cylinder of radius R along x (R = 20 and length 80 at rho = 4: about
    402,000 particles), a = 18.75, gamma = 4.5, r_c = r_cc = 1.58, w_R
    exponent s = 0.41, flux exponent 2, kappa = 5. The fluid starts at
    concentration c0; frozen wall particles (type WALL) at the same density
    fill the shell R <= distance < R + r_cc and hold the boundary
    concentration cd (the paper's effective boundary method is not stated;
    a frozen reservoir in contact over the flux cut-off stands in for it).
    Fluid particles are reflected at the cylinder surface. The box is
    Lx x W x W with W = 2 (R + r_cc) + 1, periodic."""
    rng = _rng(seed)
    rcc = 1.58
    W = float(math.ceil(2.0 * (R + rcc) + 1.0))
    d = _base('cylinder_diffusion', (Lx, W, W), (1, 1, 1), 3, 1, seed, rho, rc=1.58, s_f=0.41)
    d['a'][:] = 18.75
    d['kappa'][:] = np.float32(kappa)
    d['frozen_types'] = 1 << WALL
    n_f = int(round(rho * math.pi * R * R * Lx))
    n_w = int(round(rho * math.pi * ((R + rcc) ** 2 - R * R) * Lx))
    c = 0.5 * W
    pf = _annulus(rng, n_f, 0.0, R, Lx, c, c)
    pw = _annulus(rng, n_w, R, R + rcc, Lx, c, c)
    pos = np.concatenate([pf, pw]).astype(np.float32)
    # keep the fluid strictly inside R after rounding to float32
    r32 = np.sqrt((pos[:n_f, 1].astype(np.float64) - c) ** 2 + (pos[:n_f, 2].astype(np.float64) - c) ** 2)
    pos[np.flatnonzero(r32 > R * (1 - 1e-6)), 1:] = np.float32(c)
    vel = np.zeros((n_f + n_w, 3))
    vel[:n_f] = rng.normal(0.0, 1.0, (n_f, 3))
    vel[:n_f] -= vel[:n_f].mean(axis=0)
    conc = np.concatenate([np.full((n_f, 1), c0), np.full((n_w, 1), cd)]).astype(np.float32)
    typ = np.concatenate([np.full(n_f, SOLVENT), np.full(n_w, WALL)]).astype(np.int32)
    d['particles'] = dict(pos=pos, vel=vel.astype(np.float32), conc=conc, type=typ)
    d['cylinder_radius'] = np.float32(R)
    return d


def place_rbc(mesh_verts, mesh_tri, center, L, rng, kT=1.0, n_species=1, c_value=1.0,
              rest=None):
    """One membrane: vertices translated to ``center`` and wrapped into the box."""
    v = mesh_verts + np.asarray(center, np.float64)[None, :]
    Lf = np.asarray(L, np.float64)
    v = v - np.floor(v / Lf) * Lf
    v = np.minimum(v.astype(np.float32), np.nextafter(Lf.astype(np.float32), 0))
    nv = v.shape[0]
    vel = rng.normal(0.0, math.sqrt(kT), (nv, 3))
    vel -= vel.mean(axis=0)
    conc = np.full((nv, n_species), 0.0, np.float32)
    conc[:, 0] = c_value
    return dict(pos=v, vel=vel.astype(np.float32), conc=conc, type=MEMBRANE,
                tri=np.ascontiguousarray(mesh_tri, np.int32),
                rest=None if rest is None else np.asarray(rest, np.float32))


# Time step of the workloads with membranes. The configurations fix dt = 0.01
# only for the plain fluid; with 500-vertex membranes the bending and bond
# terms make explicit velocity Verlet unstable at 0.01 (the FP64 oracle blows
# up within a few hundred steps on the small-cell replicas) and stable at 0.005.
MEMBRANE_DT = 0.005


def single_rbc(L=20.0, rho=3.0, nv=500, diameter=8.0, permeability=0.1, seed=1002,
               kT=1.0, **kw):
    """One biconcave 500-vertex RBC in tDPD solvent (20^3 box, rho=3, 24k solvent).

    Solvent fills the box inside and outside the membrane. Species 0 starts at
    1 on the membrane and 0 in the solvent; the membrane-solvent transfer
    coefficient is the permeability, solvent-solvent and membrane-membrane 1.
    """
    kw.setdefault('dt', MEMBRANE_DT)
    d = _base('single_rbc', (L, L, L), (1, 1, 1), 2, 1, seed, rho, kT=kT, **kw)
    rng = _rng(seed)
    d['particles'] = fluid_particles(rng, d['L'], rho, 1, kT)
    d['particles']['conc'][:] = 0.0
    verts, tri = biconcave_mesh(nv, diameter)
    d['rbcs'] = [place_rbc(verts, tri, 0.5 * d['L'].astype(np.float64), d['L'], rng, kT)]
    k = d['kappa']
    k[SOLVENT, MEMBRANE, 0] = k[MEMBRANE, SOLVENT, 0] = permeability
    d['membrane'] = membrane_defaults(kT)
    return d


def rbc_channel(Lx=64.0, Ly=32.0, H=32.0, rho=3.0, n_rbc=40, nv=500, diameter=11.85,
                body_force=0.05, k_react=0.01, seed=1003, kT=1.0, permeability=0.1, **kw):
    """RBC suspension in a z-walled channel of height H (fluid region), periodic in
    x and y. Frozen wall particles fill slabs of thickness r_cc at rho outside
    the bounce-back planes. Two species, reaction A->B (rate k) in the solvent.
    40 cells of diameter ~11.85 give ~20% haematocrit."""
    rcc = float(kw.get('rcc', 1.58))
    w = rcc
    Lz = H + 2.0 * w
    kw.setdefault('dt', MEMBRANE_DT)
    d = _base('rbc_channel', (Lx, Ly, Lz), (1, 1, 0), 3, 2, seed, rho, kT=kT, **kw)
    d['wall_lo'] = np.float32(w)
    d['wall_hi'] = np.float32(Lz - w)
    rng = _rng(seed)
    fl = fluid_particles(rng, d['L'], rho, 2, kT, lo=w, hi=Lz - w)
    fl['conc'][:] = 0.0
    wl0 = fluid_particles(rng, d['L'], rho, 2, kT, lo=0.0, hi=w, ptype=WALL)
    wl1 = fluid_particles(rng, d['L'], rho, 2, kT, lo=Lz - w, hi=Lz, ptype=WALL)
    parts = {k: np.concatenate([fl[k], wl0[k], wl1[k]]) for k in fl}
    nwall = wl0['pos'].shape[0] + wl1['pos'].shape[0]
    parts['vel'][-nwall:] = 0.0
    parts['conc'][-nwall:] = 0.0
    d['particles'] = parts
    verts, tri = biconcave_mesh(nv, diameter)
    nx, ny = 4, 2
    nz = int(math.ceil(n_rbc / (nx * ny)))
    rbcs = []
    for iz in range(nz):
        for iy in range(ny):
            for ix in range(nx):
                if len(rbcs) == n_rbc:
                    break
                c = ((ix + 0.5) * Lx / nx, (iy + 0.5) * Ly / ny, w + (iz + 0.5) * H / nz)
                r = place_rbc(verts, tri, c, d['L'], rng, kT, n_species=2)
                rbcs.append(r)
    d['rbcs'] = rbcs
    d['body_force'] = np.asarray([body_force, 0.0, 0.0], np.float32)
    d['frozen_types'] = 1 << WALL
    k = d['kappa']
    k[:] = 1.0
    k[SOLVENT, MEMBRANE, :] = k[MEMBRANE, SOLVENT, :] = permeability
    k[WALL, :, :] = 0.0
    k[:, WALL, :] = 0.0
    d['reaction'] = dict(k=float(k_react), src=0, dst=1, types=1 << SOLVENT)
    d['membrane'] = membrane_defaults(kT)
    return d


def replica_ensemble(n_rep=512, seed=1004, rho=3.0, nv=500, diameter=5.0, kT=1.0,
                     max_rbc=4, side_lo=8, side_hi=16):
    """Independent replicas of uneven size: cubic periodic boxes of integer side
    in [side_lo, side_hi] at density rho, 0..max_rbc membranes (clamped to the
    non-overlapping slots of the box), permeability log-uniform in [0.01, 1],
    body force U[0, 0.1] along x. Returns a list of workload dicts."""
    rng = _rng(seed)
    verts, tri = biconcave_mesh(nv, diameter)
    thick = float(verts[:, 2].max() - verts[:, 2].min())
    reps = []
    for r in range(n_rep):
        L = float(rng.integers(side_lo, side_hi + 1))
        want = int(rng.integers(0, max_rbc + 1))
        perm = float(10.0 ** rng.uniform(-2.0, 0.0))
        fb = float(rng.uniform(0.0, 0.1))
        rseed = int(rng.integers(1, 2**62))
        d = _base('replica', (L, L, L), (1, 1, 1), 2, 1, rseed, rho, kT=kT, dt=MEMBRANE_DT)
        rr = _rng(rseed)
        d['particles'] = fluid_particles(rr, d['L'], rho, 1, kT)
        d['particles']['conc'][:] = 0.0
        sxy = int(L // (diameter + 1.0))
        sz = int(L // (thick + 1.0))
        slots = [(i, j, k) for k in range(sz) for j in range(sxy) for i in range(sxy)]
        nrbc = min(want, len(slots))
        for s in slots[:nrbc]:
            c = ((s[0] + 0.5) * L / sxy, (s[1] + 0.5) * L / sxy, (s[2] + 0.5) * L / sz)
            d['rbcs'].append(place_rbc(verts, tri, c, d['L'], rr, kT))
        d['kappa'][SOLVENT, MEMBRANE, 0] = d['kappa'][MEMBRANE, SOLVENT, 0] = perm
        d['body_force'] = np.asarray([fb, 0.0, 0.0], np.float32)
        d['membrane'] = membrane_defaults(kT)
        d['permeability'] = perm
        d['rbc_wanted'] = want
        reps.append(d)
    return reps


def n_particles(d) -> int:
    return int(d['particles']['pos'].shape[0]) + sum(int(r['pos'].shape[0]) for r in d['rbcs'])


def n_mobile(d) -> int:
    t = d['particles']['type']
    frozen = np.array([(d['frozen_types'] >> int(x)) & 1 for x in t], bool) if t.size else np.zeros(0, bool)
    return int((~frozen).sum()) + sum(int(r['pos'].shape[0]) for r in d['rbcs'])


def flat_state(d):
    """Concatenate free particles and membrane vertices in load order."""
    p = d['particles']
    pos = [p['pos']] + [r['pos'] for r in d['rbcs']]
    vel = [p['vel']] + [r['vel'] for r in d['rbcs']]
    conc = [p['conc']] + [r['conc'] for r in d['rbcs']]
    typ = [p['type']] + [np.full(r['pos'].shape[0], r['type'], np.int32) for r in d['rbcs']]
    body = [np.full(p['pos'].shape[0], -1, np.int32)] + [
        np.full(r['pos'].shape[0], b, np.int32) for b, r in enumerate(d['rbcs'])]
    return (np.concatenate(pos).astype(np.float32), np.concatenate(vel).astype(np.float32),
            np.concatenate(conc).astype(np.float32), np.concatenate(typ).astype(np.int32),
            np.concatenate(body).astype(np.int32))


def perturb(d, seed, dx=0.05, dv=0.0, rbc_scale=1.0):
    """Copy of a workload with membrane vertices displaced (uniform in
    [-dx, dx] per coordinate, then scaled about the cell centre) so that the
    membrane forces are away from their rest values; the rest geometry stays
    the original mesh."""
    import copy
    e = copy.deepcopy(d)
    rng = _rng(seed)
    L = e['L'].astype(np.float64)
    for r in e['rbcs']:
        v = r['pos'].astype(np.float64)
        if r['rest'] is None:
            r['rest'] = r['pos'].copy()
        ref = v[0]
        u = ref + (v - ref - L * np.round((v - ref) / L))
        c = u.mean(axis=0)
        u = c + rbc_scale * (u - c) + rng.uniform(-dx, dx, u.shape)
        u = u - np.floor(u / L) * L
        r['pos'] = np.minimum(u.astype(np.float32), np.nextafter(L.astype(np.float32), 0))
        if dv:
            r['vel'] = (r['vel'] + rng.normal(0, dv, r['vel'].shape)).astype(np.float32)
    return e
