/*
 * Plain FP64 CPU oracle for transport DPD with triangulated RBC membranes
 * (Blumers et al., arXiv:1611.06163, Sec. 2).
 *
 * TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the CPU
 * baseline of the benchmark call it; the CUDA library never does. It shares
 * no code with the CUDA path. Written for legibility, not speed: every
 * formula is the paper's equation written out in double precision.
 *
 * Readings of the paper taken here (the paper is silent or garbled):
 *  - w_C(r) = 1 - r/rc (Eq. 3 leaves w_C undefined; Groot-Warren form);
 *    w_R = (1 - r/rc)^(s_f/2), w_D = w_R^2 (Eq. 4).
 *  - r_ij = r_i - r_j, v_ij = v_i - v_j, e_ij = r_ij/|r_ij|; F_ij acts on i.
 *  - xi_ij from TEA (Sec. 3.1 names TEA on particle signatures) keyed on
 *    (min id, max id) with key (seed, step, stream); Box-Muller, cos branch.
 *  - Q^R (Eq. 7-8) is off unless qr_ms > 0 (Sec. 2.1 drops it since
 *    m_s << m): eps^2 = m_s^2 kappa rho (C~_i + C~_j), w_RC = w_DC^(1/2), one
 *    pair normal per species signed by the id order; Q^S is a first-order
 *    reaction A->B on the reacting types.
 *  - Integrator: Groot-Warren modified velocity Verlet with lambda (the paper
 *    cites GW for the DPD equations but names no scheme).
 *  - Bond random force (Eq. 13): F^R = sqrt(2kT/dt) [sqrt(2 gT) (Z^S - tr Z/3 I)
 *    + sqrt(3 gC - gT)/3 tr Z I] e_ij, Z a 3x3 matrix of standard normals per
 *    bond and step (the printed equation lacks the 1/dt and the "e_ij").
 *  - Bond potentials Eq. 10-11 with per-bond l_m = l0/x0 and k_p chosen so the
 *    bond is force-free at its rest length l0.
 *  - theta_j: angle between the outward normals of the two triangles on edge
 *    j, positive where the surface is convex.
 *  - Volume: sum of signed tetrahedra of each outward triangle with the origin
 *    of the membrane's unwrapped coordinates.
 *  - Area/volume constraints from the current positions, or (lagged) from the
 *    previous evaluation's totals (the concurrent variant of Sec. 3.3).
 *  - Walls: bounce-back at the planes z = wall_lo, wall_hi, or at a cylinder
 *    of radius cyl_R about the x axis through the box centre (the Dirichlet
 *    cylinder of Eq. 17, whose boundary concentration is held by frozen
 *    particles): position reflected, velocity reversed.
 *
 * Parity unpinned: the physical calibration of the membrane constants (the
 * RBC stretching data the paper fits is not available); the forces, fluxes,
 * integrator and reductions are pinned by the CPU tests (closed forms,
 * gradients of energies, conservation laws, published TEA vectors).
 */
#include "tdpd_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------ RNG */

void orc_tea(uint32_t v[2], const uint32_t k[4], int rounds)
{
    /* TEA: 64-bit block, 128-bit key, Feistel rounds with delta = 0x9E3779B9. */
    uint32_t y = v[0], z = v[1], sum = 0u;
    for (int r = 0; r < rounds; ++r) {
        sum += 0x9E3779B9u;
        y += ((z << 4) + k[0]) ^ (z + sum) ^ ((z >> 5) + k[1]);
        z += ((y << 4) + k[2]) ^ (y + sum) ^ ((y >> 5) + k[3]);
    }
    v[0] = y;
    v[1] = z;
}

void orc_uniform_pair(uint64_t seed, uint32_t i, uint32_t j, uint32_t step,
                      uint32_t stream, uint32_t bits[2], double u[2])
{
    uint32_t v[2];
    v[0] = i < j ? i : j;
    v[1] = i < j ? j : i;
    uint32_t k[4] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32), step, stream};
    orc_tea(v, k, ORC_TEA_ROUNDS);
    bits[0] = v[0];
    bits[1] = v[1];
    /* top 23 bits, centred in their bin: exactly representable in binary32 */
    u[0] = ((double)(v[0] >> 9) + 0.5) / 8388608.0;
    u[1] = ((double)(v[1] >> 9) + 0.5) / 8388608.0;
}

void orc_normal_pair(uint64_t seed, uint32_t i, uint32_t j, uint32_t step,
                     uint32_t stream, double g[2])
{
    uint32_t bits[2];
    double u[2];
    orc_uniform_pair(seed, i, j, step, stream, bits, u);
    double rad = sqrt(-2.0 * log(u[0]));
    g[0] = rad * cos(2.0 * M_PI * u[1]);
    g[1] = rad * sin(2.0 * M_PI * u[1]);
}

/* ----------------------------------------------------------- geometry */

static double min_image(double d, double L, int periodic)
{
    if (!periodic) return d;
    return d - L * floor(d / L + 0.5);
}

static int is_frozen(const orc_sys *s, int i)
{
    return (s->frozen_types >> s->type[i]) & 1u;
}

/* ------------------------------------------------------ pair (Eq. 3, 6) */

/* Contribution of particle j to particle i (force on i, flux into i). */
static void pair_term(const orc_sys *s, const double *pos, const double *vel,
                      const double *conc, uint32_t step, int i, int j,
                      double f[3], double *q)
{
    double d[3];
    for (int c = 0; c < 3; ++c)
        d[c] = min_image(pos[3 * i + c] - pos[3 * j + c], s->L[c], s->periodic[c]);
    double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    int ti = s->type[i], tj = s->type[j], T = s->ntypes;
    if (r <= 0.0) return;
    if (r < s->rcc) {
        double wdc = pow(1.0 - r / s->rcc, s->s_c);
        for (int k = 0; k < s->ns; ++k) {
            double kap = s->kappa[(ti * T + tj) * s->ns + k];
            q[k] += -kap * wdc * (conc[i * s->ns + k] - conc[j * s->ns + k]);
        }
        if (s->qr_ms > 0.0) {
            /* Eq. 7 with the strength of Eq. 8: eps^2 = m_s^2 kappa rho (C_i + C_j)
             * and w_RC = w_DC^(1/2). zeta_ij is one standard normal per species
             * (stream 6 + k/2, the (cos, sin) pair of one draw serving species k,
             * k+1), signed by the order of the ids so that zeta_ji = -zeta_ij and
             * the pair exchanges, rather than creates, solute. */
            double wrc = sqrt(wdc);
            double sgn = s->id[i] < s->id[j] ? 1.0 : -1.0;
            double g[2] = {0.0, 0.0};
            for (int k = 0; k < s->ns; ++k) {
                if ((k & 1) == 0) orc_normal_pair(s->seed, s->id[i], s->id[j], step, 6u + (uint32_t)(k / 2), g);
                double kap = s->kappa[(ti * T + tj) * s->ns + k];
                double csum = conc[i * s->ns + k] + conc[j * s->ns + k];
                double e2 = s->qr_ms * s->qr_ms * kap * s->qr_rho * csum;
                double eps = e2 > 0.0 ? sqrt(e2) : 0.0;
                q[k] += eps * wrc * sgn * g[k & 1] / sqrt(s->dt);
            }
        }
    }
    int excluded = s->exclude_same_body && s->body[i] >= 0 && s->body[i] == s->body[j];
    if (r < s->rc && !excluded) {
        double e[3] = {d[0] / r, d[1] / r, d[2] / r};
        double w = 1.0 - r / s->rc;
        double wR = pow(w, 0.5 * s->s_f);
        double wD = wR * wR;
        double ev = 0.0;
        for (int c = 0; c < 3; ++c) ev += e[c] * (vel[3 * i + c] - vel[3 * j + c]);
        double g[2];
        orc_normal_pair(s->seed, s->id[i], s->id[j], step, 0u, g);
        double fc = s->a[ti * T + tj] * w;
        double fd = -s->gamma[ti * T + tj] * wD * ev;
        double fr = s->sigma[ti * T + tj] * wR * g[0] / sqrt(s->dt);
        for (int c = 0; c < 3; ++c) f[c] += (fc + fd + fr) * e[c];
    }
}

static void add_sources(const orc_sys *s, const double *pos, const double *conc, double *F, double *Q)
{
    for (int i = 0; i < s->n; ++i) {
        const double sg = (s->fbody_flip && pos[3 * i + 2] >= 0.5 * s->L[2]) ? -1.0 : 1.0;
        if (!is_frozen(s, i))
            for (int c = 0; c < 3; ++c) F[3 * i + c] += sg * s->fbody[c];
        if (s->k_react != 0.0 && ((s->react_types >> s->type[i]) & 1u)) {
            double rate = s->k_react * conc[i * s->ns + s->r_src];
            Q[i * s->ns + s->r_src] -= rate;
            Q[i * s->ns + s->r_dst] += rate;
        }
    }
}

static int cell_coord(double x, double L, int nc)
{
    int c = (int)floor(x / L * nc);
    if (c < 0) c = 0;
    if (c >= nc) c = nc - 1;
    return c;
}

int orc_pair_forces(const orc_sys *s, const double *pos, const double *vel,
                    const double *conc, uint32_t step, int mode, double *F, double *Q)
{
    const int n = s->n, ns = s->ns;
    memset(F, 0, sizeof(double) * 3 * (size_t)n);
    memset(Q, 0, sizeof(double) * (size_t)ns * (size_t)n);
    if (mode == 0) {
        /* every unordered pair once; Newton's third law for the partner */
        double *q = (double *)calloc((size_t)ns, sizeof(double));
        for (int i = 0; i < n; ++i) {
            for (int j = i + 1; j < n; ++j) {
                double f[3] = {0, 0, 0};
                for (int k = 0; k < ns; ++k) q[k] = 0.0;
                pair_term(s, pos, vel, conc, step, i, j, f, q);
                for (int c = 0; c < 3; ++c) {
                    F[3 * i + c] += f[c];
                    F[3 * j + c] -= f[c];
                }
                for (int k = 0; k < ns; ++k) {
                    Q[i * ns + k] += q[k];
                    Q[j * ns + k] -= q[k];
                }
            }
        }
        free(q);
    } else {
        /* cell list of edge >= max(rc, rcc); each particle sums its own
         * partners, so every pair is evaluated from both sides */
        double rcut = s->rc > s->rcc ? s->rc : s->rcc;
        int nc[3];
        for (int c = 0; c < 3; ++c) {
            nc[c] = (int)floor(s->L[c] / rcut);
            if (nc[c] < 3) return -1;
        }
        int ncell = nc[0] * nc[1] * nc[2];
        int *head = (int *)malloc(sizeof(int) * (size_t)ncell);
        int *next = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
        for (int c = 0; c < ncell; ++c) head[c] = -1;
        for (int i = n - 1; i >= 0; --i) {
            int cx = cell_coord(pos[3 * i], s->L[0], nc[0]);
            int cy = cell_coord(pos[3 * i + 1], s->L[1], nc[1]);
            int cz = cell_coord(pos[3 * i + 2], s->L[2], nc[2]);
            int c = (cz * nc[1] + cy) * nc[0] + cx;
            next[i] = head[c];
            head[c] = i;
        }
#pragma omp parallel for schedule(dynamic, 64)
        for (int i = 0; i < n; ++i) {
            double f[3] = {0, 0, 0};
            double qv[64];
            double *q = ns <= 64 ? qv : (double *)malloc(sizeof(double) * (size_t)ns);
            for (int k = 0; k < ns; ++k) q[k] = 0.0;
            int ci[3];
            for (int c = 0; c < 3; ++c) ci[c] = cell_coord(pos[3 * i + c], s->L[c], nc[c]);
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        int cc[3] = {ci[0] + dx, ci[1] + dy, ci[2] + dz};
                        int skip = 0;
                        for (int c = 0; c < 3; ++c) {
                            if (cc[c] < 0 || cc[c] >= nc[c]) {
                                if (!s->periodic[c]) skip = 1;
                                cc[c] = (cc[c] + nc[c]) % nc[c];
                            }
                        }
                        if (skip) continue;
                        int cell = (cc[2] * nc[1] + cc[1]) * nc[0] + cc[0];
                        for (int j = head[cell]; j >= 0; j = next[j])
                            if (j != i) pair_term(s, pos, vel, conc, step, i, j, f, q);
                    }
            for (int c = 0; c < 3; ++c) F[3 * i + c] = f[c];
            for (int k = 0; k < ns; ++k) Q[i * ns + k] = q[k];
            if (q != qv) free(q);
        }
        free(head);
        free(next);
    }
    add_sources(s, pos, conc, F, Q);
    return 0;
}

/* ------------------------------------------------------------ membrane */

struct orc_mem {
    int nrbc, nv, ntri, ne;
    int *tri;          /* [ntri*3] */
    int *edge;         /* [ne*2], edge[0] < edge[1] */
    int *dih;          /* [ne*4]: a, b, c, d with triangles (a,b,c), (b,a,d) */
    int *first;        /* [nrbc] */
    double *A0j, *l0, *A0, *V0;
    double L[3];
    int periodic[3];
    double kT, p, x0, m, kg, kl, kv, kb, theta0, gT, gC, v_ratio;
    /* Sec. 3.3 concurrent variant: the area and volume constraints of a force
     * evaluation use the totals of the previous evaluation. lag[2b], lag[2b+1]
     * hold them; lag[2 nrbc] != 0 once they are set. */
    int lagged;
    double *lag;
};

static void cross3(const double a[3], const double b[3], double c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

static double dot3(const double a[3], const double b[3])
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

static double norm3(const double a[3]) { return sqrt(dot3(a, a)); }

/* Unwrap membrane b: start at vertex 0 and walk the edges, placing each new
 * vertex at the minimum image of its already placed neighbour. */
static void unwrap(const orc_mem *m, const double *pos, int b, double *x)
{
    int nv = m->nv;
    char *done = (char *)calloc((size_t)nv, 1);
    const double *p = pos + 3 * (size_t)m->first[b];
    for (int c = 0; c < 3; ++c) x[c] = p[c];
    done[0] = 1;
    int placed = 1, changed = 1;
    while (placed < nv && changed) {
        changed = 0;
        for (int e = 0; e < m->ne; ++e) {
            int i = m->edge[2 * e], j = m->edge[2 * e + 1];
            if (done[i] == done[j]) continue;
            int from = done[i] ? i : j, to = done[i] ? j : i;
            for (int c = 0; c < 3; ++c)
                x[3 * to + c] = x[3 * from + c] +
                    min_image(p[3 * to + c] - p[3 * from + c], m->L[c], m->periodic[c]);
            done[to] = 1;
            ++placed;
            changed = 1;
        }
    }
    free(done);
}

static void tri_area_vol(const double *x, const int *t, double *A, double *V, double n[3])
{
    const double *x1 = x + 3 * t[0], *x2 = x + 3 * t[1], *x3 = x + 3 * t[2];
    double a[3], b[3], c23[3];
    for (int c = 0; c < 3; ++c) {
        a[c] = x2[c] - x1[c];
        b[c] = x3[c] - x1[c];
    }
    cross3(a, b, n);
    *A = 0.5 * norm3(n);
    cross3(x2, x3, c23);
    *V = dot3(x1, c23) / 6.0;
}

orc_mem *orc_mem_create(int nrbc, int nv, int ntri, const int *tri, const int *first,
                        const double *rest, const double L[3], const int periodic[3],
                        const double P[13])
{
    orc_mem *m = (orc_mem *)calloc(1, sizeof(orc_mem));
    m->lagged = P[12] != 0.0;
    m->lag = (double *)calloc(2 * (size_t)nrbc + 1, sizeof(double));
    m->nrbc = nrbc;
    m->nv = nv;
    m->ntri = ntri;
    m->tri = (int *)malloc(sizeof(int) * 3 * (size_t)ntri);
    memcpy(m->tri, tri, sizeof(int) * 3 * (size_t)ntri);
    m->first = (int *)malloc(sizeof(int) * (size_t)(nrbc > 0 ? nrbc : 1));
    memcpy(m->first, first, sizeof(int) * (size_t)nrbc);
    for (int c = 0; c < 3; ++c) {
        m->L[c] = L[c];
        m->periodic[c] = periodic[c];
    }
    m->kT = P[0]; m->p = P[1]; m->x0 = P[2]; m->m = P[3];
    m->kg = P[4]; m->kl = P[5]; m->kv = P[6]; m->kb = P[7];
    m->theta0 = P[8]; m->gT = P[9]; m->gC = P[10]; m->v_ratio = P[11];

    /* edges and their dihedral quadruples from the directed triangle edges */
    m->ne = 3 * ntri / 2;
    m->edge = (int *)malloc(sizeof(int) * 2 * (size_t)m->ne);
    m->dih = (int *)malloc(sizeof(int) * 4 * (size_t)m->ne);
    int ne = 0;
    for (int t = 0; t < ntri; ++t) {
        for (int k = 0; k < 3; ++k) {
            int a = tri[3 * t + k], b = tri[3 * t + (k + 1) % 3], c = tri[3 * t + (k + 2) % 3];
            if (a > b) continue;   /* register each edge from the triangle holding a->b */
            /* find the triangle holding the reverse directed edge b->a */
            int d = -1;
            for (int u = 0; u < ntri && d < 0; ++u)
                for (int kk = 0; kk < 3; ++kk)
                    if (tri[3 * u + kk] == b && tri[3 * u + (kk + 1) % 3] == a)
                        d = tri[3 * u + (kk + 2) % 3];
            if (ne < m->ne) {
                m->edge[2 * ne] = a;
                m->edge[2 * ne + 1] = b;
                m->dih[4 * ne] = a;
                m->dih[4 * ne + 1] = b;
                m->dih[4 * ne + 2] = c;
                m->dih[4 * ne + 3] = d;
            }
            ++ne;
        }
    }
    if (ne != m->ne) {
        orc_mem_destroy(m);
        return NULL;
    }

    /* rest state */
    m->A0j = (double *)malloc(sizeof(double) * (size_t)nrbc * (size_t)ntri);
    m->l0 = (double *)malloc(sizeof(double) * (size_t)nrbc * (size_t)m->ne);
    m->A0 = (double *)malloc(sizeof(double) * (size_t)(nrbc > 0 ? nrbc : 1));
    m->V0 = (double *)malloc(sizeof(double) * (size_t)(nrbc > 0 ? nrbc : 1));
    double *x = (double *)malloc(sizeof(double) * 3 * (size_t)nv);
    /* rest positions are given per membrane; unwrap them like live ones */
    double *restpos = (double *)malloc(sizeof(double) * 3 * (size_t)nv);
    for (int b = 0; b < nrbc; ++b) {
        memcpy(restpos, rest + 3 * (size_t)nv * b, sizeof(double) * 3 * (size_t)nv);
        int save = m->first[b];
        m->first[b] = 0;
        unwrap(m, restpos, b, x);
        m->first[b] = save;
        double A = 0.0, V = 0.0;
        for (int t = 0; t < ntri; ++t) {
            double At, Vt, n[3];
            tri_area_vol(x, m->tri + 3 * t, &At, &Vt, n);
            m->A0j[(size_t)b * ntri + t] = At;
            A += At;
            V += Vt;
        }
        for (int e = 0; e < m->ne; ++e) {
            double d[3];
            for (int c = 0; c < 3; ++c)
                d[c] = x[3 * m->edge[2 * e] + c] - x[3 * m->edge[2 * e + 1] + c];
            m->l0[(size_t)b * m->ne + e] = norm3(d);
        }
        m->A0[b] = A;
        m->V0[b] = m->v_ratio > 0.0 ? m->v_ratio * pow(A, 1.5) : V;
    }
    free(restpos);
    free(x);
    return m;
}

void orc_mem_destroy(orc_mem *m)
{
    if (!m) return;
    free(m->tri); free(m->edge); free(m->dih); free(m->first);
    free(m->A0j); free(m->l0); free(m->A0); free(m->V0); free(m->lag);
    free(m);
}

int orc_mem_nedges(const orc_mem *m) { return m->ne; }

void orc_mem_reset_lag(orc_mem *m)
{
    if (m) m->lag[2 * (size_t)m->nrbc] = 0.0;
}

void orc_mem_rest(const orc_mem *m, double *A0j, double *l0, double *A0, double *V0)
{
    memcpy(A0j, m->A0j, sizeof(double) * (size_t)m->nrbc * (size_t)m->ntri);
    memcpy(l0, m->l0, sizeof(double) * (size_t)m->nrbc * (size_t)m->ne);
    memcpy(A0, m->A0, sizeof(double) * (size_t)m->nrbc);
    memcpy(V0, m->V0, sizeof(double) * (size_t)m->nrbc);
}

/* WLC (Eq. 10) + POW (Eq. 11) bond with l_m = l0/x0 and k_p making dU/dl(l0) = 0. */
static void bond_params(const orc_mem *m, double l0, double *lm, double *kp)
{
    double x0 = m->x0;
    double fwlc = m->kT / m->p * (0.25 / ((1.0 - x0) * (1.0 - x0)) - 0.25 + x0);
    *lm = l0 / x0;
    *kp = fwlc * pow(l0, m->m);
}

static double bond_energy(const orc_mem *m, double l, double l0)
{
    double lm, kp;
    bond_params(m, l0, &lm, &kp);
    double x = l / lm;
    double u = m->kT * lm / (4.0 * m->p) * x * x * (3.0 - 2.0 * x) / (1.0 - x);
    if (m->m == 1.0) u += -kp * log(l);
    else u += kp / ((m->m - 1.0) * pow(l, m->m - 1.0));
    return u;
}

/* dU/dl of bond_energy */
static double bond_dudl(const orc_mem *m, double l, double l0)
{
    double lm, kp;
    bond_params(m, l0, &lm, &kp);
    double x = l / lm;
    double fw = m->kT / m->p * (0.25 / ((1.0 - x) * (1.0 - x)) - 0.25 + x);
    return fw - kp / pow(l, m->m);
}

/* theta of dihedral (a,b,c,d) and its gradient w.r.t. the four vertices. */
static double dihedral(const double *xa, const double *xb, const double *xc, const double *xd,
                       double g[4][3])
{
    double e[3], ac[3], bd[3], ba[3], n1[3], n2[3];
    for (int k = 0; k < 3; ++k) {
        e[k] = xb[k] - xa[k];
        ac[k] = xc[k] - xa[k];
        bd[k] = xd[k] - xb[k];
        ba[k] = xa[k] - xb[k];
    }
    cross3(e, ac, n1);        /* normal of (a, b, c) */
    cross3(ba, bd, n2);       /* normal of (b, a, d) */
    double le = norm3(e), n1s = dot3(n1, n1), n2s = dot3(n2, n2);
    double n1n = sqrt(n1s), n2n = sqrt(n2s);
    double c12[3];
    cross3(n1, n2, c12);
    double sinv = dot3(c12, e) / (le * n1n * n2n);
    double cosv = dot3(n1, n2) / (n1n * n2n);
    double theta = atan2(sinv, cosv);
    if (g) {
        double ca = 0, cb = 0, da = 0, db = 0;   /* projections on the edge */
        for (int k = 0; k < 3; ++k) {
            ca += (xc[k] - xa[k]) * e[k];
            cb += (xc[k] - xb[k]) * e[k];
            da += (xd[k] - xa[k]) * e[k];
            db += (xd[k] - xb[k]) * e[k];
        }
        for (int k = 0; k < 3; ++k) {
            g[2][k] = -le * n1[k] / n1s;
            g[3][k] = -le * n2[k] / n2s;
            g[1][k] = (ca / le) * n1[k] / n1s + (da / le) * n2[k] / n2s;
            g[0][k] = -(cb / le) * n1[k] / n1s - (db / le) * n2[k] / n2s;
        }
    }
    return theta;
}

void orc_mem_angles(const orc_mem *m, const double *pos, int b, double *theta)
{
    double *x = (double *)malloc(sizeof(double) * 3 * (size_t)m->nv);
    unwrap(m, pos, b, x);
    for (int e = 0; e < m->ne; ++e) {
        const int *q = m->dih + 4 * e;
        theta[e] = dihedral(x + 3 * q[0], x + 3 * q[1], x + 3 * q[2], x + 3 * q[3], NULL);
    }
    free(x);
}

double orc_mem_energy(const orc_mem *m, const double *pos, int parts)
{
    double E = 0.0;
    double *x = (double *)malloc(sizeof(double) * 3 * (size_t)m->nv);
    for (int b = 0; b < m->nrbc; ++b) {
        unwrap(m, pos, b, x);
        if (parts & 1) {
            for (int e = 0; e < m->ne; ++e) {
                double d[3];
                for (int c = 0; c < 3; ++c)
                    d[c] = x[3 * m->edge[2 * e] + c] - x[3 * m->edge[2 * e + 1] + c];
                E += bond_energy(m, norm3(d), m->l0[(size_t)b * m->ne + e]);
            }
        }
        if (parts & 4) {
            double A = 0.0, V = 0.0;
            for (int t = 0; t < m->ntri; ++t) {
                double At, Vt, n[3];
                tri_area_vol(x, m->tri + 3 * t, &At, &Vt, n);
                double a0 = m->A0j[(size_t)b * m->ntri + t];
                E += m->kl * (At - a0) * (At - a0) / (2.0 * a0);
                A += At;
                V += Vt;
            }
            E += m->kg * (A - m->A0[b]) * (A - m->A0[b]) / (2.0 * m->A0[b]);
            E += m->kv * (V - m->V0[b]) * (V - m->V0[b]) / (2.0 * m->V0[b]);
        }
        if (parts & 8) {
            for (int e = 0; e < m->ne; ++e) {
                const int *q = m->dih + 4 * e;
                double th = dihedral(x + 3 * q[0], x + 3 * q[1], x + 3 * q[2], x + 3 * q[3], NULL);
                E += m->kb * (1.0 - cos(th - m->theta0));
            }
        }
    }
    free(x);
    return E;
}

void orc_mem_forces(const orc_mem *m, const double *pos, const double *vel,
                    const uint32_t *id, uint64_t seed, uint32_t step, double dt,
                    int parts, double *F, double *AV)
{
    orc_mem_forces_av(m, pos, vel, id, seed, step, dt, parts, F, AV, NULL);
}

void orc_mem_forces_av(const orc_mem *m, const double *pos, const double *vel,
                       const uint32_t *id, uint64_t seed, uint32_t step, double dt,
                       int parts, double *F, double *AV, const double *av_use)
{
    double *x = (double *)malloc(sizeof(double) * 3 * (size_t)m->nv);
    double *f = (double *)malloc(sizeof(double) * 3 * (size_t)m->nv);
    for (int b = 0; b < m->nrbc; ++b) {
        const int base = m->first[b];
        unwrap(m, pos, b, x);
        memset(f, 0, sizeof(double) * 3 * (size_t)m->nv);

        double A = 0.0, V = 0.0;
        for (int t = 0; t < m->ntri; ++t) {
            double At, Vt, n[3];
            tri_area_vol(x, m->tri + 3 * t, &At, &Vt, n);
            A += At;
            V += Vt;
        }
        if (AV) {
            AV[2 * b] = A;
            AV[2 * b + 1] = V;
        }

        if (parts & 4) {
            /* Eq. 14-15: -dE/dx_k with dA_j/dx_k = n_hat x (x_{k+2} - x_{k+1}) / 2
             * and dV_j/dx_k = (x_{k+1} x x_{k+2}) / 6, (k, k+1, k+2) cyclic */
            const double Au = av_use ? av_use[2 * b] : A, Vu = av_use ? av_use[2 * b + 1] : V;
            double cg = m->kg * (Au - m->A0[b]) / m->A0[b];
            double cv = m->kv * (Vu - m->V0[b]) / m->V0[b];
            for (int t = 0; t < m->ntri; ++t) {
                const int *tv = m->tri + 3 * t;
                double At, Vt, n[3];
                tri_area_vol(x, tv, &At, &Vt, n);
                double a0 = m->A0j[(size_t)b * m->ntri + t];
                double ca = cg + m->kl * (At - a0) / a0;
                double nh[3] = {n[0] / (2.0 * At), n[1] / (2.0 * At), n[2] / (2.0 * At)};
                for (int k = 0; k < 3; ++k) {
                    const double *x1 = x + 3 * tv[(k + 1) % 3], *x2 = x + 3 * tv[(k + 2) % 3];
                    double d[3], gA[3], gV[3];
                    for (int c = 0; c < 3; ++c) d[c] = x2[c] - x1[c];
                    cross3(nh, d, gA);
                    cross3(x1, x2, gV);
                    for (int c = 0; c < 3; ++c)
                        f[3 * tv[k] + c] -= ca * 0.5 * gA[c] + cv * gV[c] / 6.0;
                }
            }
        }

        if (parts & 3) {
            for (int e = 0; e < m->ne; ++e) {
                int i = m->edge[2 * e], j = m->edge[2 * e + 1];
                double d[3];
                for (int c = 0; c < 3; ++c) d[c] = x[3 * i + c] - x[3 * j + c];
                double l = norm3(d);
                double ev[3] = {d[0] / l, d[1] / l, d[2] / l};
                double fij[3] = {0, 0, 0};
                if (parts & 1) {
                    double du = bond_dudl(m, l, m->l0[(size_t)b * m->ne + e]);
                    for (int c = 0; c < 3; ++c) fij[c] += -du * ev[c];
                }
                if (parts & 2) {
                    /* Eq. 12 with v_ij = v_i - v_j */
                    double vij[3];
                    for (int c = 0; c < 3; ++c)
                        vij[c] = vel[3 * (base + i) + c] - vel[3 * (base + j) + c];
                    double ve = dot3(vij, ev);
                    for (int c = 0; c < 3; ++c) fij[c] += -m->gT * vij[c] - m->gC * ve * ev[c];
                    /* Eq. 13: 3x3 Wiener matrix from streams 1..5 */
                    double z[10];
                    for (int s = 0; s < 5; ++s)
                        orc_normal_pair(seed, id[base + i], id[base + j], step, (uint32_t)(s + 1), z + 2 * s);
                    double W[3][3], tr = z[0] + z[4] + z[8];
                    for (int r = 0; r < 3; ++r)
                        for (int c = 0; c < 3; ++c)
                            W[r][c] = 0.5 * (z[3 * r + c] + z[3 * c + r]);
                    for (int r = 0; r < 3; ++r) W[r][r] -= tr / 3.0;
                    double aT = sqrt(2.0 * m->gT), bC = sqrt(3.0 * m->gC - m->gT) / 3.0;
                    double s0 = sqrt(2.0 * m->kT / dt);
                    for (int r = 0; r < 3; ++r) {
                        double acc = 0.0;
                        for (int c = 0; c < 3; ++c) acc += aT * W[r][c] * ev[c];
                        acc += bC * tr * ev[r];
                        fij[r] += s0 * acc;
                    }
                }
                for (int c = 0; c < 3; ++c) {
                    f[3 * i + c] += fij[c];
                    f[3 * j + c] -= fij[c];
                }
            }
        }

        if (parts & 8) {
            /* Eq. 16: -k_b sin(theta - theta0) grad theta */
            for (int e = 0; e < m->ne; ++e) {
                const int *q = m->dih + 4 * e;
                double g[4][3];
                double th = dihedral(x + 3 * q[0], x + 3 * q[1], x + 3 * q[2], x + 3 * q[3], g);
                double s = m->kb * sin(th - m->theta0);
                for (int r = 0; r < 4; ++r)
                    for (int c = 0; c < 3; ++c) f[3 * q[r] + c] -= s * g[r][c];
            }
        }

        for (int v = 0; v < m->nv; ++v)
            for (int c = 0; c < 3; ++c) F[3 * (size_t)(base + v) + c] += f[3 * v + c];
    }
    free(x);
    free(f);
}

/* ------------------------------------------------------- full force */

int orc_forces(const orc_sys *s, const orc_mem *m, const double *pos, const double *vel,
               const double *conc, uint32_t step, int mode, double *F, double *Q)
{
    int rc = orc_pair_forces(s, pos, vel, conc, step, mode, F, Q);
    if (rc) return rc;
    if (m) {
        /* lagged: the previous evaluation's totals once there is one; either
         * way this evaluation's totals become the next one's */
        const int use = m->lagged && m->lag[2 * (size_t)m->nrbc] != 0.0;
        double *av = (double *)malloc(sizeof(double) * (2 * (size_t)m->nrbc + 1));
        orc_mem_forces_av(m, pos, vel, s->id, s->seed, step, s->dt, 15, F, av, use ? m->lag : NULL);
        if (m->lagged) {
            memcpy(m->lag, av, sizeof(double) * 2 * (size_t)m->nrbc);
            m->lag[2 * (size_t)m->nrbc] = 1.0;
        }
        free(av);
    }
    return 0;
}

/* ---------------------------------------------------------- integrator */

int orc_run(const orc_sys *s, const orc_mem *m, double *pos, double *vel, double *conc,
            double *F, double *Q, uint32_t step0, int nsteps, int mode)
{
    const int n = s->n, ns = s->ns;
    const double dt = s->dt, lam = s->lambda;
    double *rn = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    double *vt = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    double *ct = (double *)malloc(sizeof(double) * (size_t)ns * (size_t)(n > 0 ? n : 1));
    double *F2 = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    double *Q2 = (double *)malloc(sizeof(double) * (size_t)ns * (size_t)(n > 0 ? n : 1));
    int rc = 0;
    for (int it = 0; it < nsteps && rc == 0; ++it) {
        for (int i = 0; i < n; ++i) {
            if (is_frozen(s, i)) {
                for (int c = 0; c < 3; ++c) {
                    rn[3 * i + c] = pos[3 * i + c];
                    vt[3 * i + c] = vel[3 * i + c];
                }
                for (int k = 0; k < ns; ++k) ct[i * ns + k] = conc[i * ns + k];
                continue;
            }
            int flip = 0;
            for (int c = 0; c < 3; ++c) {
                double x = pos[3 * i + c] + dt * vel[3 * i + c] + 0.5 * dt * dt * F[3 * i + c];
                if (s->periodic[c]) {
                    if (x < 0.0) x += s->L[c];
                    else if (x >= s->L[c]) x -= s->L[c];
                } else if (c == 2) {
                    /* bounce-back at the wall planes: reflect, reverse velocity */
                    if (x < s->wall_lo) { x = 2.0 * s->wall_lo - x; flip = 1; }
                    else if (x > s->wall_hi) { x = 2.0 * s->wall_hi - x; flip = 1; }
                }
                rn[3 * i + c] = x;
            }
            if (s->cyl_R > 0.0) {
                /* bounce-back at the cylinder: distance d > R from the axis
                 * becomes 2R - d along the same radial line */
                const double cy = 0.5 * s->L[1], cz = 0.5 * s->L[2];
                const double dy = rn[3 * i + 1] - cy, dz = rn[3 * i + 2] - cz;
                const double d = sqrt(dy * dy + dz * dz);
                if (d > s->cyl_R) {
                    const double f = (2.0 * s->cyl_R - d) / d;
                    rn[3 * i + 1] = cy + dy * f;
                    rn[3 * i + 2] = cz + dz * f;
                    flip = 1;
                }
            }
            if (flip)
                for (int c = 0; c < 3; ++c) vel[3 * i + c] = -vel[3 * i + c];
            for (int c = 0; c < 3; ++c) vt[3 * i + c] = vel[3 * i + c] + lam * dt * F[3 * i + c];
            for (int k = 0; k < ns; ++k) ct[i * ns + k] = conc[i * ns + k] + lam * dt * Q[i * ns + k];
        }
        rc = orc_forces(s, m, rn, vt, ct, step0 + (uint32_t)it + 1u, mode, F2, Q2);
        for (int i = 0; i < n; ++i) {
            for (int c = 0; c < 3; ++c) pos[3 * i + c] = rn[3 * i + c];
            if (is_frozen(s, i)) continue;
            for (int c = 0; c < 3; ++c)
                vel[3 * i + c] += 0.5 * dt * (F[3 * i + c] + F2[3 * i + c]);
            for (int k = 0; k < ns; ++k)
                conc[i * ns + k] += 0.5 * dt * (Q[i * ns + k] + Q2[i * ns + k]);
        }
        memcpy(F, F2, sizeof(double) * 3 * (size_t)n);
        memcpy(Q, Q2, sizeof(double) * (size_t)ns * (size_t)n);
    }
    free(rn); free(vt); free(ct); free(F2); free(Q2);
    return rc;
}

void orc_observables(const orc_sys *s, const double *vel, const double *conc, double *out)
{
    const int n = s->n, ns = s->ns;
    double p[3] = {0, 0, 0};
    int nm = 0;
    for (int i = 0; i < n; ++i) {
        if (is_frozen(s, i)) continue;
        ++nm;
        for (int c = 0; c < 3; ++c) p[c] += vel[3 * i + c];
    }
    double vbar[3] = {0, 0, 0};
    if (nm > 0)
        for (int c = 0; c < 3; ++c) vbar[c] = p[c] / nm;
    double ke = 0.0;
    for (int i = 0; i < n; ++i) {
        if (is_frozen(s, i)) continue;
        for (int c = 0; c < 3; ++c) {
            double d = vel[3 * i + c] - vbar[c];
            ke += d * d;
        }
    }
    out[0] = nm > 1 ? ke / (3.0 * (nm - 1)) : 0.0;
    for (int c = 0; c < 3; ++c) out[1 + c] = p[c];
    for (int k = 0; k < ns; ++k) {
        double t = 0.0;
        for (int i = 0; i < n; ++i) t += conc[i * ns + k];
        out[4 + k] = t;
    }
    out[4 + ns] = nm;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
