/*
 * Plain FP64 CPU oracle for one step of transport DPD (tDPD) with
 * triangulated red-blood-cell membranes (Blumers et al., arXiv:1611.06163).
 *
 * TEST INFRASTRUCTURE ONLY. This library is the reference the CUDA path is
 * checked against; it is built and called only by the test suite, the smoke
 * check and the CPU-baseline leg of the benchmark. It shares no code, header,
 * table or constant with the CUDA library, and the CUDA library never calls it.
 *
 * Every array is caller-owned, row-major, FP64 unless stated. Particles are
 * indexed 0..n-1 in load order; pos/vel are [n*3], conc/flux are [n*ns].
 */
#ifndef TDPD_ORACLE_H
#define TDPD_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Number of TEA rounds used for the pairwise random numbers. */
#define ORC_TEA_ROUNDS 8

typedef struct {
    int n, ns, ntypes;
    double L[3];
    int periodic[3];
    double wall_lo, wall_hi;      /* bounce-back planes along z if !periodic[2] */
    const double *a, *gamma, *sigma;  /* [ntypes*ntypes] Eq. 3 coefficients */
    double rc, s_f;               /* force cutoff; w_R = (1-r/rc)^(s_f/2) */
    const double *kappa;          /* [ntypes*ntypes*ns] Eq. 6 strengths */
    double rcc, s_c;              /* flux cutoff; w_DC = (1-r/rcc)^s_c */
    uint64_t seed;
    int exclude_same_body;        /* no Eq. 3 forces inside one membrane */
    double dt, lambda;
    double fbody[3];
    uint32_t frozen_types;        /* bit t set: type t is not integrated */
    double k_react; int r_src, r_dst; uint32_t react_types;  /* A->B, rate k */
    const int *type, *body;       /* [n]; body -1 for free particles */
    const uint32_t *id;           /* [n] persistent ids keying the RNG */
    double qr_ms, qr_rho;         /* random flux (Eq. 7-8): solute mass m_s and
                                   * density rho in eps^2 = m_s^2 kappa rho (C_i + C_j);
                                   * m_s = 0: no random flux */
    int fbody_flip;               /* 1: the body force is -fbody where z >= L_z/2
                                   * (the double Poiseuille flow of Sec. 4.1) */
    double cyl_R;                 /* > 0: mobile particles stay within this distance of
                                   * the axis y = L_y/2, z = L_z/2 (reflected radially,
                                   * velocity reversed; the cylinder of Eq. 17) */
} orc_sys;

typedef struct orc_mem orc_mem;

/* TEA block cipher (Wheeler & Needham 1994) with a given round count. */
void orc_tea(uint32_t v[2], const uint32_t k[4], int rounds);
/* Two standard normals (cos, sin branch of Box-Muller) keyed on the unordered
 * pair {i, j}, the step and a stream number. */
void orc_normal_pair(uint64_t seed, uint32_t i, uint32_t j, uint32_t step,
                     uint32_t stream, double g[2]);
/* The two 24-bit-exact uniforms behind orc_normal_pair. */
void orc_uniform_pair(uint64_t seed, uint32_t i, uint32_t j, uint32_t step,
                      uint32_t stream, uint32_t bits[2], double u[2]);

/* Pairwise tDPD force (Eq. 3) and Fickian flux (Eq. 6), plus the random flux
 * of Eq. 7 when qr_ms > 0, at state (pos, vel, conc)
 * and step number `step`. mode 0: all pairs O(n^2); mode 1: cell list with
 * OpenMP. Overwrites F [n*3] and Q [n*ns]. Adds body force to non-frozen
 * particles and the first-order reaction source to Q. */
int orc_pair_forces(const orc_sys *s, const double *pos, const double *vel,
                    const double *conc, uint32_t step, int mode,
                    double *F, double *Q);

/* Membrane model. nrbc membranes of one topology (nv vertices, ntri
 * outward triangles); membrane b occupies particles first[b]..first[b]+nv-1.
 * rest [nrbc*nv*3] fixes l0 per bond, A0 per triangle, A0 = sum and
 * V0 = v_ratio * A0^1.5 (v_ratio <= 0: V0 = rest volume). params: kT, p, x0,
 * m, kg, kl, kv, kb, theta0, gammaT, gammaC, v_ratio, lagged (nonzero: the
 * area and volume constraints of orc_forces use the totals of the previous
 * orc_forces call, Sec. 3.3). */
orc_mem *orc_mem_create(int nrbc, int nv, int ntri, const int *tri, const int *first,
                        const double *rest, const double L[3], const int periodic[3],
                        const double params[13]);
void orc_mem_destroy(orc_mem *m);
int orc_mem_nedges(const orc_mem *m);
/* Rest quantities: A0j [nrbc*ntri], l0 [nrbc*ne], A0/V0 [nrbc]. */
void orc_mem_rest(const orc_mem *m, double *A0j, double *l0, double *A0, double *V0);
/* parts bit 1: WLC+POW bonds (Eq. 10-11); 2: bond viscous + random (Eq. 12-13);
 * 4: area + volume (Eq. 14-15); 8: bending (Eq. 16). Adds into F. AV [nrbc*2]
 * receives (A, V) of each membrane (may be NULL). */
/* Forget the totals a lagged membrane model carries (a new state follows). */
void orc_mem_reset_lag(orc_mem *m);
void orc_mem_forces(const orc_mem *m, const double *pos, const double *vel,
                    const uint32_t *id, uint64_t seed, uint32_t step, double dt,
                    int parts, double *F, double *AV);
/* The same with the area and volume constraints evaluated at the totals
 * av_use [nrbc*2] (NULL: this configuration's own). */
void orc_mem_forces_av(const orc_mem *m, const double *pos, const double *vel,
                       const uint32_t *id, uint64_t seed, uint32_t step, double dt,
                       int parts, double *F, double *AV, const double *av_use);
/* Conservative membrane energy of the selected parts (1, 4, 8). */
double orc_mem_energy(const orc_mem *m, const double *pos, int parts);
/* Bending angles theta_j of membrane b, per edge [ne]. */
void orc_mem_angles(const orc_mem *m, const double *pos, int b, double *theta);

/* Total force: pair + membrane (m may be NULL). */
int orc_forces(const orc_sys *s, const orc_mem *m, const double *pos, const double *vel,
               const double *conc, uint32_t step, int mode, double *F, double *Q);

/* Groot-Warren modified velocity Verlet (lambda), nsteps steps starting at
 * step number `step0` (F, Q must hold the forces at step0). Updates pos, vel,
 * conc, F, Q in place. */
int orc_run(const orc_sys *s, const orc_mem *m, double *pos, double *vel, double *conc,
            double *F, double *Q, uint32_t step0, int nsteps, int mode);

/* Observables: out[0]=kT of non-frozen particles, out[1..3]=momentum,
 * out[4..4+ns)=total amount of each species, out[4+ns]=number non-frozen. */
void orc_observables(const orc_sys *s, const double *vel, const double *conc, double *out);

int orc_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
