/*
 * tdpd.h -- C ABI of libtdpd.so: transport Dissipative Particle Dynamics
 * (tDPD) with triangulated red-blood-cell (RBC) membranes on one GB300 GPU.
 *
 * The method is that of Blumers, Tang, Li, Li & Karniadakis, "GPU-accelerated
 * red blood cell simulations with transport dissipative particle dynamics"
 * (arXiv:1611.06163), Sec. 2:
 *   - pairwise conservative, dissipative and random forces (Eq. 1-4),
 *   - Fickian concentration flux per species (Eq. 5-6; the random flux Q^R
 *     of Eq. 7-8 is off by default, as Sec. 2.1 drops it, and available
 *     through tdpd_set_random_flux; Q^S is a first-order reaction A -> B),
 *   - membrane forces: WLC + POW bonds (Eq. 10-11), bond viscosity and random
 *     force (Eq. 12-13), global/local area and global volume constraints
 *     (Eq. 14-15), bending (Eq. 16),
 *   - a Groot-Warren modified velocity-Verlet update of r, v and C.
 *
 * Conventions shared by every call:
 *   - Every function returns tdpd_status; TDPD_OK is 0. On failure the
 *     handle's message is available from tdpd_last_error(). No C++ exception
 *     crosses this boundary. Calls on one handle are not thread-safe.
 *   - Handles are opaque. The library owns every device allocation behind a
 *     handle; the caller owns every pointer it passes. Host arrays are read or
 *     written during the call only (the call copies); none is retained.
 *   - Particle arrays are in load order: the free particles of each
 *     tdpd_add_particles call in order, then the vertices of each membrane
 *     (tdpd_add_rbc) in vertex order. pos/vel/force are float[n*3] (x,y,z per
 *     particle), conc/flux are float[n*n_species] (species fastest).
 *   - A particle's id is its load-order index within its replica; the pairwise
 *     random numbers are keyed on ids (Sec. 3.1 "particle signatures").
 *   - Work is enqueued on the stream given to tdpd_set_stream (default: the
 *     library's own stream). tdpd_step does not synchronise; reads into host
 *     memory do (tdpd_read_state_device, into device memory, does not).
 */
#ifndef TDPD_H
#define TDPD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TDPD_MAX_TYPES 4
#define TDPD_MAX_SPECIES 16
#define TDPD_MAX_IDS (1 << 24)      /* particles per replica */

typedef enum {
    TDPD_OK = 0,
    TDPD_EINVAL = 1,      /* bad argument or parameter (message says which) */
    TDPD_ENOMEM = 2,      /* device or host allocation failed */
    TDPD_ECUDA = 3,       /* a CUDA runtime call failed */
    TDPD_EOVERFLOW = 4,   /* an index or size limit was exceeded */
    TDPD_ENONFINITE = 5,  /* a replica produced a non-finite force or state */
    TDPD_ETIMEOUT = 6,    /* a bounded device wait gave up */
    TDPD_ESTATE = 7       /* call not valid in the handle's current state */
} tdpd_status;

typedef struct tdpd_sys tdpd_sys;

/* One replica: box, species, cut-offs and integrator (Sec. 2.1, Eq. 3-6).
 * The cell list needs at least three cells of edge >= max(rc, rcc) per axis. */
typedef struct {
    float L[3];                 /* box edges; positions live in [0, L) */
    int32_t periodic[3];        /* 1 periodic; axis 2 may be 0 (walls) */
    float wall_lo, wall_hi;     /* bounce-back planes along z if !periodic[2] */
    int32_t n_types;            /* 1..TDPD_MAX_TYPES */
    int32_t n_species;          /* 1..TDPD_MAX_SPECIES */
    uint64_t seed;              /* keys every random number of the replica */
    float dt, lambda;           /* time step; velocity-Verlet predictor lambda */
    float rc, s_f;              /* force cut-off; w_R = (1 - r/rc)^(s_f/2) */
    float rcc, s_c;             /* flux cut-off; w_DC = (1 - r/rcc)^s_c */
    float body_force[3];        /* added to every non-frozen particle */
    uint32_t frozen_types;      /* bit t: particles of type t are not moved */
    int32_t exclude_same_body;  /* 1: no Eq. 3 forces within one membrane */
    int32_t cells_per_cutoff;   /* cell-list stencil: cells of edge >= max(rc, rcc)/m
                                 * (plus the skin with lists), m = 1, 2 or 3; 0
                                 * selects 2, or the width commit finds fastest
                                 * when it times the list shape (tdpd_list_shape) */
} tdpd_config;

/* Membrane constants (Sec. 2.2). Bond l_m = l0/x0 and k_p are set per bond
 * so each bond is force-free at its rest length l0. V0 = v_ratio * A0^1.5
 * (the A-V scaling of Sec. 2.2); v_ratio <= 0 takes the rest volume. */
typedef struct {
    float kT, p, x0, m;         /* Eq. 10-11 */
    float kg, kl, kv;           /* Eq. 14-15 */
    float kb, theta0;           /* Eq. 16 */
    float gammaT, gammaC;       /* Eq. 12-13; needs 3*gammaC >= gammaT */
    float v_ratio;
    int32_t lagged_av;          /* nonzero: the area and volume constraints of a
                                 * step use the totals of the previous step's
                                 * positions (the concurrent K-Gather / K-Apply
                                 * of Sec. 3.3); the first evaluation after a
                                 * commit or state load uses its own */
} tdpd_membrane;

/* FP64 observables of one replica at its current step. */
typedef struct {
    int64_t step;
    int32_t n_particles, n_mobile, n_species, n_rbc;
    double kT;                          /* sum |v - vbar|^2 / (3 (n_mobile-1)) */
    double momentum[3];                 /* sum v over non-frozen particles */
    double mass[TDPD_MAX_SPECIES];      /* sum C_s over all particles */
    int32_t n_membrane;                 /* membrane vertices */
    int32_t pad_;
    double mass_membrane[TDPD_MAX_SPECIES]; /* sum C_s over membrane vertices */
} tdpd_obs;

/* ---------------------------------------------------------------- set-up */

/* Create a handle holding one replica described by cfg (Sec. 2.1). Pair
 * coefficients default to zero and every kappa to zero. */
tdpd_status tdpd_create(tdpd_sys **out, const tdpd_config *cfg);

/* Eq. 3 coefficients alpha_ij, gamma_ij, sigma_ij for the type pair (set
 * symmetrically; gamma, sigma finite and >= 0). tdpd_commit checks Eq. 4
 * (sigma^2 = 2 kT gamma): every type pair of a replica whose gamma or sigma
 * is nonzero must have both nonzero and the same sigma^2 / (2 gamma) within
 * a relative 1e-5, else TDPD_EINVAL. */
tdpd_status tdpd_set_pair(tdpd_sys *s, int type_i, int type_j, float a, float gamma, float sigma);

/* Eq. 6 kappa_ij of one species for the type pair (set symmetrically). */
tdpd_status tdpd_set_kappa(tdpd_sys *s, int type_i, int type_j, int species, float kappa);

/* Source term Q^S of Eq. 5: dC_dst/dt += k C_src, dC_src/dt -= k C_src on
 * particles whose type bit is set in types. */
tdpd_status tdpd_set_reaction(tdpd_sys *s, float k, int src, int dst, uint32_t types);

/* Random flux Q^R of Eq. 7 for every species: eps w_RC zeta / sqrt(dt) per
 * pair inside r_cc, with eps^2 = m_s^2 kappa rho (C~_i + C~_j) (Eq. 8;
 * negative sums count as zero) and w_RC = w_DC^(1/2). zeta is one standard
 * normal per pair, step and species (stream 6 + s/2 of the pair generator,
 * the cosine branch for even s, the sine branch for odd s), taken with sign
 * + on the side of the smaller id, so each pair exchanges solute. m_s = 0
 * (the default) leaves it out, as the paper does (m_s << m). rho is the
 * particle number density of the model, m_s the solute mass. Before commit;
 * TDPD_EINVAL for negative or non-finite values. Handles that use it run the
 * general (any species count) pair kernel. */
tdpd_status tdpd_set_random_flux(tdpd_sys *s, float m_s, float rho);

/* Body force profile: 0 (default) the configuration's body force everywhere;
 * 1 the double Poiseuille forcing of the flow validation (Sec. 4.1): the body
 * force where z < L_z/2 and its negative where z >= L_z/2, judged at the
 * position where the force is evaluated. Before commit; TDPD_EINVAL for
 * another mode. */
tdpd_status tdpd_set_body_force_profile(tdpd_sys *s, int mode);

/* Cylindrical wall for the Dirichlet transport validation (Sec. 4.2, Eq. 17):
 * a mobile particle whose predicted position lies farther than radius from
 * the axis y = L_y/2, z = L_z/2 (along x) is reflected back across the
 * cylinder surface and its velocity reversed, as at the bounce-back planes.
 * The concentration boundary itself comes from frozen particles outside the
 * cylinder, whose C the integrator never changes. radius 0 (the default)
 * disables it. Before commit; TDPD_EINVAL unless 0 <= radius and, for
 * radius > 0, y and z are periodic and 2 radius < min(L_y, L_z). */
tdpd_status tdpd_set_cylinder_wall(tdpd_sys *s, float radius);

/* Membrane constants for every membrane of the replica (Sec. 2.2). */
tdpd_status tdpd_set_membrane(tdpd_sys *s, const tdpd_membrane *m);

/* Append n free particles (host arrays; conc may be NULL for zeros). */
tdpd_status tdpd_add_particles(tdpd_sys *s, int n, const float *pos, const float *vel,
                               const float *conc, const int32_t *type);

/* Append one membrane: nv vertices (host pos/vel/conc, all of `type`) and
 * ntri triangles (int32[ntri*3], counter-clockwise seen from outside) of a
 * closed genus-0 surface (checked: V - E + F = 2, each edge in two opposite
 * triangles). rest_pos (may be NULL = pos) fixes l0, A0_j, A0, V0. Writes the
 * membrane's index to *rbc_index if not NULL. At most 1024 vertices. */
tdpd_status tdpd_add_rbc(tdpd_sys *s, int nv, const float *pos, const float *vel,
                         const float *conc, int type, int ntri, const int32_t *tri,
                         const float *rest_pos, int *rbc_index);

/* New handle advancing the given replicas together, every phase of a step
 * launched once for all of them (batched ensemble). Copies each replica's
 * description and current state; the inputs stay valid and independent. */
tdpd_status tdpd_batch_create(tdpd_sys **out, tdpd_sys *const *replicas, int n);

/* CUDA stream (cudaStream_t) on which later work is enqueued; NULL selects
 * the library's own stream. */
tdpd_status tdpd_set_stream(tdpd_sys *s, void *cuda_stream);

/* Lanes of the pair kernel that share one particle (1, 2, 4, 8, 16 or 32),
 * or 0 (the default) to time every choice at commit and keep the fastest.
 * The lanes split the particle's neighbour rows, so the order in which its
 * pair terms are summed, and with it the last bits of F and Q, depends on
 * this number; two handles with the same lanes (for instance a batch and its
 * replicas alone) give the same bits. Must be called before tdpd_commit;
 * TDPD_EINVAL for another value, TDPD_ESTATE after commit. No counterpart in
 * the paper (a scheduling choice of this implementation). */
tdpd_status tdpd_set_lanes(tdpd_sys *s, int lanes);

/* Lanes per particle the pair kernel uses (fixed at commit; before commit the
 * value tdpd_set_lanes set, 0 when timed). */
int tdpd_lanes(const tdpd_sys *s);

/* How the pair kernel covers the pairs in neighbour-list mode: 1 the full
 * shell (each particle walks all its partners, so every pair term of Eq. 3
 * and Eq. 6 is evaluated from both sides, by the pair symmetry of the random
 * numbers with equal results), 2 the half shell (each unordered pair once,
 * from the side where the partner's cell lies in the upper half of the
 * stencil; the partner's share -f_ij, -q_ij is summed in 64-bit fixed point
 * by integer atomics, which keeps the results independent of the order in
 * which they land), 0 (the default) chosen at commit: timed against each
 * other together with the lanes when the lanes are not pinned, else the half
 * shell. Cell mode (skin 0) always uses the full stencil. The mode changes
 * the order of the floating-point sums, so the last bits of F and Q depend
 * on it; two handles with the same lanes and mode give the same bits. Before
 * tdpd_commit; TDPD_EINVAL for another value, TDPD_ESTATE after commit. No
 * counterpart in the paper (its kernels evaluate every pair from both
 * sides). */
tdpd_status tdpd_set_pair_mode(tdpd_sys *s, int mode);

/* The pair mode in use after commit (1 full shell, 2 half shell; cell mode
 * reports 1); before commit the value tdpd_set_pair_mode set. */
int tdpd_pair_mode(const tdpd_sys *s);

/* The neighbour-list shape in use (commits the handle if needed): the skin
 * (0 in cell mode; a replica whose box is too small for it uses a smaller
 * one) and the stencil width m of the first replica (cells of edge >= (rcut
 * + skin)/m). When the lanes are not pinned (tdpd_set_lanes) and the skin is
 * not set (tdpd_set_skin), commit times whole steps (16, list rebuilds
 * included) for the skins 0.2, 0.15, 0.25, 0.3 and 0.4, each with m = 2 and
 * m = 3 unless a replica sets cells_per_cutoff, and keeps the first within
 * 3 % of the fastest in that order; tuning_ms (may be NULL) receives up to
 * max_tuning of those times, in that order, and *n_tuning their count (0
 * when nothing was timed). No counterpart in the paper (it rebuilds its list
 * every few steps at a fixed radius). */
tdpd_status tdpd_list_shape(tdpd_sys *s, float *skin, int *cells_per_cutoff, float *tuning_ms, int max_tuning,
                            int *n_tuning);

/* How a neighbour-list step sorts the replicas that rebuild their lists
 * (the reorder of Sec. 3.1): 0 (default) chosen at commit, 1 a chain of
 * kernels over the whole GPU (binning, scan, scatter, gather), 2 one launch
 * of one thread-block cluster (8 or 16 CTAs) doing all four, its phases
 * separated by the cluster barrier -- for systems of at most 32,768
 * particles (16,384 where only an 8-CTA cluster fits) and 1,048,576 cells,
 * where the chain's launches cost more than its work. Both give the same sorted order and the same bits. With 0,
 * commit times 16 steps of each (one graph replay each) where the cluster
 * sort fits, and keeps it unless the chain is more than 3 % faster. Before
 * tdpd_commit; TDPD_EINVAL for another value, TDPD_ESTATE after commit;
 * commit fails with TDPD_EINVAL when 2 is set and the cluster sort does not
 * fit (cell mode: the setting is ignored). */
tdpd_status tdpd_set_sort_mode(tdpd_sys *s, int mode);

/* The sort in use after commit (1 kernel chain, 2 one cluster; cell mode
 * reports 1); before commit the value tdpd_set_sort_mode set. tuning_ms (may
 * be NULL, 2 floats): the times commit took for 16 steps with the cluster
 * and with the chain, -1 when it did not time them. */
int tdpd_sort_mode(const tdpd_sys *s, float *tuning_ms);

/* Skin of the Verlet neighbour lists of the pair kernel (length units): each
 * particle keeps the partners within max(rc, rcc) + skin found at a list
 * build; a replica rebuilds its lists (and re-sorts its cells) in the step
 * after one of its particles has moved more than skin/2 from its position at
 * the last build, which keeps every pair inside the cut-off in the lists
 * (Sec. 3.1 rebuilds the list every few steps). 0 selects cell mode: no
 * lists, the cell stencil is walked and the particles re-sorted every step.
 * Default (not called): 0.2, or, when the lanes are not pinned, the skin
 * commit finds fastest (see tdpd_list_shape). A replica whose box is too small for the skin
 * (rcut + 2 skin must not exceed half a periodic edge, and the cells of edge
 * (rcut + skin)/m must fit 2m+1 times) gets a smaller one. The skin changes
 * the order in which pair terms are summed, so results agree to rounding,
 * not bitwise, across skins. Before tdpd_commit; TDPD_EINVAL for a negative
 * or non-finite value, TDPD_ESTATE after commit. A list that overflows its
 * capacity (sized at commit to 1.5 x the longest list plus 16) marks its
 * replica TDPD_EOVERFLOW in tdpd_replica_status. */
tdpd_status tdpd_set_skin(tdpd_sys *s, float skin);

/* Number of steps since commit in which replica r rebuilt its neighbour lists
 * (0 in cell mode; the builds at commit and at state loads are not counted). */
tdpd_status tdpd_list_rebuilds(tdpd_sys *s, int r, int64_t *out);

/* Upload, bin and compute the forces F(0), Q(0) of the loaded state. Called
 * implicitly by the first step or read; afterwards no particles can be added. */
tdpd_status tdpd_commit(tdpd_sys *s);

/* --------------------------------------------------------------- advance */

/* Advance every replica by n steps (n >= 0): per step a cell-list binning and
 * sort, the membrane forces, the pair force + flux and the velocity-Verlet
 * update, all on the device and replayed from a captured CUDA graph. */
tdpd_status tdpd_step(tdpd_sys *s, int n);

/* One step (as tdpd_step(s, 1)) from a graph that also records CUDA events
 * around each of its kernels on the same stream; waits for it and writes the
 * duration in milliseconds of each kernel, in launch order, to kernel_ms
 * (at most max_kernels values; *n_kernels receives the count). Names of the
 * kernels come from tdpd_kernel_name. */
tdpd_status tdpd_step_timed(tdpd_sys *s, float *kernel_ms, int max_kernels, int *n_kernels);
const char *tdpd_kernel_name(const tdpd_sys *s, int k);

/* Wait for enqueued work; returns TDPD_ENONFINITE if any replica reported a
 * non-finite value (TDPD_EOVERFLOW: a neighbour list overflowed) since the
 * last commit or state load (see tdpd_replica_status). */
tdpd_status tdpd_sync(tdpd_sys *s);

/* Replace the state of replica r (host arrays in load order) and recompute
 * F, Q at the current step. conc may be NULL to keep the concentrations. */
tdpd_status tdpd_set_state(tdpd_sys *s, int replica, const float *pos, const float *vel,
                           const float *conc);

/* Replace the state of every replica at once and recompute F, Q at the
 * current step: pos[3 N], vel[3 N], conc[N ns] hold the replicas one after
 * another in replica order, each in its load order (N = the total particle
 * count; the layout tdpd_read_state gives replica by replica). The arrays go
 * to the device as they are (by DMA when pinned) and are read before the call
 * returns. TDPD_EINVAL for a null array, a position outside its replica's box
 * or a non-finite velocity, naming the first such particle (nothing is
 * changed then); the check runs on the device after the upload. Every state
 * load (this call, tdpd_set_state, commit) takes each membrane's reference
 * point for its area and volume sums from its vertices on the device: the
 * centroid of the vertices unwrapped along the mesh by the minimum image. */
tdpd_status tdpd_set_states(tdpd_sys *s, const float *pos, const float *vel, const float *conc);

/* Device-memory variants for callers whose arrays live on the GPU (a torch
 * tensor's data pointer, say); the caller keeps ownership of its arrays.
 * tdpd_set_states_device: as tdpd_set_states with device pointers; the
 * check of positions and velocities runs on the device (TDPD_EINVAL, nothing
 * changed, on a violation); returns when the arrays have been read.
 * tdpd_read_state_device: enqueues on the library's stream (tdpd_set_stream)
 * a copy of replica r's state in load order into pos[3 n], vel[3 n],
 * conc[n ns] (any may be NULL) and returns at once: synchronise that stream
 * before reading them. */
tdpd_status tdpd_set_states_device(tdpd_sys *s, const float *pos, const float *vel, const float *conc);
tdpd_status tdpd_read_state_device(tdpd_sys *s, int replica, float *pos, float *vel, float *conc);

/* Checkpoint and restart. tdpd_save writes the device state between two
 * steps to the file path (a binary format of this library: the sorted
 * state, predicted values, forces, fluxes, neighbour lists, binning,
 * step and membrane counters, membrane reference points and area/volume
 * totals, status words). tdpd_load reads it into a committed handle of the
 * same configuration (same replicas, parameters, particle and membrane
 * counts, skin and lane count), which then continues exactly as the saved run
 * would have: the random numbers are keyed on the step, so a restart gives
 * the same bits. TDPD_EINVAL: the file cannot be opened, is not a checkpoint,
 * belongs to another configuration or is truncated (in the last case the
 * handle must be loaded again before use). Both commit an uncommitted handle
 * first, as tdpd_step does. */
tdpd_status tdpd_save(tdpd_sys *s, const char *path);
tdpd_status tdpd_load(tdpd_sys *s, const char *path);

/* ------------------------------------------------------------------ read */

tdpd_status tdpd_read_state(tdpd_sys *s, int replica, float *pos, float *vel, float *conc);
/* Total force (pair + membrane + body force) and flux (pair + source) of the
 * current step, the values the next update uses. */
tdpd_status tdpd_read_forces(tdpd_sys *s, int replica, float *force, float *flux);
tdpd_status tdpd_read_observables(tdpd_sys *s, int replica, tdpd_obs *out);
/* Area and volume (FP64, compensated sums) of each membrane of the replica at
 * the current step, as used by the constraint forces (Eq. 14-15). */
tdpd_status tdpd_read_rbc(tdpd_sys *s, int replica, double *area, double *volume);
/* Per-replica status words (TDPD_OK, TDPD_ENONFINITE, or TDPD_EOVERFLOW for
 * an overflowed neighbour list), int32[n_replicas]. A replica whose status is
 * not TDPD_OK is quarantined from the next step on: its particles are neither
 * moved nor re-evaluated (state, forces and fluxes stay as the faulting
 * evaluation left them, and its neighbour lists are not rebuilt), while the
 * other replicas of the batch step on unaffected (each replica only ever
 * interacts with itself). Loading a state (tdpd_set_state, tdpd_set_states,
 * tdpd_set_states_device) clears every status and evaluates the forces again,
 * which sets the status again if the loaded state still faults. */
tdpd_status tdpd_replica_status(tdpd_sys *s, int32_t *status);

int tdpd_num_replicas(const tdpd_sys *s);
int tdpd_num_particles(const tdpd_sys *s, int replica);
int64_t tdpd_current_step(const tdpd_sys *s);
/* Kernel launches one tdpd_step(s, 1) enqueues (after commit). */
int tdpd_launches_per_step(const tdpd_sys *s);

const char *tdpd_last_error(const tdpd_sys *s);
void tdpd_destroy(tdpd_sys *s);

/* ----------------------------------------------------------- parity hook */

/* The device pairwise random numbers (Sec. 3.1): for each k the TEA output
 * bits[2k..2k+1] for the pair (i[k], j[k]) at step[k], stream[k], and the two
 * standard normals normal[2k..2k+1] the force kernels draw from them.
 * Host arrays; runs on the current device and synchronises. */
tdpd_status tdpd_debug_rng(uint64_t seed, int n, const uint32_t *i, const uint32_t *j,
                           const uint32_t *step, const uint32_t *stream,
                           uint32_t *bits, float *normal);

/* ------------------------------------------------------ surrogate network */

/* A learned surrogate of parameter sweeps (no counterpart in the paper, which
 * runs each parameter point as a plain simulation): an ensemble of
 * 4 -> 64 -> 64 -> 2 perceptrons with GELU hidden layers (erf form), weights
 * used rounded to bfloat16 with float accumulation, inputs and outputs
 * standardised by the training set's mean and population deviation, trained
 * by full-batch Adam (beta1 0.9, beta2 0.999, eps 1e-8) on the mean squared
 * error of the standardised outputs. The members' spread is the uncertainty.
 * Parameter vector per member (TDPD_MLP_NPARAM floats): W1[64][4], b1[64],
 * W2[64][64], b2[64], W3[2][64], b3[2], row-major (output, input). Errors
 * are reported through tdpd_last_error(NULL). */
#define TDPD_MLP_IN 4
#define TDPD_MLP_HIDDEN 64
#define TDPD_MLP_OUT 2
#define TDPD_MLP_NPARAM 4610

typedef struct tdpd_mlp tdpd_mlp;

tdpd_status tdpd_mlp_create(tdpd_mlp **out, int members);
/* float master weights of every member, host float[members * NPARAM];
 * resets the Adam moments. */
tdpd_status tdpd_mlp_set_params(tdpd_mlp *m, const float *params);
tdpd_status tdpd_mlp_get_params(tdpd_mlp *m, float *params);
/* Training set: host X float[n*4], Y float[n*2] (raw units); fixes the
 * standardisation used by training and prediction. */
tdpd_status tdpd_mlp_set_data(tdpd_mlp *m, int n, const float *X, const float *Y);
/* Loss of each member on the training set and its gradient with respect to
 * the (bfloat16-rounded) parameters: loss double[members], grad float[members
 * * NPARAM] (either may be NULL). */
tdpd_status tdpd_mlp_loss_grad(tdpd_mlp *m, double *loss, float *grad);
/* steps full-batch Adam steps of every member; loss (may be NULL) receives
 * each member's loss after the last step. */
tdpd_status tdpd_mlp_train(tdpd_mlp *m, int steps, float lr, double *loss);
/* Ensemble prediction for host X float[n*4] (raw units): mean float[n*2],
 * rel_spread float[n*2] = sample standard deviation / |mean| across members
 * (may be NULL), member_out float[members*n*2] (may be NULL). */
tdpd_status tdpd_mlp_predict(tdpd_mlp *m, int n, const float *X, float *mean, float *rel_spread,
                             float *member_out);
void tdpd_mlp_destroy(tdpd_mlp *m);

/* ------------------------------------------------ allocation-free variant */

/* Limits of tdpd_pair_forces_noalloc; its scratch is a fixed device array of
 * at most TDPD_NOALLOC_SCRATCH_BYTES that every GPU which loads this library
 * holds until the process exits. */
#define TDPD_NOALLOC_MAX_PARTICLES 16384
#define TDPD_NOALLOC_MAX_CELLS 16384
#define TDPD_NOALLOC_MAX_SPECIES 4
#define TDPD_NOALLOC_SCRATCH_BYTES (5u << 20)

/* Pair force and flux of one periodic box, computed without allocating or
 * freeing any memory. The paper has no counterpart: this serves callers that
 * cannot call cudaMalloc -- a host program that hands all device memory to its
 * own pool allocator, or a per-step callback inside another simulation
 * engine, where an allocation would synchronise the device or is not allowed.
 * Such a caller owns every buffer it passes; everything else this call needs
 * lives in one fixed scratch array inside the library.
 *
 * Computes, for n free particles (no membranes) of a box with every axis
 * periodic, the same pair force (plus the configuration's body force) and
 * the same flux as tdpd_commit followed by tdpd_read_forces, at step number
 * `step`, with the same kernels and random numbers. No reaction source is
 * applied (this call takes no reaction parameters).
 *   cfg        host; box, species, cut-offs, seed (every axis periodic); the
 *              checks of tdpd_create apply
 *   pair_coef  host float[n_types*n_types*3]: a, gamma, sigma per type pair
 *   kappa      host float[n_types*n_types*n_species]
 *   pos, vel   device float[n*3]; positions in [0, L)
 *   conc       device float[n*n_species]
 *   type       device int32[n], each in [0, n_types)
 *   force      device float[n*3] (written), flux device float[n*n_species] (written)
 *   stream     cudaStream_t on which the work is enqueued (NULL: default stream)
 * Limits: n <= TDPD_NOALLOC_MAX_PARTICLES, cells (edge >= max(rc, rcc)/m) <=
 * TDPD_NOALLOC_MAX_CELLS, n_species <= TDPD_NOALLOC_MAX_SPECIES; larger inputs
 * return TDPD_EINVAL with the reason in tdpd_last_error(NULL), before any
 * device work. The call only enqueues (no synchronisation) and returns no
 * device-side status: when a type lies outside [0, n_types) or a force comes
 * out non-finite, every element of force and flux is NaN, so the caller
 * checks the outputs for non-finite values. The first call on a device looks
 * up the scratch array's device address (cudaGetSymbolAddress) with that
 * device current and keeps it for the life of the process; make that first
 * call before any stream capture. The kept address does not survive
 * cudaDeviceReset (do not call this entry point after a reset of a device it
 * has used). Every call on a device reuses the same scratch, which keeps the
 * previous call's contents (the call clears what must start at zero): calls
 * whose work overlaps on the GPU -- from several streams or threads -- race
 * and must be serialised by the caller. */
tdpd_status tdpd_pair_forces_noalloc(const tdpd_config *cfg, const float *pair_coef,
                                     const float *kappa, int n, const float *pos, const float *vel,
                                     const float *conc, const int32_t *type, uint32_t step,
                                     float *force, float *flux, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* TDPD_H */
