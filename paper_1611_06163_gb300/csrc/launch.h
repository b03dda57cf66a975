// Host-side launchers of the device kernels (one translation unit each).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace tdpd {

// Launch with programmatic stream serialization, so the kernel may start
// while its predecessor drains (it waits in pdl_enter for the results).
template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, cudaStream_t st, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

constexpr int OBS_K = 6 + 2 * MAXS;  // px, py, pz, sum v^2, n_mobile, n_membrane, species totals (all, membrane)
constexpr int OBS_CHUNK = 1024;   // slots per observables CTA
static_assert(OBS_K <= 256, "the last observables CTA sums one quantity per thread");

struct Buffers {
    float4 *pos, *vt, *vel, *frc;
    float *C, *Ct, *Q;
};

struct PairArgs {
    Buffers b;
    // neighbour-list mode: the other buffer, which receives each particle's
    // predicted state for the next step at its slot (what the next gather
    // would write for a replica that keeps its slots, bit for bit); pre.pos
    // null: not written (cell mode)
    Buffers pre;
    const float4 *fext;          // membrane force by load index (membrane particles only)
    float4 *mx, *mv;             // out: next predicted position and v~ of membrane particles
    const RepParams *reps;
    const int *cell_start;       // [NC+1]
    int *count;                  // [NC] histogram of the next binning (zeroed by scan)
    int2 *cellrank;              // [N] (cell, rank) of the next binning
    int *tile_sum;               // [n_tiles] particles per scan tile of the next binning
    uint32_t *err;               // [n_rep] status bits
    const uint32_t *quar;        // [n_rep] nonzero: the replica is quarantined (null: none)
    const uint32_t *step_ctr;    // absolute step of this evaluation
    int n;                       // particles (slots)
    int ns;                      // species (runtime value for the generic path)
    int integrate;               // 0: forces only (commit / set_state); 1: full step
    int lpp;                     // lanes per particle: 1, 2, 4, 8, 16 or 32
    int qr;                      // some replica has the random flux (general kernel)
    int std_exp;                 // every replica has s_f = 2 and s_c = 2 (kernels with them fixed)
    // neighbour-list mode (nl != nullptr): partners from the list instead of
    // the cell stencil, no binning in the epilogue
    const int *nl;               // [warps][cap][32] partner slots per lane
    const int *nlc;              // [n*lpp] entries per lane
    int cap;                     // entries per lane
    const float4 *xb;            // [n] positions at the last list build
    uint32_t *disp_next;         // [n_rep] max squared displacement (float bits) of the next positions
    // rebuild steps: rb (null: no build in the kernel) flags the replicas
    // whose lanes build their own lists first (into nl_w, nlc_w, xb_w: the
    // same arrays as nl, nlc, xb); m2: every replica has stencil half-width 2
    const uint32_t *rb;
    int *nl_w, *nlc_w;
    float4 *xb_w;
    int m2;
    // half-shell list mode (half != 0; the lists hold the upper half of the
    // stencil, every unordered pair once): the pair kernel adds each pair's
    // share for the partner into fixed-point accumulators and writes each
    // particle's own sums; k_pair_finish adds the two, applies the epilogue
    // (membrane and body force, sources, corrector, displacement) and clears
    // the accumulators
    int half;
    long long *accF;             // [n][4] partner forces, units of 2^-32 (zero between steps)
    long long *accQ;             // [n * ns] partner fluxes, units of 2^-40 (zero between steps)
    float4 *fown;                // [n] own force sums
    float *qown;                 // [n * ns] own flux sums
};

// Neighbour-list build over the cell stencil of radius sqrt(rlist2).
struct ListArgs {
    const float4 *pos, *vel;     // sorted state (vel.w: replica)
    const RepParams *reps;
    const int *cell_start;
    const uint32_t *rb;          // [n_rep + 1] rebuild flags, rb[n_rep]: any
    const uint32_t *quar;        // [n_rep] nonzero: quarantined, no list (null: none)
    int n_rep;
    int *nl, *nlc;
    float4 *xb;
    uint32_t *err;
    int n, lpp, cap;             // cap == 0: count only
    int m2;                      // every replica has the stencil half-width 2
    int half;                    // upper half of the stencil only (half-shell lists)
};

struct MemArgs {
    const float4 *mx, *mv;       // vertex position and v~ by load index
    const RepParams *reps;
    const RbcDev *rbcs;
    const int *tri;              // triangle table (RbcDev::tri_off)
    const FanEntry *fan;         // fan table (RbcDev::fan_off, fan_stride)
    const float *a0j;
    const float2 *bond;          // (l_m, k_p) per bond
    const float4 *ref_in;        // per-membrane reference point
    float4 *ref_out;             // next reference point (centroid)
    double2 *av_out;             // per-membrane (A, V) of these positions
    float2 *cgv_out;             // their constraint coefficients k_g (A - A0)/A0, k_v (V - V0)/V0
    const float2 *cgv_seq;       // coefficients K-Apply uses (this step's) ...
    const float2 *cgv_lag;       // ... or the previous step's, for a lagged replica
    float4 *fext;                // membrane force by load index
    uint32_t *mem_ctr;           // [2] step counters of the membrane kernels: this
    int q;                       // evaluation reads mem_ctr[q], sets mem_ctr[1-q] to it + 1
    int n_rbc, max_nv;
};

// in: x[3n], v[3n], C[n*ns] in load order; wstat: (id | type << 24, replica,
// membrane or -1, 0) per particle; membrane vertices also to mx, mv
void launch_pack_state(const float *in, const int4 *wstat, const Buffers &b, float4 *mx, float4 *mv, int n,
                       int ns, cudaStream_t st);
// load-order device copies of a replica's slots [base, base + n) (any of the
// outputs may be null); *bad set if the slot map is corrupt
void launch_unpack_state(const Buffers &b, const int *inv, int base, int n, int ns, float *pos, float *vel,
                         float *conc, uint32_t *bad, cudaStream_t st);
// *bad set if a position lies outside its replica's box or a velocity is not finite
void launch_check_state(const float *x3, const float *v3, const int4 *wstat, const RepParams *reps, int n,
                        uint32_t *bad, cudaStream_t st);
void launch_bin_init(const Buffers &b, const RepParams *reps, int n, int *count, int *tile_sum,
                     int2 *cellrank, cudaStream_t st);
// exclusive scan of count[0, n_tiles * SCAN_TILE) into cell_start; reads the
// tile totals tile_read, clears tile_clear and count for the next binning
// any (optional): skip all but the step counter when *any == 0
void launch_scan(int *count, int *cell_start, int n_tiles, const int *tile_read, int *tile_clear,
                 uint32_t *step_ctr, int inc, cudaStream_t st, const uint32_t *any = nullptr);
// rb (optional): only the particles of replicas with rb[r] set (their slots
// are the only ones re-sorted); any = rb + n_rep skips everything when none
void launch_scatter_keys(const Buffers &cur, const int2 *cellrank, const int *cell_start,
                         int2 *keys, int n, cudaStream_t st, const uint32_t *any = nullptr,
                         const uint32_t *rb = nullptr);
// Quarantine (optional): err [n_reps] is each replica's status word from the
// last force evaluation; a replica with a nonzero word is not moved (no
// predictor) and quar[r] = (err[r] != 0) tells the kernels after the gather
// to skip it.
// In list mode (rb set) a replica that keeps its slots is not gathered at
// all: the last pair epilogue wrote its predicted state into nxt already;
// only a quarantined one is copied (without the predictor).
struct Quarantine {
    const uint32_t *err = nullptr;
    uint32_t *quar = nullptr;
    int n_reps = 0;
};
void launch_rank_gather(const Buffers &cur, const Buffers &nxt, const RepParams *reps,
                        const int2 *keys, const int2 *cellrank, const int *cell_start, int *inv,
                        int n, int ns, int predict, cudaStream_t st,
                        const uint32_t *rb = nullptr, int n_rep = 0, int *tile_zero = nullptr, int n_tiles = 0,
                        const Quarantine &q = Quarantine{});
// list mode: rb[n_rep + 1] rebuild flags; without any rebuild every slot keeps
// its particle, a replica that does not rebuild keeps its slots; tile_zero
// (n_tiles ints) is cleared after a rebuild
// part: PAIR_WALK the pair kernel, PAIR_FINISH the half shell's finishing
// pass (nothing in full-shell and cell mode), or both
constexpr int PAIR_WALK = 1, PAIR_FINISH = 2, PAIR_ALL = 3;
void launch_pair(const PairArgs &a, cudaStream_t st, int part = PAIR_ALL);
// rb[r] = the displacement of replica r exceeds half its skin (or force);
// rb[n_rep] = any; disp_clear zeroed for the next evaluation; advances the
// step counter and counts each replica's rebuilds in builds
void launch_rebuild_decide(const uint32_t *disp, uint32_t *disp_clear, uint32_t *rb, const RepParams *reps,
                           int n_rep, int force, uint32_t *step_ctr, uint32_t *builds, cudaStream_t st);
// the rebuild decision folded into k_bin_next (disp null: taken by
// k_rebuild_decide before it); the fields as for launch_rebuild_decide
struct DecideArgs {
    const uint32_t *disp;
    uint32_t *disp_clear, *rb, *step_ctr, *builds;
    int n_rep;
};
// The one-launch sort of a list-mode step for a small system (k_sort_small):
// rebuild decision, binning, scan, scatter and gather in one thread-block
// cluster, separated by its hardware barrier.
constexpr int SORT_SMALL_THREADS = 1024;
constexpr int SORT_SMALL_ITEMS = 2;      // particles per thread at most
struct SortSmallArgs {
    Buffers cur, nxt;
    const RepParams *reps;
    int n, ns_rt, nc;            // particles, species, cells
    int *count;                  // [nc] zero on entry and on return
    int *cell_start;             // [nc + 1]
    int *inv;
    int2 *cellrank, *keys;       // [n] scratch
    DecideArgs D;
    Quarantine Qa;
};
// CTAs of the cluster for ns species: 16 where a 16-CTA cluster of the kernel
// can be resident, else 8, else 0 (not available); it serves at most
// ctas x SORT_SMALL_THREADS x SORT_SMALL_ITEMS particles
int sort_small_ctas(int ns);
void launch_sort_small(const SortSmallArgs &a, int ctas, cudaStream_t st);
// cell and rank of the next predicted position of each particle of a
// rebuilding replica (list mode, when any replica rebuilds; rb[r]: replica r
// rebuilds, unless d.disp is set and the decision is taken here); a replica
// that keeps its slots adds its particle count to its first cell
void launch_bin_next(const Buffers &b, const RepParams *reps, int n, int *count, int *tile_sum, int2 *cellrank,
                     const uint32_t *rb, const uint32_t *any, cudaStream_t st, const DecideArgs &d = DecideArgs{});
void launch_list_build(const ListArgs &a, cudaStream_t st);
// each membrane's reference point (ref_out[b]) from the load-order positions
// x3 (three floats per particle) of a loaded state; max_nv, max_stride: the
// largest vertex count and fan stride of the membranes
void launch_mem_ref(const float *x3, const RbcDev *rbcs, const FanEntry *fan, const RepParams *reps, float4 *ref_out,
                    int n_rbc, int max_nv, int max_stride, cudaStream_t st);
// pdl: launched as a programmatic dependent of the previous kernel on st
void launch_mem_gather(const MemArgs &a, cudaStream_t st, bool pdl);
void launch_mem_forces(const MemArgs &a, cudaStream_t st);
// chunks: (replica, first slot, end slot); part: OBS_K doubles per chunk;
// total: their sums over the chunks in chunk order (binary64); done: a
// counter at zero, left at zero
void launch_observables(const Buffers &b, const RepParams *reps, const int4 *chunks, int n_chunks,
                        int ns, double *part, double *total, unsigned *done, cudaStream_t st);
// Per-replica constants from a configuration and compact coefficient tables
// (pair_coef [T*T*3] = a, gamma, sigma; kappa [T*T*S]) for a given cell grid.
RepParams build_rep_params(const tdpd_config &c, const float *pair_coef, const float *kappa,
                           const int nc[3], int m, int cell_base, int pbase, int n);
// Validity of a replica configuration: false when valid, else true with the
// reason in msg (the checks of tdpd_create).
bool config_error(const tdpd_config &c, char *msg, size_t len);
// Message returned by tdpd_last_error(NULL) on this thread.
void set_thread_error(const char *msg);

void launch_debug_rng(uint64_t seed, int n, const uint32_t *i, const uint32_t *j,
                      const uint32_t *step, const uint32_t *stream, uint32_t *bits,
                      float *normal, cudaStream_t st);

}  // namespace tdpd
