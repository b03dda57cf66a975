// Verlet neighbour lists for the pair kernel (the list of Sec. 3.1 that is
// rebuilt every few steps rather than every step).
//
// A list holds, per lane of the pair kernel, the slots of the partners within
// rlist = rcut + skin of the particle at build time, found over the same cell
// stencil rows that lane would walk (rows s, s+LPP, ... of its particle). As
// long as no particle of the replica has moved more than skin/2 since the
// build, every pair closer than rcut is in the list. The pair kernel's
// epilogue records the largest displacement of each replica's next positions;
// the next step rebuilds exactly the replicas that crossed skin/2, so a
// replica's rebuild steps -- and its summation order -- do not depend on the
// other replicas of a batch.
//
// Layout: entry k of lane l of warp w at nl[(w * cap + k) * 32 + l], so the
// 32 lanes of a warp read one 128-byte line per entry.
//
// k_list_build builds the lists of a loaded state; on a rebuild step the pair
// kernel's one- and two-species forms build their own lanes' lists
// (list_lane.cuh), and k_list_build runs only for the other forms.
#include <algorithm>
#include <type_traits>

#include "launch.h"
#include "list_lane.cuh"

namespace tdpd {

__global__ void k_rebuild_decide(const uint32_t *__restrict__ disp, uint32_t *disp_clear, uint32_t *rb,
                                 const RepParams *__restrict__ reps, int n_rep, int force, uint32_t *step_ctr,
                                 uint32_t *builds)
{
    pdl_enter();
    int any = 0;
    for (int r = threadIdx.x; r < n_rep; r += blockDim.x) {
        const bool b = force || __uint_as_float(disp[r]) > reps[r].half_skin2;
        rb[r] = b ? 1u : 0u;
        disp_clear[r] = 0u;
        if (b) builds[r] += 1u;
        any |= b;
    }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) {
        rb[n_rep] = any ? 1u : 0u;
        *step_ctr += 1u;
    }
}

// Cell and rank of the position each particle of a rebuilding replica will
// have at the next force evaluation (the predictor of the gather), for the
// sort of a rebuild step. A replica that keeps its list keeps its slots: its
// particles are not binned, and its whole count goes to its first cell, so
// that the scan still gives every replica its own slot range.
// With D.disp set (few replicas) the rebuild decision is taken here instead
// of in k_rebuild_decide: every CTA reads the replicas' maxima itself, and
// CTA 0 records the decision as k_rebuild_decide would; otherwise rb holds it.
__global__ void k_bin_next(Buffers b, const RepParams *__restrict__ reps, int n, int *count, int *tile_sum,
                           int2 *cellrank, const uint32_t *any, const uint32_t *__restrict__ rb, DecideArgs D)
{
    pdl_enter();
    if (D.disp) {
        int a = 0;
        for (int r = threadIdx.x; r < D.n_rep; r += blockDim.x) {
            const bool rebuild = __uint_as_float(D.disp[r]) > reps[r].half_skin2;
            a |= rebuild;
            if (blockIdx.x == 0) {
                D.rb[r] = rebuild ? 1u : 0u;
                D.disp_clear[r] = 0u;
                if (rebuild) D.builds[r] += 1u;
            }
        }
        a = __syncthreads_or(a);
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            D.rb[D.n_rep] = a ? 1u : 0u;
            *D.step_ctr += 1u;
        }
        if (!a) return;
    } else if (!*any) {
        return;
    }
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    int c = -1;
    if (k < n) {
        const float4 v = b.vel[k];
        const int r = wbits(v.w);
        const RepParams &P = reps[r];
        const bool rebuild = D.disp ? __uint_as_float(D.disp[r]) > P.half_skin2 : rb[r] != 0u;
        if (rebuild) {
            const float4 p = b.pos[k];
            const int type = (int)((uint32_t)wbits(p.w) >> 24);
            float3 rn = make_float3(p.x, p.y, p.z);
            if (!((P.frozen_mask >> type) & 1u)) {
                bool flip;
                rn = predict_pos(P, p, v, b.frc[k], flip);
            }
            c = cell_of(P, rn.x, rn.y, rn.z);
            const int rank = atomicAdd(count + c, 1);
            cellrank[k] = make_int2(c, rank);
        } else if (k == P.pbase) {
            atomicAdd(count + P.cell_base, P.n);
            atomicAdd(tile_sum + (P.cell_base >> SCAN_TILE_LOG2), P.n);
        }
    }
    add_tile_count(tile_sum, c);
}

// One thread per pair lane.
template <int LPP, int M, bool HALF>
__global__ void __launch_bounds__(128) k_list_build(ListArgs A)
{
    pdl_enter();
    if (!A.rb[A.n_rep]) return;                       // no replica rebuilds
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = gt / LPP, sub = gt % LPP;
    if (i >= A.n) return;
    const float4 pi = A.pos[i];
    const int rep = wbits(A.vel[i].w);
    if (!A.rb[rep]) return;
    if (A.quar && A.quar[rep]) {                      // quarantined: an empty list
        A.nlc[gt] = 0;
        return;
    }
    build_lane<LPP, M, HALF>(A, gt, i, sub, pi, rep);
}

void launch_rebuild_decide(const uint32_t *disp, uint32_t *disp_clear, uint32_t *rb, const RepParams *reps,
                           int n_rep, int force, uint32_t *step_ctr, uint32_t *builds, cudaStream_t st)
{
    launch_pdl(k_rebuild_decide, 1, 256, st, disp, disp_clear, rb, reps, n_rep, force, step_ctr, builds);
}

void launch_bin_next(const Buffers &b, const RepParams *reps, int n, int *count, int *tile_sum, int2 *cellrank,
                     const uint32_t *rb, const uint32_t *any, cudaStream_t st, const DecideArgs &d)
{
    if (n <= 0 && !d.disp) return;
    launch_pdl(k_bin_next, std::max(1, (n + 255) / 256), 256, st, b, reps, n, count, tile_sum, cellrank, any, rb, d);
}

template <bool HALF>
static void launch_list_build_h(const ListArgs &a, int g, cudaStream_t st)
{
    if (a.m2) {
        switch (a.lpp) {
        case 1: launch_pdl(k_list_build<1, 2, HALF>, g, 128, st, a); break;
        case 2: launch_pdl(k_list_build<2, 2, HALF>, g, 128, st, a); break;
        case 4: launch_pdl(k_list_build<4, 2, HALF>, g, 128, st, a); break;
        case 8: launch_pdl(k_list_build<8, 2, HALF>, g, 128, st, a); break;
        case 16: launch_pdl(k_list_build<16, 2, HALF>, g, 128, st, a); break;
        default: launch_pdl(k_list_build<32, 2, HALF>, g, 128, st, a); break;
        }
        return;
    }
    switch (a.lpp) {
    case 1: launch_pdl(k_list_build<1, 0, HALF>, g, 128, st, a); break;
    case 2: launch_pdl(k_list_build<2, 0, HALF>, g, 128, st, a); break;
    case 4: launch_pdl(k_list_build<4, 0, HALF>, g, 128, st, a); break;
    case 8: launch_pdl(k_list_build<8, 0, HALF>, g, 128, st, a); break;
    case 16: launch_pdl(k_list_build<16, 0, HALF>, g, 128, st, a); break;
    default: launch_pdl(k_list_build<32, 0, HALF>, g, 128, st, a); break;
    }
}

void launch_list_build(const ListArgs &a, cudaStream_t st)
{
    if (a.n <= 0) return;
    const int g = (int)(((long)a.n * a.lpp + 127) / 128);
    if (a.half) launch_list_build_h<true>(a, g, st);
    else launch_list_build_h<false>(a, g, st);
}

}  // namespace tdpd
