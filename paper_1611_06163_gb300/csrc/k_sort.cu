// Cell-list binning and deterministic counting sort (the reorder of Sec. 3.1,
// rebuilt every step instead of a Verlet list every few steps).
//
// Order within a cell is by particle id, so the sorted layout -- and with it
// every floating-point summation order -- depends only on the state, not on
// the order in which atomics happened to land.
#include "launch.h"

namespace tdpd {

__global__ void k_bin_init(Buffers b, const RepParams *__restrict__ reps, int n, int *count,
                           int2 *cellrank)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    float4 p = b.pos[k];
    int r = wbits(b.vel[k].w);
    const RepParams &P = reps[r];
    int c = cell_of(P, p.x, p.y, p.z);
    int rank = atomicAdd(count + c, 1);
    cellrank[k] = make_int2(c, rank);
}

// Single-CTA exclusive scan of the cell histogram; clears it for the next
// binning and advances the step counter.
__global__ void __launch_bounds__(1024) k_scan(int *count, int *cell_start, int n_cells,
                                               uint32_t *step_ctr, int inc)
{
    __shared__ int wsum[32];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int per = (n_cells + nt - 1) / nt;
    const int beg = min(tid * per, n_cells), end = min(beg + per, n_cells);
    int s = 0;
    for (int c = beg; c < end; ++c) s += count[c];
    // inclusive scan over the block
    int x = s;
    const int lane = tid & 31, w = tid >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
        int v = lane < (nt >> 5) ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        wsum[lane] = v;
    }
    __syncthreads();
    int run = x - s + (w > 0 ? wsum[w - 1] : 0);
    for (int c = beg; c < end; ++c) {
        int v = count[c];
        cell_start[c] = run;
        run += v;
        count[c] = 0;
    }
    if (tid == nt - 1) cell_start[n_cells] = run;
    if (tid == 0 && inc) *step_ctr += 1u;
}

__global__ void k_scatter_keys(const float4 *__restrict__ pos, const int2 *__restrict__ cellrank,
                               const int *__restrict__ cell_start, int2 *keys, int n)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int2 cr = cellrank[k];
    int id = wbits(pos[k].w) & ID_MASK;
    keys[cell_start[cr.x] + cr.y] = make_int2(id, k);
}

// Slot d of the new order: rank the key by id inside its cell, then gather
// the particle from its old slot, applying the velocity-Verlet predictor
// (r~ = r + dt v + dt^2/2 F, v~ = v + lambda dt F, C~ = C + lambda dt Q).
template <int NS>
__global__ void k_rank_gather(Buffers cur, Buffers nxt, const RepParams *__restrict__ reps,
                              const int2 *__restrict__ keys, const int2 *__restrict__ cellrank,
                              const int *__restrict__ cell_start, int *inv, int n, int ns_rt,
                              int predict)
{
    const int ns = NS > 0 ? NS : ns_rt;
    int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= n) return;
    int2 key = keys[d];
    const int id = key.x, src = key.y;
    const int c = cellrank[src].x;
    const int lo = cell_start[c], hi = cell_start[c + 1];
    int rank = 0;
    for (int e = lo; e < hi; ++e) rank += (keys[e].x < id);
    const int dst = lo + rank;

    float4 p = cur.pos[src];
    float4 v = cur.vel[src];
    float4 f = cur.frc[src];
    float4 vt = cur.vt[src];
    const int r = wbits(v.w);
    const RepParams &P = reps[r];
    const int type = (int)((uint32_t)wbits(p.w) >> 24);
    const bool frozen = (P.frozen_mask >> type) & 1u;
    float4 vtn = make_float4(v.x, v.y, v.z, vt.w);
    if (predict && !frozen) {
        bool flip;
        float3 rn = predict_pos(P, p, v, f, flip);
        p.x = rn.x; p.y = rn.y; p.z = rn.z;
        if (flip) { v.x = -v.x; v.y = -v.y; v.z = -v.z; }
        vtn.x = __fmaf_rn(P.ldt, f.x, v.x);
        vtn.y = __fmaf_rn(P.ldt, f.y, v.y);
        vtn.z = __fmaf_rn(P.ldt, f.z, v.z);
    }
    nxt.pos[dst] = p;
    nxt.vel[dst] = v;
    nxt.frc[dst] = f;
    nxt.vt[dst] = vtn;
    for (int s = 0; s < ns; ++s) {
        float cs = cur.C[(size_t)src * ns + s];
        float qs = cur.Q[(size_t)src * ns + s];
        nxt.C[(size_t)dst * ns + s] = cs;
        nxt.Q[(size_t)dst * ns + s] = qs;
        nxt.Ct[(size_t)dst * ns + s] = (predict && !frozen) ? __fmaf_rn(P.ldt, qs, cs) : cs;
    }
    inv[P.pbase + id] = dst;
}

static inline int nblk(int n, int t) { return (n + t - 1) / t; }

void launch_bin_init(const Buffers &b, const RepParams *reps, int n, int *count, int2 *cellrank,
                     cudaStream_t st)
{
    if (n <= 0) return;
    k_bin_init<<<nblk(n, 256), 256, 0, st>>>(b, reps, n, count, cellrank);
}

void launch_scan(int *count, int *cell_start, int n_cells, uint32_t *step_ctr, int inc,
                 cudaStream_t st)
{
    k_scan<<<1, 1024, 0, st>>>(count, cell_start, n_cells, step_ctr, inc);
}

void launch_scatter_keys(const Buffers &cur, const int2 *cellrank, const int *cell_start,
                         int2 *keys, int n, cudaStream_t st)
{
    if (n <= 0) return;
    k_scatter_keys<<<nblk(n, 256), 256, 0, st>>>(cur.pos, cellrank, cell_start, keys, n);
}

void launch_rank_gather(const Buffers &cur, const Buffers &nxt, const RepParams *reps,
                        const int2 *keys, const int2 *cellrank, const int *cell_start, int *inv,
                        int n, int ns, int predict, cudaStream_t st)
{
    if (n <= 0) return;
    const int g = nblk(n, 256);
    switch (ns) {
    case 1: k_rank_gather<1><<<g, 256, 0, st>>>(cur, nxt, reps, keys, cellrank, cell_start, inv, n, ns, predict); break;
    case 2: k_rank_gather<2><<<g, 256, 0, st>>>(cur, nxt, reps, keys, cellrank, cell_start, inv, n, ns, predict); break;
    default: k_rank_gather<0><<<g, 256, 0, st>>>(cur, nxt, reps, keys, cellrank, cell_start, inv, n, ns, predict); break;
    }
}

}  // namespace tdpd
