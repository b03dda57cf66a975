// Cell-list binning and deterministic counting sort (the reorder of Sec. 3.1).
// In cell mode the sort runs every step; in neighbour-list mode only in the
// steps that rebuild the list, and the gather then keeps every slot's
// particle in the other steps (it still applies the predictor).
//
// Order within a cell is by particle id, so the sorted layout -- and with it
// every floating-point summation order -- depends only on the state, not on
// the order in which atomics happened to land.
#include <cooperative_groups.h>

#include "launch.h"

namespace tdpd {

__global__ void k_bin_init(Buffers b, const RepParams *__restrict__ reps, int n, int *count,
                           int *tile_sum, int2 *cellrank)
{
    pdl_enter();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    int c = -1;
    if (k < n) {
        const float4 p = b.pos[k];
        const RepParams &P = reps[wbits(b.vel[k].w)];
        c = cell_of(P, p.x, p.y, p.z);
        const int rank = atomicAdd(count + c, 1);
        cellrank[k] = make_int2(c, rank);
    }
    add_tile_count(tile_sum, c);
}

// Exclusive scan of the cell histogram over all replicas at once (replicas
// occupy consecutive cells and consecutive slots, so one global scan gives
// every replica's cell_start). One CTA per tile of SCAN_TILE cells; the tile
// totals were accumulated by the binning, so each CTA finds its offset by
// summing the totals of the tiles before it -- no inter-CTA waiting.
__global__ void __launch_bounds__(1024) k_scan(int *count, int *cell_start, const int *tile_read,
                                               int *tile_clear, uint32_t *step_ctr, int inc,
                                               const uint32_t *any)
{
    pdl_enter();
    if (blockIdx.x == 0 && threadIdx.x == 0 && inc) *step_ctr += 1u;
    if (any && !*any) return;
    __shared__ int wsum[32];
    __shared__ int base_sh;
    const int t = blockIdx.x, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    // offset of this tile
    int pre = 0;
    for (int u = tid; u < t; u += blockDim.x) pre += tile_read[u];
    for (int o = 16; o > 0; o >>= 1) pre += __shfl_down_sync(0xffffffffu, pre, o);
    if (lane == 0) wsum[w] = pre;
    __syncthreads();
    if (w == 0) {
        int v = wsum[lane];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) base_sh = v;
    }
    __syncthreads();
    const int base = base_sh;
    // four consecutive cells per thread
    int4 *c4 = reinterpret_cast<int4 *>(count + (size_t)t * SCAN_TILE) + tid;
    const int4 cnt = *c4;
    const int s = cnt.x + cnt.y + cnt.z + cnt.w;
    int x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    __syncthreads();
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
        int v = wsum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        wsum[lane] = v;
    }
    __syncthreads();
    const int e = base + x - s + (w > 0 ? wsum[w - 1] : 0);
    int4 out;
    out.x = e;
    out.y = e + cnt.x;
    out.z = out.y + cnt.y;
    out.w = out.z + cnt.z;
    reinterpret_cast<int4 *>(cell_start + (size_t)t * SCAN_TILE)[tid] = out;
    *c4 = make_int4(0, 0, 0, 0);
    if (tid == 0) tile_clear[t] = 0;
}

__global__ void k_scatter_keys(const float4 *__restrict__ pos, const float4 *__restrict__ vel,
                               const int2 *__restrict__ cellrank, const int *__restrict__ cell_start, int2 *keys,
                               int n, const uint32_t *any, const uint32_t *__restrict__ rb)
{
    pdl_enter();
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n || (any && !*any)) return;
    if (rb && !rb[wbits(vel[k].w)]) return;          // a replica that keeps its slots
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
                              int predict, const uint32_t *__restrict__ rb, int n_rep, int *tile_zero,
                              int n_tiles, Quarantine Qa)
{
    pdl_enter();
    const int ns = NS > 0 ? NS : ns_rt;
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    // the quarantine of this step: every replica whose last force evaluation
    // set its status word (the word does not change before this step's pair
    // kernel, which reads quar instead)
    if (Qa.quar)
        for (int r = d; r < Qa.n_reps; r += gridDim.x * blockDim.x) Qa.quar[r] = Qa.err[r] != 0u ? 1u : 0u;
    const bool any = !rb || rb[n_rep] != 0u;
    if (tile_zero && any)
        for (int t = d; t < n_tiles; t += gridDim.x * blockDim.x) tile_zero[t] = 0;
    bool valid = d < n;
    int id = 0, src = 0, dst = 0;
    bool pred = false;          // the species rows get the predictor
    float ldt = 0.0f;
    if (valid && rb) {
        // list mode: a replica that keeps its list keeps its slots (replicas
        // own fixed slot ranges, so slot d's replica is that of the particle
        // there), and the last pair epilogue already wrote its predicted
        // state into nxt at those slots; only a quarantined replica, which
        // that epilogue skipped, is copied here
        const int r = wbits(cur.vel[d].w);
        if ((!any || rb[r] == 0u) && !(Qa.err && Qa.err[r] != 0u)) valid = false;
    }
    if (valid) {
        const bool keep = !any || (rb && rb[wbits(cur.vel[d].w)] == 0u);
        if (!keep) {
            const int2 key = keys[d];
            id = key.x;
            src = key.y;
            const int c = cellrank[src].x;
            const int lo = cell_start[c], hi = cell_start[c + 1];
            int rank = 0;
            for (int e = lo; e < hi; ++e) rank += (keys[e].x < id);
            dst = lo + rank;
        } else {
            src = dst = d;
            id = wbits(cur.pos[d].w) & ID_MASK;
        }

        float4 p = cur.pos[src];
        float4 v = cur.vel[src];
        float4 f = cur.frc[src];
        float4 vt = cur.vt[src];
        const int r = wbits(v.w);
        const RepParams &P = reps[r];
        const int type = (int)((uint32_t)wbits(p.w) >> 24);
        const bool frozen = (P.frozen_mask >> type) & 1u;
        const bool held = Qa.err && Qa.err[r] != 0u;     // quarantined: not moved
        float4 vtn = make_float4(v.x, v.y, v.z, vt.w);
        pred = predict && !frozen && !held;
        ldt = P.ldt;
        if (pred) {
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
        inv[P.pbase + id] = dst;
    }
    // species rows, the warp's 32 particles together: element e of the warp's
    // ns * 32 values is species e % ns of its particle e / ns, so consecutive
    // lanes touch consecutive floats of a row (several rows per instruction)
    const int lane = threadIdx.x & 31;
    const int total = ns * 32;
    for (int base = 0; base < total; base += 32) {
        const int e = base + lane;
        const int q = e / ns, sp = e - q * ns;           // particle (lane) and species
        const int sq = __shfl_sync(0xffffffffu, src, q);
        const int dq = __shfl_sync(0xffffffffu, dst, q);
        const int pq = __shfl_sync(0xffffffffu, pred ? 1 : 0, q);
        const float lq = __shfl_sync(0xffffffffu, ldt, q);
        const int vq = __shfl_sync(0xffffffffu, valid ? 1 : 0, q);
        if (e < total && vq) {
            const float cs = cur.C[(size_t)sq * ns + sp];
            const float qs = cur.Q[(size_t)sq * ns + sp];
            nxt.C[(size_t)dq * ns + sp] = cs;
            nxt.Q[(size_t)dq * ns + sp] = qs;
            nxt.Ct[(size_t)dq * ns + sp] = pq ? __fmaf_rn(lq, qs, cs) : cs;
        }
    }
}

// The sort of a list-mode step for a small system in one launch. The grid is
// one thread-block cluster, whose CTAs are resident together, so the phases
// are separated by the cluster's hardware barrier (no flag is polled). Each
// thread owns up to ITEMS particles (slots g, g + G, ...) and keeps their
// state in registers from the binning to the final write:
//   decision   every CTA reads each replica's largest displacement (the last
//              pair epilogue's) and takes the rebuild decision itself; CTA 0
//              records it, clears the next maxima, counts the builds,
//              advances the step counter and sets the quarantine;
//   binning    (some replica rebuilds) cell and arrival rank of each owned
//              particle's predicted position, a kept replica's count to its
//              first cell; a quarantined replica that keeps its slots is
//              copied as it stands;
//   scan       each CTA scans a contiguous range of cells, its offset the sum
//              of the lower CTAs' totals read from their shared memory;
//   scatter    each owned particle's (id, old slot) key into its cell's range;
//   placement  each owned particle's slot: its cell's start plus the number
//              of keys of the cell with a smaller id; the predicted state
//              (velocity-Verlet predictor, as in k_rank_gather) is written
//              there.
// The order (cell, then id) is unique, so the result is that of k_bin_next,
// k_scan, k_scatter_keys and k_rank_gather, bit for bit.
template <int NS, int ITEMS>
__global__ void __launch_bounds__(SORT_SMALL_THREADS, 1) k_sort_small(SortSmallArgs A)
{
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    __shared__ int wsum[SORT_SMALL_THREADS / 32];
    __shared__ int cta_total;
    pdl_enter();
    const int ns = NS > 0 ? NS : A.ns_rt;
    const int nct = gridDim.x, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int G = nct * SORT_SMALL_THREADS;
    const int g = blockIdx.x * SORT_SMALL_THREADS + tid;
    const DecideArgs &D = A.D;
    const uint32_t *err = A.Qa.err;

    int a = 0, h = 0;
    for (int r = tid; r < D.n_rep; r += SORT_SMALL_THREADS) {
        const bool rebuild = __uint_as_float(D.disp[r]) > A.reps[r].half_skin2;
        const bool held = err[r] != 0u;
        a |= rebuild;
        h |= held;
        if (blockIdx.x == 0) {
            D.rb[r] = rebuild ? 1u : 0u;
            D.disp_clear[r] = 0u;
            if (rebuild) D.builds[r] += 1u;
            A.Qa.quar[r] = held ? 1u : 0u;
        }
    }
    const bool any = __syncthreads_or(a) != 0;
    const bool any_held = __syncthreads_or(h) != 0;
    if (blockIdx.x == 0 && tid == 0) {
        D.rb[D.n_rep] = any ? 1u : 0u;
        *D.step_ctr += 1u;
    }
    // no rebuild and no quarantined replica (the common step): every slot
    // keeps its particle, whose predicted state the last epilogue wrote
    if (!any && !any_held) return;

    // binning of the owned particles (a rebuilding replica's: kept in
    // registers; a quarantined replica that keeps its slots: copied now)
    float4 p[ITEMS], v[ITEMS], f[ITEMS];
    float vtw[ITEMS];
    int cell[ITEMS], rank[ITEMS];
    bool mine[ITEMS], pred[ITEMS];
    float cs_[ITEMS][NS > 0 ? NS : 1], qs_[ITEMS][NS > 0 ? NS : 1];
    bool rebuild[ITEMS], held[ITEMS];
    // every owned particle's loads first (all in flight together), then the
    // arithmetic and the atomics
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const int k = g + i * G;
        rebuild[i] = held[i] = false;
        if (k < A.n) {
            v[i] = A.cur.vel[k];
            const int r = wbits(v[i].w);
            rebuild[i] = __uint_as_float(D.disp[r]) > A.reps[r].half_skin2;
            held[i] = err[r] != 0u;
        }
    }
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const int k = g + i * G;
        if (!rebuild[i]) continue;
        p[i] = A.cur.pos[k];
        f[i] = A.cur.frc[k];
        vtw[i] = A.cur.vt[k].w;
        if constexpr (NS > 0) {
#pragma unroll
            for (int sp = 0; sp < NS; ++sp) {
                cs_[i][sp] = A.cur.C[(size_t)k * NS + sp];
                qs_[i][sp] = A.cur.Q[(size_t)k * NS + sp];
            }
        }
    }
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const int k = g + i * G;
        mine[i] = false;
        pred[i] = false;
        cell[i] = rank[i] = 0;
        if (k >= A.n) continue;
        const RepParams &P = A.reps[wbits(v[i].w)];
        if (rebuild[i]) {
            const int type = (int)((uint32_t)wbits(p[i].w) >> 24);
            const bool frozen = (P.frozen_mask >> type) & 1u;
            float3 rn = make_float3(p[i].x, p[i].y, p[i].z);
            bool flip = false;
            if (!frozen) rn = predict_pos(P, p[i], v[i], f[i], flip);
            cell[i] = cell_of(P, rn.x, rn.y, rn.z);
            rank[i] = atomicAdd(A.count + cell[i], 1);
            mine[i] = true;
            pred[i] = !frozen && !held[i];
            if (pred[i]) {
                p[i].x = rn.x; p[i].y = rn.y; p[i].z = rn.z;
                if (flip) { v[i].x = -v[i].x; v[i].y = -v[i].y; v[i].z = -v[i].z; }
            }
        } else {
            if (k == P.pbase && any) atomicAdd(A.count + P.cell_base, P.n);
            if (held[i]) {
                // as the gather copies a quarantined replica: no predictor
                const float4 q = v[i];
                A.nxt.pos[k] = A.cur.pos[k];
                A.nxt.vel[k] = q;
                A.nxt.frc[k] = A.cur.frc[k];
                A.nxt.vt[k] = make_float4(q.x, q.y, q.z, A.cur.vt[k].w);
                for (int sp = 0; sp < ns; ++sp) {
                    const float c = A.cur.C[(size_t)k * ns + sp];
                    A.nxt.C[(size_t)k * ns + sp] = c;
                    A.nxt.Q[(size_t)k * ns + sp] = A.cur.Q[(size_t)k * ns + sp];
                    A.nxt.Ct[(size_t)k * ns + sp] = c;
                }
                A.inv[P.pbase + (wbits(A.cur.pos[k].w) & ID_MASK)] = k;
            }
        }
    }
    if (!any) return;              // uniform over the cluster: no barrier follows
    // (the cluster barrier's arrive has release and its wait acquire
    // semantics at cluster scope, which orders these global writes for the
    // other CTAs; their reads of them go through L2)
    cl.sync();

    // scan: CTA b owns cells [c0, c1), each thread a run of `per` of them
    {
        const int chunk = (A.nc + nct - 1) / nct;
        const int c0 = min(blockIdx.x * chunk, A.nc), c1 = min(c0 + chunk, A.nc);
        const int per = (chunk + SORT_SMALL_THREADS - 1) / SORT_SMALL_THREADS;
        const int lo = min(c0 + tid * per, c1), hi = min(lo + per, c1);
        int s = 0;
        for (int c = lo; c < hi; ++c) s += __ldcg(A.count + c);
        int x = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[w] = x;
        __syncthreads();
        if (w == 0) {
            int t = wsum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += y;
            }
            wsum[lane] = t;
            if (lane == 31) cta_total = t;
        }
        cl.sync();                                   // every CTA's total in its shared memory
        // the lower CTAs' totals, one per lane (at most 16 CTAs)
        int base = lane < (int)blockIdx.x ? *cl.map_shared_rank(&cta_total, lane) : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) base += __shfl_xor_sync(0xffffffffu, base, o);
        int e = base + x - s + (w > 0 ? wsum[w - 1] : 0);
        for (int c = lo; c < hi; ++c) {
            const int cnt = __ldcg(A.count + c);
            A.cell_start[c] = e;
            A.count[c] = 0;
            e += cnt;
        }
        if (blockIdx.x == nct - 1 && tid == 0) A.cell_start[A.nc] = base + cta_total;
    }
    cl.sync();

    // scatter the owned keys
    int lo_[ITEMS], hi_[ITEMS];
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        if (!mine[i]) continue;
        lo_[i] = __ldcg(A.cell_start + cell[i]);
        hi_[i] = __ldcg(A.cell_start + cell[i] + 1);
        A.keys[lo_[i] + rank[i]] = make_int2(wbits(p[i].w) & ID_MASK, g + i * G);
    }
    cl.sync();

    // place the owned particles
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        if (!mine[i]) continue;
        const int k = g + i * G;
        const int id = wbits(p[i].w) & ID_MASK;
        int rk = 0;
        for (int e = lo_[i]; e < hi_[i]; e += 4) {
            int kx[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) kx[u] = e + u < hi_[i] ? __ldcg(A.keys + e + u).x : id;
#pragma unroll
            for (int u = 0; u < 4; ++u) rk += kx[u] < id;
        }
        const int dst = lo_[i] + rk;
        const RepParams &P = A.reps[wbits(v[i].w)];
        float4 vtn = make_float4(v[i].x, v[i].y, v[i].z, vtw[i]);
        if (pred[i]) {
            vtn.x = __fmaf_rn(P.ldt, f[i].x, v[i].x);
            vtn.y = __fmaf_rn(P.ldt, f[i].y, v[i].y);
            vtn.z = __fmaf_rn(P.ldt, f[i].z, v[i].z);
        }
        A.nxt.pos[dst] = p[i];
        A.nxt.vel[dst] = v[i];
        A.nxt.frc[dst] = f[i];
        A.nxt.vt[dst] = vtn;
        A.inv[P.pbase + id] = dst;
        for (int sp = 0; sp < ns; ++sp) {
            float c, q;
            if constexpr (NS > 0) {
                c = cs_[i][sp];
                q = qs_[i][sp];
            } else {
                c = A.cur.C[(size_t)k * ns + sp];
                q = A.cur.Q[(size_t)k * ns + sp];
            }
            A.nxt.C[(size_t)dst * ns + sp] = c;
            A.nxt.Q[(size_t)dst * ns + sp] = q;
            A.nxt.Ct[(size_t)dst * ns + sp] = pred[i] ? __fmaf_rn(P.ldt, q, c) : c;
        }
    }
}

static inline int nblk(int n, int t) { return (n + t - 1) / t; }

void launch_bin_init(const Buffers &b, const RepParams *reps, int n, int *count, int *tile_sum,
                     int2 *cellrank, cudaStream_t st)
{
    if (n <= 0) return;
    launch_pdl(k_bin_init, nblk(n, 256), 256, st, b, reps, n, count, tile_sum, cellrank);
}

void launch_scan(int *count, int *cell_start, int n_tiles, const int *tile_read, int *tile_clear,
                 uint32_t *step_ctr, int inc, cudaStream_t st, const uint32_t *any)
{
    static_assert(SCAN_TILE == 4 * 1024, "one CTA of 1024 threads scans four cells per thread");
    launch_pdl(k_scan, n_tiles, 1024, st, count, cell_start, tile_read, tile_clear, step_ctr, inc, any);
}

void launch_scatter_keys(const Buffers &cur, const int2 *cellrank, const int *cell_start,
                         int2 *keys, int n, cudaStream_t st, const uint32_t *any, const uint32_t *rb)
{
    if (n <= 0) return;
    launch_pdl(k_scatter_keys, nblk(n, 256), 256, st, cur.pos, cur.vel, cellrank, cell_start, keys, n, any, rb);
}

void launch_rank_gather(const Buffers &cur, const Buffers &nxt, const RepParams *reps,
                        const int2 *keys, const int2 *cellrank, const int *cell_start, int *inv,
                        int n, int ns, int predict, cudaStream_t st, const uint32_t *rb, int n_rep,
                        int *tile_zero, int n_tiles, const Quarantine &q)
{
    if (n <= 0) return;
    const int g = nblk(n, 256);
    switch (ns) {
    case 1: launch_pdl(k_rank_gather<1>, g, 256, st, cur, nxt, reps, keys, cellrank, cell_start, inv, n, ns, predict, rb, n_rep, tile_zero, n_tiles, q); break;
    case 2: launch_pdl(k_rank_gather<2>, g, 256, st, cur, nxt, reps, keys, cellrank, cell_start, inv, n, ns, predict, rb, n_rep, tile_zero, n_tiles, q); break;
    default: launch_pdl(k_rank_gather<0>, g, 256, st, cur, nxt, reps, keys, cellrank, cell_start, inv, n, ns, predict, rb, n_rep, tile_zero, n_tiles, q); break;
    }
}


template <int NS>
static int sort_small_ctas_ns()
{
    auto k = k_sort_small<NS, SORT_SMALL_ITEMS>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
        cudaGetLastError();
    for (int c : {16, 8}) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(c);
        cfg.blockDim = dim3(SORT_SMALL_THREADS);
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = c;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, k, &cfg) == cudaSuccess && n >= 1) {
            // the one-item form launches with the same cluster shape
            if (cudaFuncSetAttribute(k_sort_small<NS, 1>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                cudaSuccess)
                cudaGetLastError();
            return c;
        }
        cudaGetLastError();
    }
    return 0;
}

int sort_small_ctas(int ns)
{
    switch (ns) {
    case 1: return sort_small_ctas_ns<1>();
    case 2: return sort_small_ctas_ns<2>();
    default: return sort_small_ctas_ns<0>();
    }
}

template <int NS, int ITEMS>
static void launch_sort_small_ns(const SortSmallArgs &a, int ctas, cudaStream_t st)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ctas);
    cfg.blockDim = dim3(SORT_SMALL_THREADS);
    cfg.stream = st;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = ctas;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 2;
    cudaLaunchKernelEx(&cfg, k_sort_small<NS, ITEMS>, a);
}

template <int NS>
static void launch_sort_small_items(const SortSmallArgs &a, int ctas, cudaStream_t st)
{
    if (a.n <= ctas * SORT_SMALL_THREADS) launch_sort_small_ns<NS, 1>(a, ctas, st);
    else launch_sort_small_ns<NS, SORT_SMALL_ITEMS>(a, ctas, st);
}

void launch_sort_small(const SortSmallArgs &a, int ctas, cudaStream_t st)
{
    // the caller checks the size (commit never selects a larger system)
    if (a.n <= 0 || ctas <= 0 || a.n > ctas * SORT_SMALL_THREADS * SORT_SMALL_ITEMS) return;
    switch (a.ns_rt) {
    case 1: launch_sort_small_items<1>(a, ctas, st); break;
    case 2: launch_sort_small_items<2>(a, ctas, st); break;
    default: launch_sort_small_items<0>(a, ctas, st); break;
    }
}

}  // namespace tdpd

namespace tdpd {

// Load-order state of a loaded or replaced configuration: raw x, v (3 floats
// each) and C from the upload area, with each particle's fixed bits (id and
// type, replica, membrane) from wstat; F and Q start at zero. Membrane
// vertices also go to mx, mv (load order), where the membrane kernels read them.
__global__ void k_pack_state(const float *__restrict__ x3, const float *__restrict__ v3,
                             const float *__restrict__ c, const int4 *__restrict__ wstat, Buffers b,
                             float4 *mx, float4 *mv, int n, int ns)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    const int4 w = wstat[g];
    const float vx = v3[3 * (size_t)g], vy = v3[3 * (size_t)g + 1], vz = v3[3 * (size_t)g + 2];
    const float4 p = make_float4(x3[3 * (size_t)g], x3[3 * (size_t)g + 1], x3[3 * (size_t)g + 2], __int_as_float(w.x));
    const float4 vt = make_float4(vx, vy, vz, __int_as_float(w.z));
    b.pos[g] = p;
    b.vel[g] = make_float4(vx, vy, vz, __int_as_float(w.y));
    b.vt[g] = vt;
    if (w.z >= 0) {
        mx[g] = p;
        mv[g] = vt;
    }
    b.frc[g] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int s = 0; s < ns; ++s) {
        const size_t k = (size_t)g * ns + s;
        b.C[k] = c[k];
        b.Ct[k] = c[k];
        b.Q[k] = 0.0f;
    }
}

// Load-order copy of slots [base, base + n) of the current buffer: entry i
// of the output is the particle at slot inv[base + i] (a slot outside the
// range sets *bad and is skipped).
__global__ void k_unpack_state(Buffers b, const int *__restrict__ inv, int base, int n, int ns, float *pos,
                               float *vel, float *conc, uint32_t *bad)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int k = inv[base + i];
    if (k < base || k >= base + n) {
        atomicOr(bad, 1u);
        return;
    }
    if (pos) {
        const float4 p = b.pos[k];
        pos[3 * (size_t)i] = p.x;
        pos[3 * (size_t)i + 1] = p.y;
        pos[3 * (size_t)i + 2] = p.z;
    }
    if (vel) {
        const float4 v = b.vel[k];
        vel[3 * (size_t)i] = v.x;
        vel[3 * (size_t)i + 1] = v.y;
        vel[3 * (size_t)i + 2] = v.z;
    }
    if (conc)
        for (int sp = 0; sp < ns; ++sp) conc[(size_t)i * ns + sp] = b.C[(size_t)k * ns + sp];
}

// A loaded state's validity: every position inside its replica's box and
// every velocity finite; a violation sets *bad.
__global__ void k_check_state(const float *__restrict__ x3, const float *__restrict__ v3,
                              const int4 *__restrict__ wstat, const RepParams *__restrict__ reps, int n,
                              uint32_t *bad)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const RepParams &P = reps[wstat[i].y];
    bool ok = true;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float x = x3[3 * (size_t)i + c], v = v3[3 * (size_t)i + c];
        ok = ok && x >= 0.0f && x < P.L[c] && isfinite(v);
    }
    if (!ok) atomicOr(bad, 1u);
}

void launch_unpack_state(const Buffers &b, const int *inv, int base, int n, int ns, float *pos, float *vel,
                         float *conc, uint32_t *bad, cudaStream_t st)
{
    if (n <= 0) return;
    k_unpack_state<<<(n + 255) / 256, 256, 0, st>>>(b, inv, base, n, ns, pos, vel, conc, bad);
}

void launch_check_state(const float *x3, const float *v3, const int4 *wstat, const RepParams *reps, int n,
                        uint32_t *bad, cudaStream_t st)
{
    if (n <= 0) return;
    k_check_state<<<(n + 255) / 256, 256, 0, st>>>(x3, v3, wstat, reps, n, bad);
}

void launch_pack_state(const float *in, const int4 *wstat, const Buffers &b, float4 *mx, float4 *mv, int n,
                       int ns, cudaStream_t st)
{
    if (n <= 0) return;
    k_pack_state<<<(n + 255) / 256, 256, 0, st>>>(in, in + 3 * (size_t)n, in + 6 * (size_t)n, wstat, b, mx, mv,
                                                  n, ns);
}

}  // namespace tdpd
