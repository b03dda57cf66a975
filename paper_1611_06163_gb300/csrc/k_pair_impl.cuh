// The pair kernels (included by k_pair.cu and k_pair_std.cu, which
// instantiate them).
//
// Pairwise tDPD force (Eq. 3) and Fickian flux (Eq. 6), fused with the
// velocity-Verlet corrector. Two ways to find the partners:
//   - cell mode: over the cell stencil, every step; the epilogue also bins
//     the next predicted position for the next step's sort;
//   - list mode: over the lane's Verlet list (k_list.cu), separations by
//     minimum image; the epilogue records how far the next position has moved
//     from the list build instead of binning. On a rebuild step the one- and
//     two-species forms first build the lane's own list (list_lane.cuh).
//
// Layout of the work in cell mode:
//   - cells have edge >= rcut/m, so the partners of particle i lie in the
//     (2m+1)^2 rows (dy, dz) of 2m+1 cells along x around its cell; a row is
//     one contiguous range of the cell-sorted arrays (two at a periodic wrap);
//   - LPP lanes share particle i and split its rows (lane s takes rows
//     s, s+LPP, ...); a butterfly of shuffles sums their partial results in a
//     fixed order, so small systems still fill the GPU;
//   - (list mode: lane s holds the partners found in those rows at build)
//   - the flux (about a quarter of the candidates) is summed inline by the
//     lane that found it; the force pairs (a few per cent of the candidates,
//     each needing a TEA draw) are pushed to a per-warp queue and evaluated
//     32 at a time with every lane busy. Each owner adds its
//     pairs' forces one by one in push order (that is, candidate order), so
//     the sums do not depend on how particles are grouped into warps.
// In cell mode and with full-shell lists every unordered pair is evaluated
// from both sides; the random number is keyed on (min id, max id, step), so
// both sides draw the same xi_ij. With half-shell lists each pair is
// evaluated once and the partner's share goes to fixed-point accumulators
// (k_pair_finish completes the sums).
#pragma once

#include "launch.h"
#include "list_lane.cuh"

namespace tdpd {

namespace {

// The force pairs are queued per warp and evaluated DRAIN_W x 32 at a time,
// DRAIN_W per lane (two per lane, which interleaves two TEA chains, measured
// 1 % slower on the ensemble and the 786k fluid: the dependent latency of one
// chain is already hidden by the other warps). The ring holds one drain plus
// a push (32).
constexpr int DRAIN_W = 1;
constexpr int QCAP = 64;
constexpr int UNR = 2;       // candidates loaded per trip of a stencil row (cell mode)
constexpr int UNR_LIST = 2;  // list entries per trip (list mode; fetched a trip ahead)

struct __align__(16) QEntry {
    int j;          // partner slot
    uint32_t wj;    // partner id | type << 24
    int owner;      // lane that owns particle i
    int pad;
    float dx, dy, dz, r2;
};

struct LaneInfo {
    float4 vt;      // v~_i, w = bits(body)
    uint32_t wi;    // id | type << 24
    int rep;
};

static_assert(QCAP >= 32 * DRAIN_W + 32 && (QCAP & (QCAP - 1)) == 0, "queue ring");

struct WarpSmem {
    QEntry q[QCAP];
    float4 res[32 * DRAIN_W];
    float4 acc[32];
    LaneInfo li[32];
};

// Force on the owner from one queued pair (zero if the pair is excluded).
// STD: every replica has s_f = 2 (w_R = w_D^(1/2) = w) and s_c = 2, known at
// compile time.
template <bool STD>
__device__ __forceinline__ float3 pair_force(const RepParams &P, const LaneInfo &I, const QEntry &E,
                                             const float4 *__restrict__ vt, uint32_t step_ctr)
{
    const float4 vj = vt[E.j];
    const int bi = wbits(I.vt.w), bj = wbits(vj.w);
    if (P.exclude_same_body && bi >= 0 && bi == bj) return make_float3(0.f, 0.f, 0.f);
    const float rinv = rsqrtf(E.r2);
    const float r = E.r2 * rinv;
    const float ex = E.dx * rinv, ey = E.dy * rinv, ez = E.dz * rinv;
    const float w = 1.0f - r * P.inv_rc;
    const float wR = (STD || P.sR_is1) ? w : __powf(w, P.sR);
    const float ev = ex * (I.vt.x - vj.x) + ey * (I.vt.y - vj.y) + ez * (I.vt.z - vj.z);
    const uint32_t step = step_ctr + P.step0;
    const float xi = normal_cos(pair_bits(I.wi & ID_MASK, E.wj & ID_MASK, P.seed_lo, P.seed_hi, step, 0u));
    const int T = P.ntypes;
    const int tp = (int)(I.wi >> 24) * T + (int)(E.wj >> 24);
    const float f = P.a[tp] * w - P.gamma[tp] * (wR * wR) * ev + P.sigma[tp] * wR * xi * P.inv_sqrt_dt;
    return make_float3(f * ex, f * ey, f * ez);
}

// Evaluate queue entries [head, head+n) (n <= 32 DRAIN_W; lane l takes the
// entries l, l + 32, ...) and add each result to its owner's accumulator in
// push order; HALF: the partner's share (-f) goes to its fixed-point
// accumulator.
template <bool HALF, bool STD>
__device__ __forceinline__ void drain(WarpSmem &W, int head, int n, const RepParams *__restrict__ reps,
                                      const float4 *__restrict__ vt, uint32_t step_ctr, int lane,
                                      long long *accF, uint32_t *err)
{
    int owner[DRAIN_W];
#pragma unroll
    for (int u = 0; u < DRAIN_W; ++u) {
        const int e = 32 * u + lane;
        owner[u] = 32 + lane;
        if (e < n) {
            const QEntry E = W.q[(head + e) & (QCAP - 1)];
            owner[u] = E.owner;
            const LaneInfo I = W.li[E.owner];
            const float3 f = pair_force<STD>(reps[I.rep], I, E, vt, step_ctr);
            W.res[e] = make_float4(f.x, f.y, f.z, 0.f);
            if (HALF) {
                long long *a = accF + 4 * (size_t)E.j;
                acc_add(a, -f.x, ACC_F_SCALE, ACC_F_LIMIT, err + I.rep);
                acc_add(a + 1, -f.y, ACC_F_SCALE, ACC_F_LIMIT, err + I.rep);
                acc_add(a + 2, -f.z, ACC_F_SCALE, ACC_F_LIMIT, err + I.rep);
            }
        }
    }
    __syncwarp();
#pragma unroll
    for (int u = 0; u < DRAIN_W; ++u) {
        const int e = 32 * u + lane;
        const unsigned same = __match_any_sync(0xffffffffu, owner[u]);
        if (e < n && lane == __ffs(same) - 1) {
            float4 a = W.acc[owner[u]];
            for (unsigned m = same; m; m &= m - 1) {
                const float4 r = W.res[32 * u + __ffs(m) - 1];
                a.x += r.x;
                a.y += r.y;
                a.z += r.z;
            }
            W.acc[owner[u]] = a;
        }
        __syncwarp();
    }
}

// The epilogue of particle i (slot i, lane 0 of its LPP lanes) once its
// pair force (fx, fy, fz) and flux q are complete: membrane and body force,
// reaction source, non-finite check, corrector, the predicted position of
// the next step (written for membrane vertices), and either its displacement
// from the list build (LIST) or its next binning (cell mode).
template <int NS, bool LIST>
__device__ __forceinline__ void epilogue(const PairArgs &A, const RepParams &P, int i, float4 pi, float4 vi,
                                         float4 vo, uint32_t wi, int rep, float fx, float fy, float fz,
                                         float *q, int &cell, float &disp2)
{
    const int ns = NS > 0 ? NS : A.ns;
    const int ti = (int)(wi >> 24);
    const int bi = wbits(vi.w);
    const int gi = P.pbase + (int)(wi & ID_MASK);     // load index
    float *C = A.b.C, *Q = A.b.Q;
    // every load before the first store, so that they are in flight together
    const float4 fm = bi >= 0 ? A.fext[gi] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 fo = A.b.frc[i];
    const float4 xb = LIST ? A.xb[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    const bool reacts = P.k_react != 0.0f && ((P.react_mask >> ti) & 1u);
    const float c_src = reacts ? A.b.Ct[(size_t)i * ns + P.r_src] : 0.0f;
    float c_old[NS > 0 ? NS : MAXS], q_old[NS > 0 ? NS : MAXS];
    for (int s = 0; s < ns; ++s) {
        c_old[s] = C[(size_t)i * ns + s];
        q_old[s] = Q[(size_t)i * ns + s];
    }
    fx += fm.x; fy += fm.y; fz += fm.z;
    const bool frozen = (P.frozen_mask >> ti) & 1u;
    if (!frozen) {
        const float sg = (P.fbody_flip && pi.z >= 0.5f * P.L[2]) ? -1.0f : 1.0f;
        fx += sg * P.fbody[0];
        fy += sg * P.fbody[1];
        fz += sg * P.fbody[2];
    }
    if (reacts) {
        const float rate = P.k_react * c_src;
        for (int s = 0; s < ns; ++s) {
            if (s == P.r_src) q[s] -= rate;
            if (s == P.r_dst) q[s] += rate;
        }
    }
    if (!isfinite(fx) || !isfinite(fy) || !isfinite(fz)) atomicOr(A.err + rep, 1u);

    float4 vn = vo;
    const bool moves = A.integrate && !frozen;
    if (moves) {
        vn.x = __fmaf_rn(P.hdt, fo.x + fx, vo.x);
        vn.y = __fmaf_rn(P.hdt, fo.y + fy, vo.y);
        vn.z = __fmaf_rn(P.hdt, fo.z + fz, vo.z);
        A.b.vel[i] = vn;
        for (int s = 0; s < ns; ++s) {
            c_old[s] = __fmaf_rn(P.hdt, q_old[s] + q[s], c_old[s]);    // now C_{k+1}
            C[(size_t)i * ns + s] = c_old[s];
        }
    }
    const float4 fn = make_float4(fx, fy, fz, 0.0f);
    A.b.frc[i] = fn;
    for (int s = 0; s < ns; ++s) Q[(size_t)i * ns + s] = q[s];

    float3 rn = make_float3(pi.x, pi.y, pi.z);
    float4 vtn = vn;
    bool flip = false;
    if (!frozen) {
        rn = predict_pos(P, pi, vn, fn, flip);
        if (flip) { vtn.x = -vtn.x; vtn.y = -vtn.y; vtn.z = -vtn.z; }
        vtn.x = __fmaf_rn(P.ldt, fn.x, vtn.x);
        vtn.y = __fmaf_rn(P.ldt, fn.y, vtn.y);
        vtn.z = __fmaf_rn(P.ldt, fn.z, vtn.z);
    }
    if constexpr (LIST) {
        if (A.pre.pos) {
            // the next step's predicted state at this slot, in the other
            // buffer: the same values the gather's predictor would write (a
            // wall bounce reverses the stored velocity too)
            const Buffers &O = A.pre;
            const float sv = flip ? -1.0f : 1.0f;
            O.pos[i] = make_float4(rn.x, rn.y, rn.z, pi.w);
            O.vel[i] = make_float4(sv * vn.x, sv * vn.y, sv * vn.z, vo.w);
            O.frc[i] = fn;
            O.vt[i] = make_float4(vtn.x, vtn.y, vtn.z, vi.w);
            for (int s = 0; s < ns; ++s) {
                const size_t k = (size_t)i * ns + s;
                O.C[k] = c_old[s];
                O.Q[k] = q[s];
                O.Ct[k] = frozen ? c_old[s] : __fmaf_rn(P.ldt, q[s], c_old[s]);
            }
        }
    }
    if (bi >= 0) {
        // the next step's membrane kernels start from these (the same
        // arithmetic as the predictor of the gather), before the sort
        A.mx[gi] = make_float4(rn.x, rn.y, rn.z, 0.0f);
        A.mv[gi] = vtn;
    }
    if constexpr (LIST) {
        // displacement of the next position from the list build
        float ex = rn.x - xb.x, ey = rn.y - xb.y, ez = rn.z - xb.z;
        ex = __fmaf_rn(-P.L[0], rintf(ex * P.inv_L[0]), ex);
        ey = __fmaf_rn(-P.L[1], rintf(ey * P.inv_L[1]), ey);
        ez = __fmaf_rn(-P.L[2], rintf(ez * P.inv_L[2]), ez);
        disp2 = ex * ex + ey * ey + ez * ez;
    } else {
        cell = cell_of(P, rn.x, rn.y, rn.z);
        const int rank = atomicAdd(A.count + cell, 1);
        A.cellrank[i] = make_int2(cell, rank);
    }
}

// Largest squared displacement per replica (non-negative floats order like
// their bit patterns); one atomic per warp when the warp holds one replica.
// Every lane of the warp calls it; mine: this lane reports disp2.
__device__ __forceinline__ void record_displacement(uint32_t *disp_next, int rep, float disp2, bool mine, int lane)
{
    const uint32_t bits = __float_as_uint(disp2);
    const int rep0 = __shfl_sync(0xffffffffu, rep, 0);
    if (__all_sync(0xffffffffu, rep == rep0)) {
        const uint32_t mx = __reduce_max_sync(0xffffffffu, bits);
        if (lane == 0) atomicMax(disp_next + rep0, mx);
    } else if (mine) {
        atomicMax(disp_next + rep, bits);
    }
}

}  // namespace

template <int NS, int LPP, bool LIST, bool HALF, bool STD>
__global__ void __launch_bounds__(128, 6) k_pair(PairArgs A)
{
    static_assert(LIST || !HALF, "the half shell needs neighbour lists");
    pdl_enter();
    __shared__ WarpSmem smem[4];
    const int ns = NS > 0 ? NS : A.ns;
    const int lane = threadIdx.x & 31;
    WarpSmem &W = smem[threadIdx.x >> 5];
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = gt / LPP;
    const int sub = gt % LPP;
    const bool valid = i < A.n;
    const float4 *__restrict__ pos = A.b.pos;
    const float4 *__restrict__ vt = A.b.vt;
    const float *__restrict__ Ct = A.b.Ct;
    const int *__restrict__ cs = A.cell_start;
    const uint32_t step_ctr = *A.step_ctr;

    const int ic = valid ? i : 0;
    const float4 pi = pos[ic];
    const float4 vi = vt[ic];
    const float4 vo = A.b.vel[ic];
    const int rep = wbits(vo.w);
    const RepParams &P = A.reps[rep];
    // a quarantined replica (a non-finite force or an overflowed list in an
    // earlier evaluation) is neither evaluated nor moved; its particles keep
    // their slots and, in cell mode, are binned where they are
    const bool held = valid && A.quar && A.quar[rep] != 0u;
    const bool live = valid && !held;
    const uint32_t wi = (uint32_t)wbits(pi.w);
    const int ti = (int)(wi >> 24);
    const int T = P.ntypes;

    W.li[lane].vt = vi;
    W.li[lane].wi = wi;
    W.li[lane].rep = rep;
    W.acc[lane] = make_float4(0.f, 0.f, 0.f, 0.f);

    float ci[NS > 0 ? NS : MAXS];
    float q[NS > 0 ? NS : MAXS];
    for (int s = 0; s < ns; ++s) {
        ci[s] = Ct[(size_t)ic * ns + s];
        q[s] = 0.0f;
    }

    const int m = P.m_stencil;
    const int width = 2 * m + 1;
    const int nrow = width * width;
    const int cx = cell_coord(pi.x, P.cell_scale[0], P.nc[0]);
    const int cy = cell_coord(pi.y, P.cell_scale[1], P.nc[1]);
    const int cz = cell_coord(pi.z, P.cell_scale[2], P.nc[2]);
    const float rcut2 = P.rcut2, rc2 = P.rc2, rcc2 = P.rcc2, inv_rcc = P.inv_rcc;
    const bool sc2 = STD || P.sc_is2;
    const float s_c = P.s_c;
    const float *kap_row = P.kappa + ti * T * ns;
    // one species: the kappa row of type ti in registers
    float kr[MAXT] = {0.f, 0.f, 0.f, 0.f};
    if (NS == 1)
        for (int t = 0; t < T; ++t) kr[t] = kap_row[t];
    // offsets of particle i inside its own cell, for trimming the rows
    const float hx = P.h[0], hy = P.h[1], hz = P.h[2];
    const float oy = pi.y - (float)cy * hy, oz = pi.z - (float)cz * hz;
    const float eps = 1e-4f * fmaxf(hx, fmaxf(hy, hz));
    const float rtrim2 = rcut2 * 1.0002f;

    __syncwarp();
    int qhead = 0, qcount = 0;
    // one candidate j at separation (dx, dy, dz) from i, with its id/type
    // bits wj and first concentration cj0 loaded
    auto consider = [&](bool in_range, int j, float dx, float dy, float dz, uint32_t wj, float cj0) {
        const float r2 = dx * dx + dy * dy + dz * dz;
        const bool near = in_range && r2 > 0.0f;
        // flux without a branch: the terms of candidates outside r_cc (or of
        // dead lanes) are computed and dropped by the select
        const bool inc = near && r2 < rcc2;
        const float r = r2 * rsqrtf(r2);
        const float w = 1.0f - r * inv_rcc;
        const float wdc = sc2 ? w * w : __powf(w, s_c);
        const int tj = (int)(wj >> 24);
        if (NS == 1) {
            float kap = kr[0];
            kap = tj == 1 ? kr[1] : kap;
            kap = tj == 2 ? kr[2] : kap;
            kap = tj == 3 ? kr[3] : kap;
            const float qd = kap * wdc * (ci[0] - cj0);
            const float qn = q[0] - qd;
            q[0] = inc ? qn : q[0];
            if (HALF && inc) acc_add(A.accQ + j, qd, ACC_Q_SCALE, ACC_Q_LIMIT, A.err + rep);
        } else if (inc) {
            const float *kap = kap_row + tj * ns;
            const float qd0 = kap[0] * wdc * (ci[0] - cj0);
            q[0] -= qd0;
            if (HALF) acc_add(A.accQ + (size_t)j * ns, qd0, ACC_Q_SCALE, ACC_Q_LIMIT, A.err + rep);
            for (int s = 1; s < ns; ++s) {
                const float qd = kap[s] * wdc * (ci[s] - Ct[(size_t)j * ns + s]);
                q[s] -= qd;
                if (HALF) acc_add(A.accQ + (size_t)j * ns + s, qd, ACC_Q_SCALE, ACC_Q_LIMIT, A.err + rep);
            }
            if (NS == 0 && P.qr_coef > 0.0f) {
                // random flux (Eq. 7): eps w_RC zeta / sqrt(dt), eps^2 =
                // m_s^2 kappa rho (C_i + C_j), w_RC = w_DC^(1/2) (Eq. 8); one
                // pair normal per species (the (cos, sin) pair of stream
                // 6 + s/2), signed by the id order so that zeta_ji = -zeta_ij
                const uint32_t idi = wi & ID_MASK, idj = wj & ID_MASK;
                const float amp = (idi < idj ? 1.0f : -1.0f) * P.qr_coef * sqrtf(wdc) * P.inv_sqrt_dt;
                float2 z = make_float2(0.f, 0.f);
                for (int s = 0; s < ns; ++s) {
                    if ((s & 1) == 0)
                        z = normal2(pair_bits(idi, idj, P.seed_lo, P.seed_hi, step_ctr + P.step0, 6u + (uint32_t)(s >> 1)));
                    const float cs = ci[s] + (s == 0 ? cj0 : Ct[(size_t)j * ns + s]);
                    const float qr = amp * sqrtf(fmaxf(kap[s] * cs, 0.0f)) * ((s & 1) ? z.y : z.x);
                    q[s] += qr;
                    if (HALF) acc_add(A.accQ + (size_t)j * ns + s, -qr, ACC_Q_SCALE, ACC_Q_LIMIT, A.err + rep);
                }
            }
        }
        const bool push = near && r2 < rc2;
        const unsigned bal = __ballot_sync(0xffffffffu, push);
        if (push) {
            const int slot = (qhead + qcount + __popc(bal & ((1u << lane) - 1u))) & (QCAP - 1);
            int4 *e = reinterpret_cast<int4 *>(&W.q[slot]);
            e[0] = make_int4(j, (int)wj, lane, 0);
            e[1] = make_int4(__float_as_int(dx), __float_as_int(dy), __float_as_int(dz), __float_as_int(r2));
        }
        qcount += __popc(bal);
        if (qcount >= 32 * DRAIN_W) {
            __syncwarp();
            drain<HALF, STD>(W, qhead, 32 * DRAIN_W, A.reps, vt, step_ctr, lane, A.accF, A.err);
            qhead = (qhead + 32 * DRAIN_W) & (QCAP - 1);
            qcount -= 32 * DRAIN_W;
        }
    };
    if constexpr (LIST) {
        // the lane's list, UNR_LIST entries per trip (index loads, then partner
        // loads, then the visits in list order); separations by minimum image
        if constexpr (NS == 1 || NS == 2) {
            // rebuild step: this lane's list first (the lists are only ever
            // read by the lane that owns them, so no other thread waits);
            // the kernels for more species keep the separate list build
            // (the build's registers would cost them more than the launch)
            if (A.rb && live && A.rb[rep]) {
                ListArgs L{};
                L.pos = pos; L.vel = A.b.vel; L.reps = A.reps; L.cell_start = A.cell_start; L.rb = A.rb;
                L.nl = A.nl_w; L.nlc = A.nlc_w; L.xb = A.xb_w; L.err = A.err; L.n = A.n; L.lpp = LPP; L.cap = A.cap;
                if (A.m2) build_lane<LPP, 2, HALF>(L, gt, i, sub, pi, rep);
                else build_lane<LPP, 0, HALF>(L, gt, i, sub, pi, rep);
            }
        }
        // (plain loads: on a rebuild step this thread has just written them)
        const int *nl = A.nl + (size_t)(gt >> 5) * A.cap * 32 + (gt & 31);
        const int cnt = live ? A.nlc[gt] : 0;
        const int nit = __reduce_max_sync(0xffffffffu, cnt);
        const float Lx = P.L[0], Ly = P.L[1], Lz = P.L[2];
        const float iLx = P.inv_L[0], iLy = P.inv_L[1], iLz = P.inv_L[2];
        // software pipeline: a trip's partners are fetched one trip ahead
        // and its indices two trips ahead, so the visits of a trip overlap
        // the loads of the next one
        int jj[UNR_LIST], jn[UNR_LIST];
        float4 pp[UNR_LIST];
        float cc[UNR_LIST];
#pragma unroll
        for (int u = 0; u < UNR_LIST; ++u) jj[u] = u < cnt ? nl[(size_t)u * 32] : 0;
#pragma unroll
        for (int u = 0; u < UNR_LIST; ++u) {
            pp[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            cc[u] = 0.f;
            if (u < cnt) {
                pp[u] = pos[jj[u]];
                cc[u] = Ct[(size_t)jj[u] * ns];
            }
        }
#pragma unroll
        for (int u = 0; u < UNR_LIST; ++u) jn[u] = UNR_LIST + u < cnt ? nl[(size_t)(UNR_LIST + u) * 32] : 0;
        // (a slot beyond the lane's list keeps an earlier partner's values;
        // its visit is masked by in_range)
        int jq[UNR_LIST];
        float4 pq[UNR_LIST];
        float cq[UNR_LIST];
#pragma unroll
        for (int u = 0; u < UNR_LIST; ++u) {
            pq[u] = pp[u];
            cq[u] = cc[u];
        }
        for (int t = 0; t < nit; t += UNR_LIST) {
#pragma unroll
            for (int u = 0; u < UNR_LIST; ++u) {
                jq[u] = jn[u];
                if (t + UNR_LIST + u < cnt) {
                    pq[u] = pos[jq[u]];
                    cq[u] = Ct[(size_t)jq[u] * ns];
                }
            }
#pragma unroll
            for (int u = 0; u < UNR_LIST; ++u)
                jn[u] = t + 2 * UNR_LIST + u < cnt ? nl[(size_t)(t + 2 * UNR_LIST + u) * 32] : 0;
#pragma unroll
            for (int u = 0; u < UNR_LIST; ++u)
                if (u == 0 || t + u < nit) {
                    float dx = pi.x - pp[u].x, dy = pi.y - pp[u].y, dz = pi.z - pp[u].z;
                    dx = __fmaf_rn(-Lx, rintf(dx * iLx), dx);
                    dy = __fmaf_rn(-Ly, rintf(dy * iLy), dy);
                    dz = __fmaf_rn(-Lz, rintf(dz * iLz), dz);
                    consider(t + u < cnt, jj[u], dx, dy, dz, (uint32_t)wbits(pp[u].w), cc[u]);
                }
#pragma unroll
            for (int u = 0; u < UNR_LIST; ++u) {
                jj[u] = jq[u];
                pp[u] = pq[u];
                cc[u] = cq[u];
            }
        }
    } else {
        // rows are split round-robin over the LPP lanes of the particle; the
        // loop trip counts are warp-uniform (maxima over the warp)
        const int kmax = (nrow + LPP - 1) / LPP;
        const int kw = __reduce_max_sync(0xffffffffu, live ? kmax : 0);
        for (int k = 0; k < kw; ++k) {
            const int row = sub + k * LPP;
            RowSeg g = {{0, 0}, {0, 0}, 0.f, 0.f, 0.f};
            if (live && row < nrow) stencil_row(P, cs, pi, cx, cy, cz, row, oy, oz, eps, rtrim2, g);
            const float py = pi.y + g.sy, pz = pi.z + g.sz;
#pragma unroll
            for (int sg = 0; sg < 2; ++sg) {
                const float px = pi.x + (sg ? g.sx1 : 0.f);
                const int j0 = g.jb[sg];
                const int len = g.je[sg] - j0;
                const int nit = __reduce_max_sync(0xffffffffu, len);
                // UNR candidates per trip: their loads are all in flight
                // before the first is used; the visits keep the order of t,
                // so each lane's queue entries come in the same order as one
                // per trip
                for (int t = 0; t < nit; t += UNR) {
                    float4 pp[UNR];
                    float cc[UNR];
#pragma unroll
                    for (int u = 0; u < UNR; ++u) {
                        pp[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                        cc[u] = 0.f;
                        if (t + u < len) {
                            pp[u] = pos[j0 + t + u];
                            cc[u] = Ct[(size_t)(j0 + t + u) * ns];
                        }
                    }
#pragma unroll
                    for (int u = 0; u < UNR; ++u)
                        if (u == 0 || t + u < nit)
                            consider(t + u < len, j0 + t + u, px - pp[u].x, py - pp[u].y, pz - pp[u].z,
                                     (uint32_t)wbits(pp[u].w), cc[u]);
                }
            }
        }
    }
    if (qcount > 0) {
        __syncwarp();
        drain<HALF, STD>(W, qhead, qcount, A.reps, vt, step_ctr, lane, A.accF, A.err);
    }
    __syncwarp();
    const float4 fa = W.acc[lane];
    float fx = fa.x, fy = fa.y, fz = fa.z;
    // sum the LPP lanes of the particle (butterfly: every lane gets the total)
#pragma unroll
    for (int o = LPP / 2; o > 0; o >>= 1) {
        fx += __shfl_xor_sync(0xffffffffu, fx, o);
        fy += __shfl_xor_sync(0xffffffffu, fy, o);
        fz += __shfl_xor_sync(0xffffffffu, fz, o);
        for (int s = 0; s < ns; ++s) q[s] += __shfl_xor_sync(0xffffffffu, q[s], o);
    }
    int cell = -1;
    float disp2 = 0.0f;
    if constexpr (!LIST) {
        if (held && sub == 0) {
            cell = cell_of(P, pi.x, pi.y, pi.z);
            const int rank = atomicAdd(A.count + cell, 1);
            A.cellrank[i] = make_int2(cell, rank);
        }
    }
    if (live && sub == 0) {
        if constexpr (HALF) {
            // the own sums; k_pair_finish adds the partners' shares and
            // applies the epilogue
            A.fown[i] = make_float4(fx, fy, fz, 0.0f);
            for (int s = 0; s < ns; ++s) A.qown[(size_t)i * ns + s] = q[s];
        } else {
            epilogue<NS, LIST>(A, P, i, pi, vi, vo, wi, rep, fx, fy, fz, q, cell, disp2);
        }
    }
    if constexpr (HALF) {
    } else if constexpr (LIST) {
        record_displacement(A.disp_next, rep, disp2, valid && sub == 0, lane);
    } else {
        add_tile_count(A.tile_sum, cell);
    }
}

// Half-shell list mode, after k_pair: each particle's force and flux are its
// own sums plus the partners' shares from the fixed-point accumulators (exact
// integer sums, converted once); the accumulators are cleared for the next
// evaluation and the epilogue follows. One thread per particle.
template <int NS>
__global__ void __launch_bounds__(256) k_pair_finish(PairArgs A)
{
    pdl_enter();
    const int ns = NS > 0 ? NS : A.ns;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const bool valid = i < A.n;
    const int ic = valid ? i : 0;
    // the particle's inputs first (independent loads, all in flight together)
    const float4 vo = A.b.vel[ic];
    const float4 pi = A.b.pos[ic];
    const float4 vi = A.b.vt[ic];
    const float4 fo = A.fown[ic];
    long long *af = A.accF + 4 * (size_t)ic;
    const longlong2 a01 = *reinterpret_cast<const longlong2 *>(af);
    const long long a2 = af[2];
    float q[NS > 0 ? NS : MAXS];
    long long aq[NS > 0 ? NS : MAXS];
    for (int s = 0; s < ns; ++s) {
        q[s] = A.qown[(size_t)ic * ns + s];
        aq[s] = A.accQ[(size_t)ic * ns + s];
    }
    const int rep = wbits(vo.w);
    float disp2 = 0.0f;
    if (valid) {
        const RepParams &P = A.reps[rep];
        for (int s = 0; s < ns; ++s) q[s] += __ll2float_rn(aq[s]) * ACC_Q_UNIT;
        if (!(A.quar && A.quar[rep] != 0u)) {
            const float fx = fo.x + __ll2float_rn(a01.x) * ACC_F_UNIT;
            const float fy = fo.y + __ll2float_rn(a01.y) * ACC_F_UNIT;
            const float fz = fo.z + __ll2float_rn(a2) * ACC_F_UNIT;
            int cell = -1;
            epilogue<NS, true>(A, P, i, pi, vi, vo, (uint32_t)wbits(pi.w), rep, fx, fy, fz, q, cell, disp2);
        }
        // cleared for the next evaluation
        *reinterpret_cast<longlong2 *>(af) = make_longlong2(0, 0);
        af[2] = 0;
        for (int s = 0; s < ns; ++s) A.accQ[(size_t)i * ns + s] = 0;
    }
    record_displacement(A.disp_next, rep, disp2, valid, lane);
}

// the half shell's finishing pass (k_pair_finish, instantiated once in
// k_pair.cu)
void launch_pair_finish(const PairArgs &a, cudaStream_t st);
// the pair kernels with the standard exponents (k_pair_std.cu; one or two
// species, no random flux)
void launch_pair_std(const PairArgs &a, cudaStream_t st, int part);

template <int NS, bool LIST, bool HALF, bool STD>
static void launch_lanes(const PairArgs &a, cudaStream_t st)
{
    const int t = 128;
    const long threads = (long)a.n * a.lpp;
    const int g = (int)((threads + t - 1) / t);
    switch (a.lpp) {
    case 1: launch_pdl(k_pair<NS, 1, LIST, HALF, STD>, g, t, st, a); break;
    case 2: launch_pdl(k_pair<NS, 2, LIST, HALF, STD>, g, t, st, a); break;
    case 4: launch_pdl(k_pair<NS, 4, LIST, HALF, STD>, g, t, st, a); break;
    case 8: launch_pdl(k_pair<NS, 8, LIST, HALF, STD>, g, t, st, a); break;
    case 16: launch_pdl(k_pair<NS, 16, LIST, HALF, STD>, g, t, st, a); break;
    default: launch_pdl(k_pair<NS, 32, LIST, HALF, STD>, g, t, st, a); break;
    }
}

template <int NS, bool LIST, bool STD>
static void launch_ns(const PairArgs &a, cudaStream_t st, int part)
{
    if constexpr (LIST) {
        if (a.half) {
            if (part & PAIR_WALK) launch_lanes<NS, true, true, STD>(a, st);
            if (part & PAIR_FINISH) launch_pair_finish(a, st);
            return;
        }
    }
    if (part & PAIR_WALK) launch_lanes<NS, LIST, false, STD>(a, st);
}

}  // namespace tdpd
