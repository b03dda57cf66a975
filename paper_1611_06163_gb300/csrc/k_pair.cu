// Pairwise tDPD force (Eq. 3) and Fickian flux (Eq. 6) over the cell list,
// fused with the velocity-Verlet corrector and the binning of the next step.
//
// One thread owns one particle i (cell-sorted order) and sums its partners
// over the 27 neighbouring cells, so F_i and Q_i are written once, without
// atomics, in a fixed order. Each unordered pair is thus evaluated from both
// sides; the pair random number is keyed on (min id, max id, step) so both
// sides draw the same xi_ij and F_ij = -F_ji holds to rounding.
#include "launch.h"

namespace tdpd {

template <int NS>
__global__ void __launch_bounds__(128) k_pair(PairArgs A)
{
    const int ns = NS > 0 ? NS : A.ns;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.n) return;
    const float4 *__restrict__ pos = A.b.pos;
    const float4 *__restrict__ vt = A.b.vt;
    const float *__restrict__ Ct = A.b.Ct;
    const int *__restrict__ cs = A.cell_start;

    const float4 pi = pos[i];
    const float4 vi = vt[i];
    const float4 vo = A.b.vel[i];
    const int rep = wbits(vo.w);
    const RepParams &P = A.reps[rep];
    const uint32_t wi = (uint32_t)wbits(pi.w);
    const uint32_t idi = wi & ID_MASK;
    const int ti = (int)(wi >> 24);
    const int bi = wbits(vi.w);
    const uint32_t step = *A.step_ctr + P.step0;
    const int T = P.ntypes;

    float ci[NS > 0 ? NS : MAXS];
    float q[NS > 0 ? NS : MAXS];
    for (int s = 0; s < ns; ++s) {
        ci[s] = Ct[(size_t)i * ns + s];
        q[s] = 0.0f;
    }
    float fx = 0.f, fy = 0.f, fz = 0.f;

    const int cx = cell_coord(pi.x, P.cell_scale[0], P.nc[0]);
    const int cy = cell_coord(pi.y, P.cell_scale[1], P.nc[1]);
    const int cz = cell_coord(pi.z, P.cell_scale[2], P.nc[2]);
    const float rcut2 = P.rcut2, rc2 = P.rc2, rcc2 = P.rcc2;

    for (int dz = -1; dz <= 1; ++dz) {
        int z = cz + dz;
        float sz = 0.f;
        if (z < 0) { if (!P.periodic[2]) continue; z += P.nc[2]; sz = P.L[2]; }
        else if (z >= P.nc[2]) { if (!P.periodic[2]) continue; z -= P.nc[2]; sz = -P.L[2]; }
        for (int dy = -1; dy <= 1; ++dy) {
            int y = cy + dy;
            float sy = 0.f;
            if (y < 0) { if (!P.periodic[1]) continue; y += P.nc[1]; sy = P.L[1]; }
            else if (y >= P.nc[1]) { if (!P.periodic[1]) continue; y -= P.nc[1]; sy = -P.L[1]; }
            for (int dx = -1; dx <= 1; ++dx) {
                int x = cx + dx;
                float sx = 0.f;
                if (x < 0) { if (!P.periodic[0]) continue; x += P.nc[0]; sx = P.L[0]; }
                else if (x >= P.nc[0]) { if (!P.periodic[0]) continue; x -= P.nc[0]; sx = -P.L[0]; }
                const int c = P.cell_base + (z * P.nc[1] + y) * P.nc[0] + x;
                const int jend = cs[c + 1];
                for (int j = cs[c]; j < jend; ++j) {
                    const float4 pj = pos[j];
                    // difference first (exact for nearby coordinates), image shift after
                    const float ddx = (pi.x - pj.x) + sx;
                    const float ddy = (pi.y - pj.y) + sy;
                    const float ddz = (pi.z - pj.z) + sz;
                    const float r2 = ddx * ddx + ddy * ddy + ddz * ddz;
                    if (!(r2 < rcut2) || j == i || r2 == 0.0f) continue;
                    const uint32_t wj = (uint32_t)wbits(pj.w);
                    const int tj = (int)(wj >> 24);
                    const float rinv = rsqrtf(r2);
                    const float r = r2 * rinv;
                    if (r2 < rcc2) {
                        const float w = 1.0f - r * P.inv_rcc;
                        const float wdc = P.sc_is2 ? w * w : __powf(w, P.s_c);
                        const float *kap = P.kappa + (ti * T + tj) * ns;
                        for (int s = 0; s < ns; ++s)
                            q[s] -= kap[s] * wdc * (ci[s] - Ct[(size_t)j * ns + s]);
                    }
                    if (r2 < rc2) {
                        const float4 vj = vt[j];
                        const int bj = wbits(vj.w);
                        if (P.exclude_same_body && bi >= 0 && bi == bj) continue;
                        const float ex = ddx * rinv, ey = ddy * rinv, ez = ddz * rinv;
                        const float w = 1.0f - r * P.inv_rc;
                        const float wR = P.sR_is1 ? w : __powf(w, P.sR);
                        const float ev = ex * (vi.x - vj.x) + ey * (vi.y - vj.y) + ez * (vi.z - vj.z);
                        const float xi = normal_cos(pair_bits(idi, wj & ID_MASK, P.seed_lo, P.seed_hi, step, 0u));
                        const int tp = ti * T + tj;
                        const float f = P.a[tp] * w - P.gamma[tp] * (wR * wR) * ev +
                                        P.sigma[tp] * wR * xi * P.inv_sqrt_dt;
                        fx += f * ex;
                        fy += f * ey;
                        fz += f * ez;
                    }
                }
            }
        }
    }

    // ---- epilogue: membrane force, sources, corrector, next binning
    if (bi >= 0) {
        const float4 fm = A.fext[i];
        fx += fm.x; fy += fm.y; fz += fm.z;
    }
    const bool frozen = (P.frozen_mask >> ti) & 1u;
    if (!frozen) { fx += P.fbody[0]; fy += P.fbody[1]; fz += P.fbody[2]; }
    if (P.k_react != 0.0f && ((P.react_mask >> ti) & 1u)) {
        const float rate = P.k_react * ci[P.r_src];
        q[P.r_src] -= rate;
        q[P.r_dst] += rate;
    }
    if (!isfinite(fx) || !isfinite(fy) || !isfinite(fz)) atomicOr(A.err + rep, 1u);

    float4 vn = vo;
    float *C = A.b.C, *Q = A.b.Q;
    const float4 fo = A.b.frc[i];
    if (A.integrate && !frozen) {
        vn.x = __fmaf_rn(P.hdt, fo.x + fx, vo.x);
        vn.y = __fmaf_rn(P.hdt, fo.y + fy, vo.y);
        vn.z = __fmaf_rn(P.hdt, fo.z + fz, vo.z);
        A.b.vel[i] = vn;
        for (int s = 0; s < ns; ++s) {
            const size_t k = (size_t)i * ns + s;
            C[k] = __fmaf_rn(P.hdt, Q[k] + q[s], C[k]);
        }
    }
    const float4 fn = make_float4(fx, fy, fz, 0.0f);
    A.b.frc[i] = fn;
    for (int s = 0; s < ns; ++s) Q[(size_t)i * ns + s] = q[s];

    float3 rn = make_float3(pi.x, pi.y, pi.z);
    if (!frozen) {
        bool flip;
        rn = predict_pos(P, pi, vn, fn, flip);
    }
    const int cell = cell_of(P, rn.x, rn.y, rn.z);
    const int rank = atomicAdd(A.count + cell, 1);
    A.cellrank[i] = make_int2(cell, rank);
}

void launch_pair(const PairArgs &a, cudaStream_t st)
{
    if (a.n <= 0) return;
    const int t = 128, g = (a.n + t - 1) / t;
    switch (a.ns) {
    case 1: k_pair<1><<<g, t, 0, st>>>(a); break;
    case 2: k_pair<2><<<g, t, 0, st>>>(a); break;
    default: k_pair<0><<<g, t, 0, st>>>(a); break;
    }
}

}  // namespace tdpd
