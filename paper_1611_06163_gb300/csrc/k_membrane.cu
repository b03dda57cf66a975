// Membrane forces of the triangulated RBC model (Sec. 2.2, Eq. 10-16).
//
// k_mem_gather (K-Gather of Sec. 3.3): one CTA per membrane sums the
//   triangle areas and signed tetrahedron volumes in FP64 with compensation,
//   the constraint coefficients they give, and the vertex centroid that
//   becomes the next step's reference point. A lagged membrane's K-Apply
//   uses the previous step's coefficients, so it need not wait for this.
// k_mem_forces (K-Apply, bonds and bending): eight lanes per vertex; lane l
//   takes the l-th entry of the vertex's one-ring fan and adds
//     - the bond (v, nb[l]): WLC + POW, viscous and random parts,
//     - the dihedral on edge (v, nb[l]) (v as an edge end),
//     - the triangle (v, nb[l], nb[l+1]): area and volume constraints,
//     - the dihedral on edge (nb[l], nb[l+1]) (v as the opposite vertex);
//   a shuffle sums the lanes. Every vertex force is written once, no atomics.
//
// Both kernels read the vertices' predicted positions and v~ from arrays in
// load order (written by the previous step's pair kernel, or by the packing of
// a loaded state) and write the force in load order, so they do not
// depend on the cell sort and run beside it.
//
// Coordinates are taken relative to a per-membrane reference point with the
// minimum image, so a membrane may straddle the periodic boundary as long as
// it spans less than half a box. K-Gather's vertex centroid is the next
// step's reference point; a loaded state's comes from k_mem_ref.
#include "launch.h"

namespace tdpd {

__device__ __forceinline__ float3 f3(float4 a) { return make_float3(a.x, a.y, a.z); }
__device__ __forceinline__ float3 sub(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 add(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 scl(float s, float3 a) { return make_float3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float dot(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross(float3 a, float3 b)
{
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

__device__ __forceinline__ float3 rel_pos(const RepParams &P, float4 x, float4 ref)
{
    return make_float3(min_image(x.x - ref.x, P.L[0], P.periodic[0]),
                       min_image(x.y - ref.y, P.L[1], P.periodic[1]),
                       min_image(x.z - ref.z, P.L[2], P.periodic[2]));
}

// Vertices of a membrane staged in shared memory by K-Gather (larger
// membranes read their triangle corners from global memory).
constexpr int GATHER_STAGE_NV = 2048;
constexpr int GATHER_THREADS = 512;
constexpr int REF_THREADS = 256;

// K-Gather: one CTA of GATHER_THREADS per membrane (512 at 64 registers: two
// CTAs per SM, twice the resident membranes of 1024-thread CTAs; 46 -> 28 us
// on the 512-replica ensemble); each thread takes two triangles and one
// vertex of a 500-vertex cell (prefetched together); the
// binary32 terms are reduced with compensated float-float sums (warp
// shuffles, then one warp over the warp totals) and converted to binary64 once.
// The triangle indices and the vertex positions are loaded together (the
// positions, relative to the reference point, into shared memory), so a cold
// start costs two dependent memory round trips, not three.
__global__ void __launch_bounds__(GATHER_THREADS, 2) k_mem_gather(MemArgs A)
{
    pdl_enter();
    const int b = blockIdx.x;
    if (b == 0 && threadIdx.x == 0) A.mem_ctr[1 - A.q] = A.mem_ctr[A.q] + 1u;   // the next evaluation's
    const RbcDev R = A.rbcs[b];
    const RepParams &P = A.reps[R.rep];
    const float4 ref = A.ref_in[b];
    const int *tri = A.tri + R.tri_off;
    __shared__ float4 xs[GATHER_STAGE_NV];
    const bool staged = R.nv <= GATHER_STAGE_NV;
    int3 pre[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int t = threadIdx.x + u * blockDim.x;
        pre[u] = t < R.ntri ? make_int3(tri[3 * t], tri[3 * t + 1], tri[3 * t + 2]) : make_int3(0, 0, 0);
    }
    FF v[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) v[k] = FF{0.0f, 0.0f};
    for (int k = threadIdx.x; k < R.nv; k += blockDim.x) {
        const float3 x = rel_pos(P, A.mx[R.gbase + k], ref);
        if (staged) xs[k] = make_float4(x.x, x.y, x.z, 0.0f);
        v[2] = ff_add(v[2], x.x);
        v[3] = ff_add(v[3], x.y);
        v[4] = ff_add(v[4], x.z);
    }
    __syncthreads();
    int u = 0;
    for (int t = threadIdx.x; t < R.ntri; t += blockDim.x, ++u) {
        const int3 tv = u == 0 ? pre[0] : u == 1 ? pre[1] : make_int3(tri[3 * t], tri[3 * t + 1], tri[3 * t + 2]);
        float3 x0, x1, x2;
        if (staged) {
            x0 = f3(xs[tv.x]);
            x1 = f3(xs[tv.y]);
            x2 = f3(xs[tv.z]);
        } else {
            x0 = rel_pos(P, A.mx[R.gbase + tv.x], ref);
            x1 = rel_pos(P, A.mx[R.gbase + tv.y], ref);
            x2 = rel_pos(P, A.mx[R.gbase + tv.z], ref);
        }
        const float3 n = cross(sub(x1, x0), sub(x2, x0));
        v[0] = ff_add(v[0], 0.5f * sqrtf(dot(n, n)));
        v[1] = ff_add(v[1], dot(x0, cross(x1, x2)) * (1.0f / 6.0f));
    }
    __shared__ FF sh[32][5];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < 5; ++k) v[k] = ff_add(v[k], ff_shfl_down(v[k], o));
    if (lane == 0)
        for (int k = 0; k < 5; ++k) sh[w][k] = v[k];
    __syncthreads();
    if (w != 0) return;
#pragma unroll
    for (int k = 0; k < 5; ++k) v[k] = lane < nw ? sh[lane][k] : FF{0.0f, 0.0f};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < 5; ++k) v[k] = ff_add(v[k], ff_shfl_down(v[k], o));
    if (lane == 0) {
        const double Ab = ff_value(v[0]), Vb = ff_value(v[1]);
        A.av_out[b] = make_double2(Ab, Vb);
        // constraint coefficients of Eq. 14-15, once per membrane in binary64
        // (divisions by A0, V0 and nv were done once on the host)
        A.cgv_out[b] = make_float2((float)((Ab - R.A0) * R.kgA0), (float)((Vb - R.V0) * R.kvV0));
        const double inv = R.inv_nv;
        float c3[3] = {(float)(ref.x + ff_value(v[2]) * inv), (float)(ref.y + ff_value(v[3]) * inv),
                       (float)(ref.z + ff_value(v[4]) * inv)};
        for (int c = 0; c < 3; ++c)
            if (P.periodic[c]) {
                if (c3[c] < 0.0f) c3[c] += P.L[c];
                else if (c3[c] >= P.L[c]) c3[c] -= P.L[c];
            }
        A.ref_out[b] = make_float4(c3[0], c3[1], c3[2], 0.0f);
    }
}

// Gradient of the angle theta between the outward normals of triangles
// (a, b, c) and (b, a, d) (positive on a convex fold). Returns sin and cos of
// theta; role selects the vertex whose gradient is written to g.
struct Dihedral {
    float sin_t, cos_t;
    float3 g;
};

__device__ __forceinline__ Dihedral dihedral(float3 xa, float3 xb, float3 xc, float3 xd, int role)
{
    const float3 e = sub(xb, xa);
    const float3 n1 = cross(e, sub(xc, xa));
    const float3 n2 = cross(sub(xa, xb), sub(xd, xb));
    const float le2 = dot(e, e), n1s = dot(n1, n1), n2s = dot(n2, n2);
    const float le = sqrtf(le2);
    const float inv12 = rsqrtf(n1s * n2s);
    Dihedral D;
    D.cos_t = dot(n1, n2) * inv12;
    D.sin_t = dot(cross(n1, n2), e) * inv12 / le;
    const float3 u1 = scl(1.0f / n1s, n1), u2 = scl(1.0f / n2s, n2);
    if (role == 0) {          // a
        const float p1 = dot(sub(xc, xb), e) / le, p2 = dot(sub(xd, xb), e) / le;
        D.g = scl(-1.0f, add(scl(p1, u1), scl(p2, u2)));
    } else {                  // c
        D.g = scl(-le, u1);
    }
    return D;
}

// Four CTAs per SM (64 registers, a few spilled to L1): faster than two or
// three on the ensemble of many membranes.
__global__ void __launch_bounds__(256, 4) k_mem_forces(MemArgs A)
{
    pdl_enter();
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) A.mem_ctr[1 - A.q] = A.mem_ctr[A.q] + 1u;
    const int b = blockIdx.y;
    const RbcDev R = A.rbcs[b];
    const int v = (blockIdx.x * blockDim.x + threadIdx.x) >> 3;
    const int lane8 = threadIdx.x & 7;
    const bool live = v < R.nv;
    const RepParams &P = A.reps[R.rep];
    float3 f = make_float3(0.f, 0.f, 0.f);
    if (live) {
        const float4 ref = A.ref_in[b];
        const float2 cgv = P.m_lagged ? A.cgv_lag[b] : A.cgv_seq[b];
        const float cg = cgv.x, cv = cgv.y;
        const FanEntry *fan = A.fan + R.fan_off + (size_t)v * R.fan_stride;
        const float3 xv = rel_pos(P, A.mx[R.gbase + v], ref);
        const float4 vv = A.mv[R.gbase + v];
        const uint32_t idv = (uint32_t)(R.gbase + v - P.pbase);
        const uint32_t step = A.mem_ctr[A.q] + P.step0;
        for (int l = lane8; l < R.fan_stride; l += 8) {
            const FanEntry E = fan[l];
            if (E.nb < 0) break;                      // past the vertex's degree
            const float3 xl = rel_pos(P, A.mx[R.gbase + E.nb], ref);
            const float3 xn = rel_pos(P, A.mx[R.gbase + E.nb_next], ref);
            const float3 xp = rel_pos(P, A.mx[R.gbase + E.nb_prev], ref);
            const float3 xw = rel_pos(P, A.mx[R.gbase + E.across], ref);

            // bond (v, nb[l]): Eq. 10-13
            {
                const float3 d = sub(xv, xl);
                const float l2 = dot(d, d);
                const float il = rsqrtf(l2);
                const float len = l2 * il;
                const float3 e = scl(il, d);
                const float2 bp = A.bond[R.bond_off + E.edge];   // (l_m, k_p)
                const float x = len / bp.x;
                const float omx = 1.0f - x;
                const float pw = P.m_m == 2.0f ? len * len : __powf(len, P.m_m);
                const float dudl = P.m_wlc0 * (0.25f / (omx * omx) - 0.25f + x) - bp.y / pw;
                f = add(f, scl(-dudl, e));
                const float4 vl = A.mv[R.gbase + E.nb];
                const float3 vij = make_float3(vv.x - vl.x, vv.y - vl.y, vv.z - vl.z);
                const float ve = dot(vij, e);
                f = add(f, add(scl(-P.m_gT, vij), scl(-P.m_gC * ve, e)));
                const uint32_t idl = (uint32_t)(R.gbase + E.nb - P.pbase);
                float z[10];
#pragma unroll
                for (int s = 0; s < 5; ++s) {
                    const float2 g = normal2(pair_bits(idv, idl, P.seed_lo, P.seed_hi, step, 1u + s));
                    z[2 * s] = g.x;
                    z[2 * s + 1] = g.y;
                }
                const float tr = z[0] + z[4] + z[8];
                // (W^S - tr/3 I) e with W^S the symmetric part of Z
                const float s01 = 0.5f * (z[1] + z[3]), s02 = 0.5f * (z[2] + z[6]), s12 = 0.5f * (z[5] + z[7]);
                const float t3 = tr * (1.0f / 3.0f);
                const float3 we = make_float3((z[0] - t3) * e.x + s01 * e.y + s02 * e.z,
                                              s01 * e.x + (z[4] - t3) * e.y + s12 * e.z,
                                              s02 * e.x + s12 * e.y + (z[8] - t3) * e.z);
                f = add(f, add(scl(P.m_rand_T, we), scl(P.m_rand_C * tr, e)));
            }
            // dihedral on edge (v, nb[l]): triangles (v, nb[l], nb[l+1]), (nb[l], v, nb[l-1])
            {
                const Dihedral D = dihedral(xv, xl, xn, xp, 0);
                const float s = P.m_kb * (D.sin_t * P.m_cos0 - D.cos_t * P.m_sin0);
                f = sub(f, scl(s, D.g));
            }
            // triangle (v, nb[l], nb[l+1]): Eq. 14-15
            {
                const float3 n = cross(sub(xl, xv), sub(xn, xv));
                const float nn = sqrtf(dot(n, n));
                const float At = 0.5f * nn;
                const float a0 = A.a0j[R.a0j_off + E.tri];
                const float ca = cg + P.m_kl * (At - a0) / a0;
                const float3 gA = scl(0.5f / nn, cross(n, sub(xn, xl)));
                const float3 gV = scl(1.0f / 6.0f, cross(xl, xn));
                f = sub(f, add(scl(ca, gA), scl(cv, gV)));
            }
            // dihedral on edge (nb[l], nb[l+1]) with v opposite: (nb[l], nb[l+1], v), (nb[l+1], nb[l], w)
            {
                const Dihedral D = dihedral(xl, xn, xv, xw, 2);
                const float s = P.m_kb * (D.sin_t * P.m_cos0 - D.cos_t * P.m_sin0);
                f = sub(f, scl(s, D.g));
            }
        }
    }
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) {
        f.x += __shfl_xor_sync(0xffffffffu, f.x, o);
        f.y += __shfl_xor_sync(0xffffffffu, f.y, o);
        f.z += __shfl_xor_sync(0xffffffffu, f.z, o);
    }
    if (live && lane8 == 0) A.fext[R.gbase + v] = make_float4(f.x, f.y, f.z, 0.0f);
}

// Reference point of each membrane of a loaded state, from the uploaded
// load-order positions x3 (three floats per particle): the centroid of its
// vertices unwrapped along the mesh's edges from vertex 0 by the minimum
// image, folded into the box. Each round, every unlabelled vertex takes its
// image offsets k (per axis) from a labelled neighbour, k_u = k_v -
// rint((p_u - p_v) / L); for a mesh whose edges are shorter than half the
// box every path gives the same k. The coordinates relative to vertex 0,
// (p_u - p_0) + k_u L, are summed with float-float compensation in a fixed
// tree (as K-Gather sums its terms) and combined with p_0 once in binary64.
// All arithmetic but that last step is binary32 (the FP64 unit of this GPU
// is narrow). One CTA per membrane; the labels in shared memory (0: not
// reached; else the three offsets, biased by 64, in the low bytes and bit
// 24 set), and with STAGED the vertices' positions and neighbours too. A
// vertex no edge reaches is left out of the sum.
template <bool STAGED>
__global__ void __launch_bounds__(REF_THREADS) k_mem_ref(const float *__restrict__ x3,
                                                         const RbcDev *__restrict__ rbcs,
                                                         const FanEntry *__restrict__ fan,
                                                         const RepParams *__restrict__ reps, float4 *ref_out,
                                                         int max_nv, int max_stride)
{
    extern __shared__ int sm[];
    __shared__ FF wsum[REF_THREADS / 32][3];
    const int b = blockIdx.x;
    const RbcDev R = rbcs[b];
    const RepParams &P = reps[R.rep];
    const int nv = R.nv, stride = R.fan_stride;
    volatile int *lab = sm;
    float *ps = reinterpret_cast<float *>(sm + max_nv);             // STAGED: [3 nv]
    int *nbs = sm + 4 * max_nv;                                     // STAGED: [nv stride]
    const float *pg = x3 + 3 * (size_t)R.gbase;
    const FanEntry *fg = fan + R.fan_off;
    constexpr int SET = 1 << 24, ZERO = 64 | 64 << 8 | 64 << 16;
    if (STAGED) {
        for (int i = threadIdx.x; i < 3 * nv; i += blockDim.x) ps[i] = pg[i];
        for (int i = threadIdx.x; i < nv * stride; i += blockDim.x) nbs[i] = fg[i].nb;
    }
    for (int u = threadIdx.x; u < nv; u += blockDim.x) lab[u] = u == 0 ? (SET | ZERO) : 0;
    __syncthreads();
    const float *p = STAGED ? ps : pg;
    bool changed;
    do {
        changed = false;
        for (int u = threadIdx.x; u < nv; u += blockDim.x) {
            if (lab[u]) continue;
            for (int l = 0; l < stride; ++l) {
                const int v = STAGED ? nbs[u * stride + l] : fg[(size_t)u * stride + l].nb;
                if (v < 0) break;
                const int lv = lab[v];
                if (!lv) continue;
                int code = SET;
                for (int c = 0; c < 3; ++c) {
                    const int k = ((lv >> (8 * c)) & 255) - 64 - (int)rintf((p[3 * u + c] - p[3 * v + c]) * P.inv_L[c]);
                    code |= (k + 64) << (8 * c);
                }
                lab[u] = code;
                changed = true;
                break;
            }
        }
    } while (__syncthreads_or(changed));
    FF acc[3] = {FF{0.0f, 0.0f}, FF{0.0f, 0.0f}, FF{0.0f, 0.0f}};
    for (int u = threadIdx.x; u < nv; u += blockDim.x) {
        const int lu = lab[u];
        if (!lu) continue;
        for (int c = 0; c < 3; ++c)
            acc[c] = ff_add(acc[c], __fmaf_rn((float)(((lu >> (8 * c)) & 255) - 64), P.L[c], p[3 * u + c] - p[c]));
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        for (int c = 0; c < 3; ++c) acc[c] = ff_add(acc[c], ff_shfl_down(acc[c], o));
    if (lane == 0)
        for (int c = 0; c < 3; ++c) wsum[w][c] = acc[c];
    __syncthreads();
    if (threadIdx.x != 0) return;
    float cf[3];
    for (int c = 0; c < 3; ++c) {
        FF t = wsum[0][c];
        for (int k = 1; k < REF_THREADS / 32; ++k) t = ff_add(t, wsum[k][c]);
        double y = (double)p[c] + ff_value(t) / (double)nv;
        if (P.periodic[c]) y -= (double)P.L[c] * floor(y / (double)P.L[c]);
        cf[c] = (float)y;
        if (!(cf[c] < P.L[c])) cf[c] = 0.0f;      // rounded up onto L
    }
    ref_out[b] = make_float4(cf[0], cf[1], cf[2], 0.0f);
}

void launch_mem_ref(const float *x3, const RbcDev *rbcs, const FanEntry *fan, const RepParams *reps, float4 *ref_out,
                    int n_rbc, int max_nv, int max_stride, cudaStream_t st)
{
    if (n_rbc <= 0) return;
    constexpr size_t SMEM_MAX = 200 * 1024;
    const size_t staged = sizeof(int) * ((size_t)4 * max_nv + (size_t)max_nv * max_stride);
    const size_t plain = sizeof(int) * (size_t)max_nv;
    if (staged <= SMEM_MAX) {
        if (staged > 48 * 1024)
            cudaFuncSetAttribute(k_mem_ref<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)staged);
        k_mem_ref<true><<<n_rbc, REF_THREADS, staged, st>>>(x3, rbcs, fan, reps, ref_out, max_nv, max_stride);
    } else {
        if (plain > 48 * 1024)
            cudaFuncSetAttribute(k_mem_ref<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plain);
        k_mem_ref<false><<<n_rbc, REF_THREADS, plain, st>>>(x3, rbcs, fan, reps, ref_out, max_nv, max_stride);
    }
}

void launch_mem_gather(const MemArgs &a, cudaStream_t st, bool pdl)
{
    if (a.n_rbc <= 0) return;
    if (pdl) launch_pdl(k_mem_gather, a.n_rbc, GATHER_THREADS, st, a);
    else k_mem_gather<<<a.n_rbc, GATHER_THREADS, 0, st>>>(a);
}

void launch_mem_forces(const MemArgs &a, cudaStream_t st)
{
    if (a.n_rbc <= 0) return;
    dim3 g((a.max_nv * 8 + 255) / 256, a.n_rbc);
    launch_pdl(k_mem_forces, g, 256, st, a);
}

}  // namespace tdpd
