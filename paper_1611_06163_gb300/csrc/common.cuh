// Device data layout and small device helpers shared by the tDPD kernels.
//
// Storage (all replicas concatenated, replica-major, cell-sorted):
//   pos  float4[N]  x, y, z, w = bits(id | type << 24)      predicted r_{k+1}
//   vt   float4[N]  predicted velocity v~, w = bits(body)   (-1: free particle)
//   vel  float4[N]  velocity v_k, w = bits(replica)
//   frc  float4[N]  force F_k (pair + membrane + body force)
//   C, Ct, Q        float[N * NS] concentration, predicted concentration, flux
// Two copies of every array alternate between steps (sorted gather A -> B).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "tdpd.h"

namespace tdpd {

constexpr int MAXT = TDPD_MAX_TYPES;
constexpr int MAXS = TDPD_MAX_SPECIES;
constexpr uint32_t ID_MASK = 0x00FFFFFFu;
constexpr int SCAN_TILE_LOG2 = 12;            // 4096 cells per scan tile
constexpr int SCAN_TILE = 1 << SCAN_TILE_LOG2;

// Per-replica constants, read through the read-only path.
struct RepParams {
    float L[3];
    float cell_scale[3];     // cells per unit length (nc / L)
    float h[3];              // cell edge (L / nc)
    int nc[3];
    int periodic[3];
    int cell_base, n_cells;  // global cell index range of the replica
    int m_stencil;           // cells have edge >= rcut / m_stencil
    int pbase, n;            // slot (and load-order) range of the replica
    float wall_lo, wall_hi;
    uint32_t seed_lo, seed_hi;
    uint32_t step0;          // RNG step offset of the replica
    int ntypes, ns;
    float dt, hdt, hdt2, ldt, inv_sqrt_dt;
    float rc2, inv_rc, rcc2, inv_rcc, rcut2;
    float rlist2;            // neighbour-list radius (rcut + skin) squared
    float half_skin2;        // (skin / 2)^2: a larger displacement forces a rebuild
    float inv_L[3];          // 1/L on periodic axes, 0 on walled ones (minimum image)
    float sR;                // exponent of w_R: s_f / 2
    float s_c;
    int sR_is1, sc_is2;      // integer fast paths
    float a[MAXT * MAXT], gamma[MAXT * MAXT], sigma[MAXT * MAXT];
    float kappa[MAXT * MAXT * MAXS];
    float fbody[3];
    uint32_t frozen_mask, react_mask;
    float k_react;
    int r_src, r_dst;
    int exclude_same_body;
    // membrane constants
    float m_kT, m_p, m_x0, m_m, m_kg, m_kl, m_kv, m_kb, m_cos0, m_sin0, m_gT, m_gC;
    float m_wlc0;            // kT/p
    float m_rand_T, m_rand_C;  // sqrt(2kT/dt) sqrt(2 gT), sqrt(2kT/dt) sqrt(3gC-gT)/3
    int m_lagged;            // area/volume constraints from the previous step's totals
    float qr_coef;           // random flux: m_s sqrt(rho) (Eq. 7-8); 0: off
    int fbody_flip;          // body force negated where z >= L_z/2 (double Poiseuille)
    float cyl_R;             // bounce-back cylinder radius about the x axis through the box centre; 0: none
    float cyl_c[2];          // the axis: (y, z) = (L_y/2, L_z/2)
};

// One membrane.
struct RbcDev {
    int gbase;      // load-order (global) index of vertex 0
    int rep;        // replica
    int topo;       // topology index
    int nv, ntri, ne;
    int a0j_off;    // offset of per-triangle rest areas
    int bond_off;   // offset of per-edge (l_m, k_p)
    int tri_off;    // offset of its triangles (int[3 ntri]) in the triangle table
    int fan_off;    // offset of vertex 0's fan in the fan table
    int fan_stride; // fan entries per vertex: the mesh's largest degree
    int pad_;
    double A0, V0;
    double kgA0, kvV0;  // k_g / A0, k_v / V0 (Eq. 14-15 coefficients per unit excess)
    double inv_nv;      // 1 / nv
};

// Ring (one-ring fan) entry of a vertex v, counter-clockwise seen from
// outside: triangles (v, nb[l], nb[l+1]) are the mesh triangles around v.
struct RingEntry {
    int nb;       // neighbour vertex nb[l]
    int edge;     // edge index of (v, nb[l])
    int tri;      // triangle index of (v, nb[l], nb[l+1])
    int across;   // vertex opposite v across the edge (nb[l], nb[l+1])
};

// The device form of fan entry l of vertex v, at a fixed stride per vertex
// (entry v * fan_stride + l of its mesh), with the cyclic neighbours nb[l+1]
// and nb[l-1] included: a lane reaches all its vertex indices with one
// 32-byte load and no offset table. Entries past the degree have nb = -1.
struct __align__(16) FanEntry {
    int nb, edge, tri, across;
    int nb_next, nb_prev;
    int pad0, pad1;
};

// Programmatic dependent launch: let the next kernel in the stream begin
// launching, then wait until the previous kernel has finished and its writes
// are visible. Both are no-ops for a kernel launched without the attribute.
// Every step kernel calls this before its first global-memory access.
__device__ __forceinline__ void pdl_enter()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

__device__ __forceinline__ int wbits(float w) { return __float_as_int(w); }
__device__ __forceinline__ float bitsw(int b) { return __int_as_float(b); }

// ---------------------------------------------------------------- RNG
// TEA (Wheeler & Needham 1994), 8 rounds, 64-bit block = the unordered pair
// of ids, 128-bit key = (seed, step, stream).
__device__ __forceinline__ uint2 tea8(uint32_t y, uint32_t z, uint32_t k0, uint32_t k1,
                                      uint32_t k2, uint32_t k3)
{
    uint32_t sum = 0u;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        sum += 0x9E3779B9u;
        y += ((z << 4) + k0) ^ (z + sum) ^ ((z >> 5) + k1);
        z += ((y << 4) + k2) ^ (y + sum) ^ ((y >> 5) + k3);
    }
    return make_uint2(y, z);
}

__device__ __forceinline__ uint2 pair_bits(uint32_t i, uint32_t j, uint32_t seed_lo,
                                           uint32_t seed_hi, uint32_t step, uint32_t stream)
{
    uint32_t lo = min(i, j), hi = max(i, j);
    return tea8(lo, hi, seed_lo, seed_hi, step, stream);
}

// Uniform in (0, 1) from the top 23 bits, centred in its bin: exact in fp32.
__device__ __forceinline__ float u23(uint32_t b)
{
    return __fmaf_rn((float)(b >> 9), 0x1p-23f, 0x1p-24f);
}

// Box-Muller: (r cos(2 pi u2), r sin(2 pi u2)), r = sqrt(-2 ln u1). The angle
// is taken in [-pi, pi) as 2 pi (u2 - 1/2), where the fast sine/cosine are
// accurate, and the half turn is undone by the sign.
__device__ __forceinline__ float2 normal2(uint2 b)
{
    float u1 = u23(b.x), u2 = u23(b.y);
    float rad = sqrtf(-2.0f * __logf(u1));
    float s, c;
    __sincosf(6.28318530717958648f * (u2 - 0.5f), &s, &c);
    return make_float2(-rad * c, -rad * s);
}

__device__ __forceinline__ float normal_cos(uint2 b)
{
    float u1 = u23(b.x), u2 = u23(b.y);
    float rad = sqrtf(-2.0f * __logf(u1));
    return -rad * __cosf(6.28318530717958648f * (u2 - 0.5f));
}

// ---------------------------------------------------------- geometry
__device__ __forceinline__ int cell_coord(float x, float scale, int n)
{
    int c = __float2int_rd(__fmul_rn(x, scale));
    return min(max(c, 0), n - 1);
}

__device__ __forceinline__ int cell_of(const RepParams &P, float x, float y, float z)
{
    int cx = cell_coord(x, P.cell_scale[0], P.nc[0]);
    int cy = cell_coord(y, P.cell_scale[1], P.nc[1]);
    int cz = cell_coord(z, P.cell_scale[2], P.nc[2]);
    return P.cell_base + (cz * P.nc[1] + cy) * P.nc[0] + cx;
}

// Count one particle (cell c >= 0) into its scan tile; lanes of a warp that
// share a tile add once. Every lane of the warp must call it (c < 0: none).
__device__ __forceinline__ void add_tile_count(int *tile_sum, int c)
{
    const int tile = c >= 0 ? (c >> SCAN_TILE_LOG2) : -1 - (int)(threadIdx.x & 31);
    const unsigned same = __match_any_sync(0xffffffffu, tile);
    if (c >= 0 && (int)(threadIdx.x & 31) == __ffs(same) - 1) atomicAdd(tile_sum + tile, __popc(same));
}

// One row (dy, dz) of the cell stencil of particle i, whose cell is
// (cx, cy, cz) and whose offsets inside it along y and z are oy, oz: the
// cells cx-m..cx+m of that row that come within sqrt(rtrim2) of the particle
// (less a margin eps for the rounding of cell assignment), as at most two
// contiguous slot ranges [jb, je) -- two where the row wraps around x -- and
// the periodic image shifts to add to x_i. g must come in zeroed; false (g
// untouched apart from the shifts) when the row has no such cell.
struct RowSeg {
    int jb[2], je[2];
    float sx1, sy, sz;       // x shift of the second range; y and z shifts
};

// Row (dy, dz) of the stencil, |dy|, |dz| <= m.
__device__ __forceinline__ bool stencil_row_d(const RepParams &P, const int *__restrict__ cs, float4 pi, int cx,
                                              int cy, int cz, int dy, int dz, int m, float oy, float oz,
                                              float eps, float rtrim2, RowSeg &g)
{
    const float hy = P.h[1], hz = P.h[2];
    // distance from particle i to the slab of the row's cells
    const float ay = dy == 0 ? 0.f : (dy > 0 ? (float)dy * hy - oy : oy - (float)(dy + 1) * hy);
    const float az = dz == 0 ? 0.f : (dz > 0 ? (float)dz * hz - oz : oz - (float)(dz + 1) * hz);
    const float by = fmaxf(ay - eps, 0.f), bz = fmaxf(az - eps, 0.f);
    const float rem = rtrim2 - by * by - bz * bz;
    int y = cy + dy, z = cz + dz;
    bool ok = rem > 0.f;
    if (y < 0) { y += P.nc[1]; g.sy = P.L[1]; }
    else if (y >= P.nc[1]) { y -= P.nc[1]; g.sy = -P.L[1]; }
    if (z < 0) { if (P.periodic[2]) { z += P.nc[2]; g.sz = P.L[2]; } else ok = false; }
    else if (z >= P.nc[2]) { if (P.periodic[2]) { z -= P.nc[2]; g.sz = -P.L[2]; } else ok = false; }
    if (!ok) return false;
    const float rx = sqrtf(rem) + eps;
    const int x0 = max(cx - m, __float2int_rd((pi.x - rx) * P.cell_scale[0]));
    const int x1 = min(cx + m, __float2int_rd((pi.x + rx) * P.cell_scale[0]));
    const int base = P.cell_base + (z * P.nc[1] + y) * P.nc[0];
    const int nx = P.nc[0];
    if (x0 >= 0 && x1 < nx) {
        g.jb[0] = cs[base + x0];
        g.je[0] = cs[base + x1 + 1];
    } else if (x0 < 0) {
        g.jb[0] = cs[base];
        g.je[0] = cs[base + x1 + 1];
        g.jb[1] = cs[base + nx + x0];
        g.je[1] = cs[base + nx];
        g.sx1 = P.L[0];
    } else {
        g.jb[0] = cs[base + x0];
        g.je[0] = cs[base + nx];
        g.jb[1] = cs[base];
        g.je[1] = cs[base + x1 - nx + 1];
        g.sx1 = -P.L[0];
    }
    return true;
}

__device__ __forceinline__ bool stencil_row(const RepParams &P, const int *__restrict__ cs, float4 pi, int cx,
                                            int cy, int cz, int row, float oy, float oz, float eps,
                                            float rtrim2, RowSeg &g)
{
    const int m = P.m_stencil, width = 2 * m + 1;
    return stencil_row_d(P, cs, pi, cx, cy, cz, row % width - m, row / width - m, m, oy, oz, eps, rtrim2, g);
}

// Fold a coordinate back into [0, L) after a move of less than one box.
__device__ __forceinline__ float wrap_coord(float x, float L)
{
    if (x < 0.0f) x = __fadd_rn(x, L);
    else if (x >= L) x = __fsub_rn(x, L);
    if (!(x >= 0.0f && x < L)) {         // far jump, rounding onto L, or NaN
        x = __fsub_rn(x, __fmul_rn(L, floorf(__fdiv_rn(x, L))));
        if (!(x >= 0.0f && x < L)) x = 0.0f;
    }
    return x;
}

// Position predictor r_{k+1} = r_k + dt v_k + dt^2/2 F_k with periodic wrap
// and bounce-back at the z walls. Explicit rounding keeps the result
// bit-identical wherever it is recomputed. flip: velocity must be reversed.
__device__ __forceinline__ float3 predict_pos(const RepParams &P, float4 p, float4 v, float4 f,
                                              bool &flip)
{
    float r[3] = {__fmaf_rn(P.hdt2, f.x, __fmaf_rn(P.dt, v.x, p.x)),
                  __fmaf_rn(P.hdt2, f.y, __fmaf_rn(P.dt, v.y, p.y)),
                  __fmaf_rn(P.hdt2, f.z, __fmaf_rn(P.dt, v.z, p.z))};
    flip = false;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        if (P.periodic[c]) {
            r[c] = wrap_coord(r[c], P.L[c]);
        } else {
            if (r[c] < P.wall_lo) { r[c] = __fsub_rn(2.0f * P.wall_lo, r[c]); flip = true; }
            else if (r[c] > P.wall_hi) { r[c] = __fsub_rn(2.0f * P.wall_hi, r[c]); flip = true; }
            if (!(r[c] >= 0.0f && r[c] < P.L[c])) r[c] = fminf(fmaxf(r[c], 0.0f), P.L[c] * 0.99999994f);
        }
    }
    if (P.cyl_R > 0.0f) {
        // bounce-back at the cylinder: a point at distance d > R from the
        // axis goes to distance 2R - d on the same radial line
        const float dy = __fsub_rn(r[1], P.cyl_c[0]), dz = __fsub_rn(r[2], P.cyl_c[1]);
        const float d = __fsqrt_rn(__fadd_rn(__fmul_rn(dy, dy), __fmul_rn(dz, dz)));
        if (d > P.cyl_R) {
            const float s = __fdiv_rn(__fsub_rn(__fmul_rn(2.0f, P.cyl_R), d), d);
            r[1] = __fadd_rn(P.cyl_c[0], __fmul_rn(dy, s));
            r[2] = __fadd_rn(P.cyl_c[1], __fmul_rn(dz, s));
            flip = true;
        }
    }
    return make_float3(r[0], r[1], r[2]);
}

__device__ __forceinline__ float min_image(float d, float L, int periodic)
{
    if (periodic) {
        if (d > 0.5f * L) d -= L;
        else if (d < -0.5f * L) d += L;
    }
    return d;
}

// ------------------------------------------- fixed-point accumulation
// The half-shell pair kernel hands each pair's share for the partner to a
// 64-bit fixed-point accumulator with integer atomics: integer sums do not
// depend on the order in which the atomics land, so results stay
// bit-reproducible. Forces in units of 2^-32, fluxes in units of 2^-40; a
// single contribution must stay below 2^23 (force) or 2^16 (flux), which
// keeps a particle's sum of up to 256 of them inside the 64-bit range; a
// larger or non-finite contribution is dropped and flags the replica
// (status bit 1, as a non-finite force).
constexpr float ACC_F_SCALE = 0x1p32f, ACC_F_UNIT = 0x1p-32f, ACC_F_LIMIT = 0x1p23f;
constexpr float ACC_Q_SCALE = 0x1p40f, ACC_Q_UNIT = 0x1p-40f, ACC_Q_LIMIT = 0x1p16f;

__device__ __forceinline__ void acc_add(long long *p, float x, float scale, float limit, uint32_t *err)
{
    if (!(fabsf(x) < limit)) {
        atomicOr(err, 1u);
        return;
    }
    atomicAdd(reinterpret_cast<unsigned long long *>(p), (unsigned long long)__float2ll_rn(x * scale));
}

// ---------------------------------------------------- FP64 compensated sum
// (sum, compensation) pair; merging two pairs adds the rounding error of the
// leading sum exactly (Knuth's TwoSum), branch-free.
struct KSum {
    double s, c;
    __device__ __forceinline__ void add(double x)
    {
        const double t = s + x;
        const double bp = t - s;
        c += (s - (t - bp)) + (x - bp);
        s = t;
    }
    __device__ __forceinline__ double value() const { return s + c; }
};

__device__ __forceinline__ void ksum_merge(KSum &a, const KSum &b)
{
    a.add(b.s);
    a.c += b.c;
}

// ------------------------------------------ float-float compensated sum
// (hi, lo) with hi + lo carrying ~48 significant bits; additions use the
// exact TwoSum of the leading parts. GB300 runs binary64 at a small fraction
// of the binary32 rate, so long sums are carried in float-float and only the
// last few partials are combined in binary64.
struct FF {
    float hi, lo;
};

__device__ __forceinline__ FF ff_add(FF a, FF b)
{
    const float s = __fadd_rn(a.hi, b.hi);
    const float bp = __fsub_rn(s, a.hi);
    float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bp)), __fsub_rn(b.hi, bp));
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    const float h = __fadd_rn(s, e);
    return FF{h, __fsub_rn(e, __fsub_rn(h, s))};
}

__device__ __forceinline__ FF ff_add(FF a, float x) { return ff_add(a, FF{x, 0.0f}); }

// x*x exactly as a float-float (the FMA recovers the rounding error)
__device__ __forceinline__ FF ff_sqr(float x)
{
    const float p = __fmul_rn(x, x);
    return FF{p, __fmaf_rn(x, x, -p)};
}

__device__ __forceinline__ FF ff_shfl_down(FF a, int o)
{
    return FF{__shfl_down_sync(0xffffffffu, a.hi, o), __shfl_down_sync(0xffffffffu, a.lo, o)};
}

__device__ __forceinline__ double ff_value(FF a) { return (double)a.hi + (double)a.lo; }

}  // namespace tdpd
