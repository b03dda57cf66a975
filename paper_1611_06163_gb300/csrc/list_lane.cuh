// The per-lane Verlet list build (the list of Sec. 3.1), shared by the
// list-build kernel and the pair kernel, which on a rebuild step builds the
// lists of its own lanes before walking them.
#pragma once

#include <type_traits>

#include "launch.h"

namespace tdpd {

// The list of one pair lane (particle i, lane sub of LPP, thread gt of the
// pair kernel's layout) over the cell stencil, its count in nlc and, for lane
// 0, the build position xb[i]. M: the stencil half-width when it is known at
// compile time (2, the default cell size), else 0 (read per replica). Used by
// k_list_build and, on rebuild steps, by the pair kernel for its own lanes.
//
// HALF: only the upper half of the stencil, so that every unordered pair is
// listed once. A cell's offset (dx, dy, dz) from particle i's cell has one
// representative in [-m, m]^3 (a periodic axis holds at least 2m + 1 cells),
// and the pair belongs to the side from which that offset is upper: rows
// with dz > 0, or dz = 0 and dy > 0 (the rows after the home row), and in
// the home row the cells with dx > 0 and, in i's own cell, the slots after
// i. Cells of a row are consecutive slots, so the home row's upper part is
// the slot range after i up to the row's end, plus the segment that wraps
// around to the right.
template <int LPP, int M, bool HALF = false>
__device__ __forceinline__ void build_lane(const ListArgs &A, int gt, int i, int sub, float4 pi, int rep)
{
    const RepParams &P = A.reps[rep];
    const int m = M > 0 ? M : P.m_stencil, width = 2 * m + 1, nrow = width * width;
    const int cx = cell_coord(pi.x, P.cell_scale[0], P.nc[0]);
    const int cy = cell_coord(pi.y, P.cell_scale[1], P.nc[1]);
    const int cz = cell_coord(pi.z, P.cell_scale[2], P.nc[2]);
    const float oy = pi.y - (float)cy * P.h[1], oz = pi.z - (float)cz * P.h[2];
    const float eps = 1e-4f * fmaxf(P.h[0], fmaxf(P.h[1], P.h[2]));
    const float rl2 = P.rlist2;
    int *out = A.nl + (size_t)(gt >> 5) * A.cap * 32 + (gt & 31);   // next entry
    const int cap = A.cap;
    int c = 0;
    // the row's candidates, four per trip with their loads in flight together,
    // appended in slot order (the capacity test once per trip while four more
    // entries fit); SELF: the home row, which holds particle i itself
    auto walk = [&](const RowSeg &g, auto self) {
        constexpr bool SELF = decltype(self)::value;
        const float py = pi.y + g.sy, pz = pi.z + g.sz;
#pragma unroll
        for (int sg = 0; sg < 2; ++sg) {
            const float px = pi.x + (sg ? g.sx1 : 0.f);
            const int je = g.je[sg];
            for (int j0 = g.jb[sg]; j0 < je; j0 += 4) {
                float4 pj[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) pj[u] = j0 + u < je ? A.pos[j0 + u] : make_float4(1e30f, 0.f, 0.f, 0.f);
                bool ok[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const float dx = px - pj[u].x, dy = py - pj[u].y, dz = pz - pj[u].z;
                    ok[u] = dx * dx + dy * dy + dz * dz < rl2 && (!SELF || j0 + u != i);
                }
                if (c + 4 <= cap) {
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        if (ok[u]) {
                            *out = j0 + u;
                            out += 32;
                            ++c;
                        }
                } else {
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        if (ok[u]) {
                            if (c < cap) {
                                *out = j0 + u;
                                out += 32;
                            }
                            ++c;
                        }
                }
            }
        }
    };
    for (int row = (HALF ? nrow / 2 : 0) + sub; row < nrow; row += LPP) {
        const int dy = row % width - m, dz = row / width - m;
        RowSeg g = {{0, 0}, {0, 0}, 0.f, 0.f, 0.f};
        if (!stencil_row_d(P, A.cell_start, pi, cx, cy, cz, dy, dz, m, oy, oz, eps, rl2 * 1.0002f, g)) continue;
        if (dy == 0 && dz == 0) {
            if (HALF) {
                // the home row from the slot after i; a segment that wraps
                // around to the left (x shift +L) holds only cells with dx < 0
                g.jb[0] = i + 1;
                if (g.sx1 > 0.f) g.je[1] = g.jb[1];
            }
            walk(g, std::true_type{});
        } else {
            walk(g, std::false_type{});
        }
    }
    A.nlc[gt] = A.cap > 0 ? min(c, A.cap) : c;
    if (A.cap > 0 && c > A.cap) atomicOr(A.err + rep, 2u);
    if (sub == 0) A.xb[i] = pi;
}

}  // namespace tdpd
