// FP64 observables (compensated sums) and the random-number parity hook.
#include "launch.h"

namespace tdpd {

// One CTA per replica: sums of v, |v|^2 and of the non-frozen count over the
// non-frozen particles, and of each species over all particles. out holds,
// per replica, [px, py, pz, v2, n_mobile, mass_0 .. mass_{ns-1}].
template <int K>
__device__ void block_reduce_ksum(KSum (&v)[K], double *out)
{
    __shared__ double sh[32][K][2];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k = 0; k < K; ++k)
        for (int o = 16; o > 0; o >>= 1) {
            KSum t;
            t.s = __shfl_down_sync(0xffffffffu, v[k].s, o);
            t.c = __shfl_down_sync(0xffffffffu, v[k].c, o);
            if (lane + o < 32) ksum_merge(v[k], t);
        }
    if (lane == 0)
        for (int k = 0; k < K; ++k) { sh[w][k][0] = v[k].s; sh[w][k][1] = v[k].c; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int ww = 1; ww < nw; ++ww)
            for (int k = 0; k < K; ++k) {
                KSum t;
                t.s = sh[ww][k][0];
                t.c = sh[ww][k][1];
                ksum_merge(v[k], t);
            }
        for (int k = 0; k < K; ++k) out[k] = v[k].value();
    }
}

constexpr int OBS_K = 5 + MAXS;

__global__ void __launch_bounds__(256) k_observables(Buffers b, const RepParams *__restrict__ reps,
                                                     int ns, double *out)
{
    const RepParams &P = reps[blockIdx.x];
    KSum acc[OBS_K];
    for (int k = 0; k < OBS_K; ++k) acc[k].s = acc[k].c = 0.0;
    for (int k = P.pbase + threadIdx.x; k < P.pbase + P.n; k += blockDim.x) {
        const int type = (int)((uint32_t)wbits(b.pos[k].w) >> 24);
        if (!((P.frozen_mask >> type) & 1u)) {
            const float4 v = b.vel[k];
            acc[0].add(v.x);
            acc[1].add(v.y);
            acc[2].add(v.z);
            acc[3].add((double)v.x * v.x + (double)v.y * v.y + (double)v.z * v.z);
            acc[4].add(1.0);
        }
        for (int s = 0; s < ns; ++s) acc[5 + s].add(b.C[(size_t)k * ns + s]);
    }
    block_reduce_ksum<OBS_K>(acc, out + (size_t)blockIdx.x * OBS_K);
}

__global__ void k_debug_rng(uint64_t seed, int n, const uint32_t *i, const uint32_t *j,
                            const uint32_t *step, const uint32_t *stream, uint32_t *bits,
                            float *normal)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const uint2 b = pair_bits(i[k], j[k], (uint32_t)seed, (uint32_t)(seed >> 32), step[k], stream[k]);
    bits[2 * k] = b.x;
    bits[2 * k + 1] = b.y;
    const float2 g = normal2(b);
    normal[2 * k] = g.x;
    normal[2 * k + 1] = g.y;
}

void launch_observables(const Buffers &b, const RepParams *reps, int n_rep, int ns, double *out,
                        cudaStream_t st)
{
    if (n_rep <= 0) return;
    k_observables<<<n_rep, 256, 0, st>>>(b, reps, ns, out);
}

void launch_debug_rng(uint64_t seed, int n, const uint32_t *i, const uint32_t *j,
                      const uint32_t *step, const uint32_t *stream, uint32_t *bits, float *normal,
                      cudaStream_t st)
{
    if (n <= 0) return;
    k_debug_rng<<<(n + 255) / 256, 256, 0, st>>>(seed, n, i, j, step, stream, bits, normal);
}

}  // namespace tdpd
