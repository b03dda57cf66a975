// FP64 observables (compensated sums) and the random-number parity hook.
#include "launch.h"

namespace tdpd {

// One CTA per chunk of a replica's slots: compensated float-float sums of v,
// |v|^2 (exact squares) and the non-frozen count over non-frozen particles,
// and of each species over all particles; binary64 partials per chunk. The
// CTA that finishes last adds the partials in chunk order into total
// (OBS_K values, zero for species beyond ns) and re-arms the counter.
template <int NS>
__global__ void __launch_bounds__(256) k_observables(Buffers b, const RepParams *__restrict__ reps,
                                                     const int4 *__restrict__ chunks, int n_chunks, int ns_rt,
                                                     double *part, double *total, unsigned *done)
{
    constexpr int NSP = NS > 0 ? NS : MAXS;   // species carried
    constexpr int NQ = 6 + 2 * NSP;
    const int ns = NS > 0 ? NS : ns_rt;
    const int4 ch = chunks[blockIdx.x];
    const RepParams &P = reps[ch.x];
    FF acc[NQ];
#pragma unroll
    for (int k = 0; k < NQ; ++k) acc[k] = FF{0.0f, 0.0f};
    for (int k = ch.y + threadIdx.x; k < ch.z; k += blockDim.x) {
        const int type = (int)((uint32_t)wbits(b.pos[k].w) >> 24);
        if (!((P.frozen_mask >> type) & 1u)) {
            const float4 v = b.vel[k];
            acc[0] = ff_add(acc[0], v.x);
            acc[1] = ff_add(acc[1], v.y);
            acc[2] = ff_add(acc[2], v.z);
            acc[3] = ff_add(ff_add(ff_add(acc[3], ff_sqr(v.x)), ff_sqr(v.y)), ff_sqr(v.z));
            acc[4] = ff_add(acc[4], 1.0f);
        }
        const bool mem = wbits(b.vt[k].w) >= 0;
        if (mem) acc[5] = ff_add(acc[5], 1.0f);
#pragma unroll
        for (int s = 0; s < NSP; ++s)
            if (s < ns) {
                const float c = b.C[(size_t)k * ns + s];
                acc[6 + s] = ff_add(acc[6 + s], c);
                if (mem) acc[6 + NSP + s] = ff_add(acc[6 + NSP + s], c);
            }
    }
    __shared__ FF sh[8][NQ];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < NQ; ++k) acc[k] = ff_add(acc[k], ff_shfl_down(acc[k], o));
    if (lane == 0)
        for (int k = 0; k < NQ; ++k) sh[w][k] = acc[k];
    __syncthreads();
    if (threadIdx.x < NQ) {
        const int q = threadIdx.x;
        FF a = sh[0][q];
        for (int ww = 1; ww < nw; ++ww) a = ff_add(a, sh[ww][q]);
        const int k = q < 6 + NSP ? q : 6 + MAXS + (q - 6 - NSP);    // slot in the OBS_K layout
        part[(size_t)blockIdx.x * OBS_K + k] = ff_value(a);
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(done, 1u) == (unsigned)n_chunks - 1u;
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x < OBS_K) {
        const int k = threadIdx.x;
        const bool used = k < 6 || (k < 6 + MAXS ? k - 6 < ns : k - 6 - MAXS < ns);
        double a = 0.0;
        if (used)
            for (int c = 0; c < n_chunks; ++c) a += __ldcg(part + (size_t)c * OBS_K + k);
        total[k] = a;
    }
    if (threadIdx.x == 0) *done = 0u;
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

void launch_observables(const Buffers &b, const RepParams *reps, const int4 *chunks, int n_chunks,
                        int ns, double *part, double *total, unsigned *done, cudaStream_t st)
{
    if (n_chunks <= 0) return;
    switch (ns) {
    case 1: k_observables<1><<<n_chunks, 256, 0, st>>>(b, reps, chunks, n_chunks, ns, part, total, done); break;
    case 2: k_observables<2><<<n_chunks, 256, 0, st>>>(b, reps, chunks, n_chunks, ns, part, total, done); break;
    default: k_observables<0><<<n_chunks, 256, 0, st>>>(b, reps, chunks, n_chunks, ns, part, total, done); break;
    }
}

void launch_debug_rng(uint64_t seed, int n, const uint32_t *i, const uint32_t *j,
                      const uint32_t *step, const uint32_t *stream, uint32_t *bits, float *normal,
                      cudaStream_t st)
{
    if (n <= 0) return;
    k_debug_rng<<<(n + 255) / 256, 256, 0, st>>>(seed, n, i, j, step, stream, bits, normal);
}

}  // namespace tdpd
