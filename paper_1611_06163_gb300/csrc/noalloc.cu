// Pair force + flux without any device allocation (tdpd_pair_forces_noalloc).
//
// Every scratch buffer this entry point needs -- the cell histogram and
// offsets, the two sorted copies of the particle state, the slot maps -- lives
// in one file-scope __device__ array of fixed size, g_noalloc_scratch, which
// every GPU that loads the library holds until the process exits. The caller
// supplies inputs and outputs; nothing is allocated or freed per call.
//
// In host code the name g_noalloc_scratch is only a host-side stand-in for the
// symbol, not a device address: handing it to a kernel would fault or, where
// the GPU can reach host memory, silently use the wrong memory. The device
// address is obtained once per device with cudaGetSymbolAddress, with that
// device current, and cached.
#include <cmath>
#include <cstdio>
#include <mutex>

#include "launch.h"

using namespace tdpd;

namespace {

constexpr int NA_N = TDPD_NOALLOC_MAX_PARTICLES;
constexpr int NA_C = TDPD_NOALLOC_MAX_CELLS;
constexpr int NA_S = TDPD_NOALLOC_MAX_SPECIES;
constexpr int NA_TILES = (NA_C + SCAN_TILE - 1) / SCAN_TILE;
static_assert(NA_C % SCAN_TILE == 0, "the cell capacity is whole scan tiles");

// Layout of the scratch array (only its size and offsets are used on the host).
struct __align__(256) NoAllocLayout {
    RepParams params;
    float4 pos[2][NA_N], vt[2][NA_N], vel[2][NA_N], frc[2][NA_N];
    float C[2][NA_N * NA_S], Ct[2][NA_N * NA_S], Q[2][NA_N * NA_S];
    float4 fext[NA_N];
    int inv[NA_N];
    int2 cellrank[NA_N], keys[NA_N];
    int count[NA_C];
    int cell_start[NA_C + 4];
    int tile_sum[2][NA_TILES];
    uint32_t err[4];
    uint32_t step_ctr[4];
};
static_assert(sizeof(NoAllocLayout) <= TDPD_NOALLOC_SCRATCH_BYTES, "scratch size as documented in tdpd.h");

static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocLayout)];

std::mutex g_mu;
constexpr int MAX_DEVICES = 64;
NoAllocLayout *g_dev_ptr[MAX_DEVICES] = {};

tdpd_status na_fail(tdpd_status code, const char *msg)
{
    set_thread_error(msg);
    return code;
}

// Copy the inputs into sorted-state buffer 0, clear what the binning counts
// into, and set the step counter.
__global__ void k_na_pack(RepParams P, int n, int ns, const float *__restrict__ pos,
                          const float *__restrict__ vel, const float *__restrict__ conc,
                          const int32_t *__restrict__ type, uint32_t step, NoAllocLayout *S)
{
    const int stride = gridDim.x * blockDim.x;
    const int g0 = blockIdx.x * blockDim.x + threadIdx.x;
    if (g0 == 0) {
        S->params = P;
        S->err[0] = 0u;
        S->step_ctr[0] = step;
    }
    for (int c = g0; c < NA_C; c += stride) S->count[c] = 0;
    // cells past the scanned tiles end at the particle count
    for (int c = g0; c <= NA_C; c += stride) S->cell_start[c] = n;
    for (int t = g0; t < 2 * NA_TILES; t += stride) S->tile_sum[t / NA_TILES][t % NA_TILES] = 0;
    for (int k = g0; k < n; k += stride) {
        // a type outside [0, n_types) is recorded (the outputs become NaN)
        // and replaced by type 0, so that no table lookup leaves its range
        int t = type[k];
        if (t < 0 || t >= P.ntypes) {
            atomicOr(&S->err[1], 4u);
            t = 0;
        }
        const uint32_t w = (uint32_t)k | ((uint32_t)t << 24);
        S->pos[0][k] = make_float4(pos[3 * k], pos[3 * k + 1], pos[3 * k + 2], __int_as_float((int)w));
        S->vel[0][k] = make_float4(vel[3 * k], vel[3 * k + 1], vel[3 * k + 2], __int_as_float(0));
        S->vt[0][k] = make_float4(vel[3 * k], vel[3 * k + 1], vel[3 * k + 2], __int_as_float(-1));
        S->frc[0][k] = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int s = 0; s < ns; ++s) {
            const float c = conc[(size_t)k * ns + s];
            S->C[0][(size_t)k * ns + s] = c;
            S->Ct[0][(size_t)k * ns + s] = c;
            S->Q[0][(size_t)k * ns + s] = 0.f;
        }
    }
}

// Clear the input check word of this call (before k_na_pack may set it).
__global__ void k_na_clear(NoAllocLayout *S)
{
    S->err[1] = 0u;
}

// Load-order outputs; every output is NaN when an input type was out of
// range or some force came out non-finite (the caller checks the outputs).
__global__ void k_na_unpack(int n, int ns, const NoAllocLayout *S, float *force, float *flux)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const bool bad = (S->err[0] | S->err[1]) != 0u;
    const float nan = __int_as_float(0x7fc00000);
    const int slot = S->inv[k];
    const float4 f = S->frc[1][slot];
    force[3 * k] = bad ? nan : f.x;
    force[3 * k + 1] = bad ? nan : f.y;
    force[3 * k + 2] = bad ? nan : f.z;
    for (int s = 0; s < ns; ++s) flux[(size_t)k * ns + s] = bad ? nan : S->Q[1][(size_t)slot * ns + s];
}

Buffers buffers(NoAllocLayout *S, int b)
{
    Buffers B;
    B.pos = S->pos[b];
    B.vt = S->vt[b];
    B.vel = S->vel[b];
    B.frc = S->frc[b];
    B.C = S->C[b];
    B.Ct = S->Ct[b];
    B.Q = S->Q[b];
    return B;
}

}  // namespace

extern "C" tdpd_status tdpd_pair_forces_noalloc(const tdpd_config *cfg, const float *pair_coef,
                                                const float *kappa, int n, const float *pos,
                                                const float *vel, const float *conc,
                                                const int32_t *type, uint32_t step, float *force,
                                                float *flux, void *stream)
{
    if (!cfg || !pair_coef || !kappa) return na_fail(TDPD_EINVAL, "noalloc: null parameter pointer");
    if (n < 1 || n > NA_N) return na_fail(TDPD_EINVAL, "noalloc: particle count must be 1..TDPD_NOALLOC_MAX_PARTICLES");
    if (!pos || !vel || !conc || !type || !force || !flux) return na_fail(TDPD_EINVAL, "noalloc: null device array");
    const tdpd_config &c = *cfg;
    {
        // the checks of tdpd_create, then this entry point's own limits
        char why[200], msg[240];
        if (config_error(c, why, sizeof why)) {
            std::snprintf(msg, sizeof msg, "noalloc: %s", why);
            return na_fail(TDPD_EINVAL, msg);
        }
    }
    if (c.n_species > NA_S) return na_fail(TDPD_EINVAL, "noalloc: n_species must be 1..TDPD_NOALLOC_MAX_SPECIES");
    if (!c.periodic[2]) return na_fail(TDPD_EINVAL, "noalloc: the box must be periodic on every axis");
    const int m = c.cells_per_cutoff > 0 ? c.cells_per_cutoff : 2;
    const float rcut = c.rc > c.rcc ? c.rc : c.rcc;
    int nc[3];
    long ncell = 1;
    for (int k = 0; k < 3; ++k) {
        if (!(c.L[k] > 0) || (double)c.L[k] < 3.0 * rcut * 1.0001)
            return na_fail(TDPD_EINVAL, "noalloc: every box edge must hold three cut-offs");
        const double ncd = std::floor((double)c.L[k] * m / ((double)rcut * 1.0001));
        if (ncd > NA_C) return na_fail(TDPD_EINVAL, "noalloc: the box needs more than TDPD_NOALLOC_MAX_CELLS cells");
        nc[k] = (int)ncd;
        if (nc[k] < 2 * m + 1) return na_fail(TDPD_EINVAL, "noalloc: too few cells");
        ncell *= nc[k];
    }
    if (ncell > NA_C) return na_fail(TDPD_EINVAL, "noalloc: the box needs more than TDPD_NOALLOC_MAX_CELLS cells");

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES)
        return na_fail(TDPD_ECUDA, "noalloc: no usable current device");
    NoAllocLayout *S = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_dev_ptr[dev]) {
            void *p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) return na_fail(TDPD_ECUDA, "noalloc: cudaGetSymbolAddress of the scratch array failed");
            g_dev_ptr[dev] = static_cast<NoAllocLayout *>(p);
        }
        S = g_dev_ptr[dev];
    }

    const int ns = c.n_species;
    const RepParams P = build_rep_params(c, pair_coef, kappa, nc, m, 0, 0, n);
    cudaStream_t st = (cudaStream_t)stream;
    k_na_clear<<<1, 1, 0, st>>>(S);
    k_na_pack<<<64, 256, 0, st>>>(P, n, ns, pos, vel, conc, type, step, S);
    const Buffers b0 = buffers(S, 0), b1 = buffers(S, 1);
    const RepParams *dP = &S->params;
    const int n_tiles = (int)((ncell + SCAN_TILE - 1) / SCAN_TILE);
    launch_bin_init(b0, dP, n, S->count, S->tile_sum[0], S->cellrank, st);
    launch_scan(S->count, S->cell_start, n_tiles, S->tile_sum[0], S->tile_sum[1], S->step_ctr, 0, st);
    launch_scatter_keys(b0, S->cellrank, S->cell_start, S->keys, n, st);
    launch_rank_gather(b0, b1, dP, S->keys, S->cellrank, S->cell_start, S->inv, n, ns, 0, st);
    PairArgs a{};
    a.b = b1;
    a.fext = S->fext;
    a.reps = dP;
    a.cell_start = S->cell_start;
    a.count = S->count;
    a.cellrank = S->cellrank;
    a.tile_sum = S->tile_sum[1];
    a.err = S->err;
    a.step_ctr = S->step_ctr;
    a.n = n;
    a.ns = ns;
    a.integrate = 0;
    a.lpp = 1;
    while (a.lpp < 8 && (long)n * a.lpp < 300000) a.lpp *= 2;
    launch_pair(a, st);
    k_na_unpack<<<(n + 255) / 256, 256, 0, st>>>(n, ns, S, force, flux);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return na_fail(TDPD_ECUDA, cudaGetErrorString(e));
    return TDPD_OK;
}
