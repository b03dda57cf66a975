// Surrogate network: an ensemble of 4 -> 64 -> 64 -> 2 perceptrons with
// GELU hidden layers, bfloat16 weights (float master copies) and float
// accumulation, trained by full-batch Adam on the mean squared error of
// standardised outputs. Forward, backward and update are this file's kernels;
// the ensemble spread is the prediction's uncertainty.
//
// Parameter layout per member (TDPD_MLP_NPARAM floats): W1[64][4], b1[64],
// W2[64][64], b2[64], W3[2][64], b3[2], rows = outputs.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "launch.h"

using namespace tdpd;

namespace {

constexpr int IN = TDPD_MLP_IN, HID = TDPD_MLP_HIDDEN, OUT = TDPD_MLP_OUT;
constexpr int NP = TDPD_MLP_NPARAM;
constexpr int OW1 = 0, OB1 = OW1 + HID * IN, OW2 = OB1 + HID, OB2 = OW2 + HID * HID,
              OW3 = OB2 + HID, OB3 = OW3 + OUT * HID;
static_assert(OB3 + OUT == NP, "parameter layout");
constexpr int TPB = 128;

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }

__device__ __forceinline__ float gelu_grad(float z)
{
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

__device__ void load_weights(float *w, const float *params)
{
    for (int k = threadIdx.x; k < NP; k += blockDim.x) w[k] = bf16r(params[k]);
    __syncthreads();
}

// Forward pass (prediction) of one sample per thread.
__global__ void __launch_bounds__(TPB) k_mlp_fwd(const float *__restrict__ params, const float *__restrict__ X,
                                                 int n, float *Y)
{
    __shared__ float w[NP];
    const int mbr = blockIdx.y;
    load_weights(w, params + (size_t)mbr * NP);
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    float x[IN];
#pragma unroll
    for (int i = 0; i < IN; ++i) x[i] = X[(size_t)s * IN + i];
    float h1[HID];
#pragma unroll
    for (int o = 0; o < HID; ++o) {
        float z = w[OB1 + o];
#pragma unroll
        for (int i = 0; i < IN; ++i) z = fmaf(w[OW1 + o * IN + i], x[i], z);
        h1[o] = gelu(z);
    }
    float y0 = w[OB3], y1 = w[OB3 + 1];
    // four outputs at a time: four independent multiply-add chains
    for (int o0 = 0; o0 < HID; o0 += 4) {
        float z[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) z[q] = w[OB2 + o0 + q];
#pragma unroll
        for (int i = 0; i < HID; ++i)
#pragma unroll
            for (int q = 0; q < 4; ++q) z[q] = fmaf(w[OW2 + (o0 + q) * HID + i], h1[i], z[q]);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float h = gelu(z[q]);
            y0 = fmaf(w[OW3 + o0 + q], h, y0);
            y1 = fmaf(w[OW3 + HID + o0 + q], h, y1);
        }
    }
    const size_t yo = ((size_t)mbr * n + s) * OUT;
    Y[yo] = y0;
    Y[yo + 1] = y1;
}

// One training pass over a chunk of CH samples (one per thread) of one
// member: forward, back-propagation, and the chunk's share of every
// parameter's gradient, in one launch. The chunk's activations and error
// signals stay in shared memory, feature-major with rows padded to CH + 1 so
// that the per-sample writes and the per-parameter reads are free of bank
// conflicts. Each gradient entry is the chunk's samples summed in sample
// order; k_mlp_reduce adds the chunks in chunk order (float-float), so the
// gradient is deterministic.
constexpr int CH = 128;
constexpr int LD = CH + 1;

struct ChunkSmem {
    float w[NP];
    float X[IN][LD];
    float H1[HID][LD], A1[HID][LD];   // A1: z1, then the error signal d1
    float H2[HID][LD], A2[HID][LD];   // A2: z2, then the error signal d2
    float D3[OUT][LD];
    float red[CH / 32];
};

__global__ void __launch_bounds__(CH) k_mlp_chunk(const float *__restrict__ params, const float *__restrict__ X,
                                                 const float *__restrict__ T, int n, float *part, float *loss_part)
{
    extern __shared__ float4 smem_raw[];
    ChunkSmem &S = *reinterpret_cast<ChunkSmem *>(smem_raw);
    const int mbr = blockIdx.y, c = blockIdx.x, nch = gridDim.x;
    const int t = threadIdx.x;
    const int smp = c * CH + t;
    const bool valid = smp < n;
    for (int k = t; k < NP; k += CH) S.w[k] = bf16r(params[(size_t)mbr * NP + k]);
    __syncthreads();
    const float *w = S.w;

    // ---- forward
    float x[IN];
#pragma unroll
    for (int i = 0; i < IN; ++i) {
        x[i] = valid ? X[(size_t)smp * IN + i] : 0.0f;
        S.X[i][t] = x[i];
    }
    float h1[HID];
#pragma unroll
    for (int o = 0; o < HID; ++o) {
        float z = w[OB1 + o];
#pragma unroll
        for (int i = 0; i < IN; ++i) z = fmaf(w[OW1 + o * IN + i], x[i], z);
        h1[o] = valid ? gelu(z) : 0.0f;
        S.A1[o][t] = z;
        S.H1[o][t] = h1[o];
    }
    float y0 = w[OB3], y1 = w[OB3 + 1];
    for (int o0 = 0; o0 < HID; o0 += 4) {
        float z[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) z[q] = w[OB2 + o0 + q];
#pragma unroll
        for (int i = 0; i < HID; ++i)
#pragma unroll
            for (int q = 0; q < 4; ++q) z[q] = fmaf(w[OW2 + (o0 + q) * HID + i], h1[i], z[q]);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int o = o0 + q;
            const float h = valid ? gelu(z[q]) : 0.0f;
            S.A2[o][t] = z[q];
            S.H2[o][t] = h;
            y0 = fmaf(w[OW3 + o], h, y0);
            y1 = fmaf(w[OW3 + HID + o], h, y1);
        }
    }
    float d30 = 0.0f, d31 = 0.0f, err2 = 0.0f;
    if (valid) {
        const float e0 = y0 - T[(size_t)smp * OUT], e1 = y1 - T[(size_t)smp * OUT + 1];
        const float sc = 2.0f / (float)(n * OUT);
        d30 = sc * e0;
        d31 = sc * e1;
        err2 = e0 * e0 + e1 * e1;
    }
    S.D3[0][t] = d30;
    S.D3[1][t] = d31;

    // ---- back-propagation (this thread's sample)
    float d2[HID];
#pragma unroll
    for (int o = 0; o < HID; ++o) {
        const float g = fmaf(d30, w[OW3 + o], d31 * w[OW3 + HID + o]);
        d2[o] = g * gelu_grad(S.A2[o][t]);
        S.A2[o][t] = d2[o];
    }
    for (int i0 = 0; i0 < HID; i0 += 4) {
        float a[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int o = 0; o < HID; ++o)
#pragma unroll
            for (int q = 0; q < 4; ++q) a[q] = fmaf(d2[o], w[OW2 + o * HID + i0 + q], a[q]);
#pragma unroll
        for (int q = 0; q < 4; ++q) S.A1[i0 + q][t] = a[q] * gelu_grad(S.A1[i0 + q][t]);
    }
    for (int o = 16; o > 0; o >>= 1) err2 += __shfl_down_sync(0xffffffffu, err2, o);
    if ((t & 31) == 0) S.red[t >> 5] = err2;
    __syncthreads();

    // ---- the chunk's gradient: sums over its samples in sample order
    float *out = part + ((size_t)mbr * nch + c) * NP;
    {
        // dW2[o][i] = sum_s d2[o][s] h1[i][s]: a 4 x 8 tile per thread
        const int o0 = 4 * (t >> 3), i0 = 8 * (t & 7);
        float acc[4][8];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 8; ++b) acc[a][b] = 0.0f;
        for (int k = 0; k < CH; ++k) {
            float da[4], hb[8];
#pragma unroll
            for (int a = 0; a < 4; ++a) da[a] = S.A2[o0 + a][k];
#pragma unroll
            for (int b = 0; b < 8; ++b) hb[b] = S.H1[i0 + b][k];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(da[a], hb[b], acc[a][b]);
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 8; ++b) out[OW2 + (o0 + a) * HID + i0 + b] = acc[a][b];
    }
    if (t < HID) {
        // row o of dW1, db1 and db2
        const int o = t;
        float g1[IN] = {0.0f, 0.0f, 0.0f, 0.0f}, gb1 = 0.0f, gb2 = 0.0f;
        for (int k = 0; k < CH; ++k) {
            const float d1 = S.A1[o][k];
#pragma unroll
            for (int i = 0; i < IN; ++i) g1[i] = fmaf(d1, S.X[i][k], g1[i]);
            gb1 += d1;
            gb2 += S.A2[o][k];
        }
#pragma unroll
        for (int i = 0; i < IN; ++i) out[OW1 + o * IN + i] = g1[i];
        out[OB1 + o] = gb1;
        out[OB2 + o] = gb2;
    } else {
        // column i of dW3, and db3
        const int i = t - HID;
        float g0 = 0.0f, g1 = 0.0f, gb = 0.0f;
        for (int k = 0; k < CH; ++k) {
            const float h = S.H2[i][k];
            g0 = fmaf(S.D3[0][k], h, g0);
            g1 = fmaf(S.D3[1][k], h, g1);
            if (i < OUT) gb += S.D3[i][k];
        }
        out[OW3 + i] = g0;
        out[OW3 + HID + i] = g1;
        if (i < OUT) out[OB3 + i] = gb;
    }
    if (t == 0) {
        float l = 0.0f;
        for (int k = 0; k < CH / 32; ++k) l += S.red[k];
        loss_part[(size_t)mbr * nch + c] = l;
    }
}

// Each parameter's gradient: its chunks' sums added in chunk order
// (float-float); with adam, the Adam step (Kingma & Ba) on the float master
// weights, bc1 and bc2 being the bias corrections 1 - beta^t.
__global__ void __launch_bounds__(TPB) k_mlp_reduce(const float *__restrict__ part, int nch, int total,
                                                    float *grad, int adam, float *params, float *m, float *v,
                                                    float lr, float beta1, float beta2, float eps, float bc1,
                                                    float bc2)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= total) return;
    const int mbr = k / NP, p = k - mbr * NP;
    FF acc{0.0f, 0.0f};
    for (int c = 0; c < nch; ++c) acc = ff_add(acc, part[((size_t)mbr * nch + c) * NP + p]);
    const float g = acc.hi + acc.lo;
    grad[k] = g;
    if (adam) {
        const float mk = fmaf(beta1, m[k], (1.0f - beta1) * g);
        const float vk = fmaf(beta2, v[k], (1.0f - beta2) * g * g);
        m[k] = mk;
        v[k] = vk;
        params[k] -= lr * (mk / bc1) / (sqrtf(vk / bc2) + eps);
    }
}

}  // namespace

struct tdpd_mlp {
    int members = 0, n = 0, cap = 0;
    int64_t t = 0;
    float *params = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
    float *X = nullptr, *T = nullptr, *loss_part = nullptr;
    float *gpart = nullptr;     // [members][chunks][NP] per-chunk gradient sums
    double mx[IN] = {}, sx[IN] = {}, my[OUT] = {}, sy[OUT] = {};
    bool have_data = false;
    cudaStream_t st = nullptr;
    std::vector<void *> data_allocs;
};

namespace {

tdpd_status mfail(tdpd_status c, const std::string &msg)
{
    set_thread_error(msg.c_str());
    return c;
}

#define MCU(call)                                                                             \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) return mfail(TDPD_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

void free_data(tdpd_mlp *m)
{
    for (void *p : m->data_allocs) cudaFree(p);
    m->data_allocs.clear();
    m->cap = 0;
}

tdpd_status alloc_data(tdpd_mlp *m, int n)
{
    if (n <= m->cap) return TDPD_OK;
    cudaStreamSynchronize(m->st);
    free_data(m);
    const size_t M = m->members, nch = (size_t)(n + CH - 1) / CH;
    float **bufs[] = {&m->X, &m->T, &m->loss_part, &m->gpart};
    const size_t sizes[] = {(size_t)n * IN, (size_t)n * OUT, M * nch, M * nch * NP};
    for (int k = 0; k < 4; ++k) {
        void *p = nullptr;
        if (cudaMalloc(&p, sizes[k] * sizeof(float)) != cudaSuccess) {
            free_data(m);
            return mfail(TDPD_ENOMEM, "tdpd_mlp: device allocation failed");
        }
        m->data_allocs.push_back(p);
        *bufs[k] = (float *)p;
    }
    m->cap = n;
    return TDPD_OK;
}

// One pass over the data: the chunks' gradients, then their sums (and, with
// lr > 0, one Adam step); loss (may be NULL) receives each member's loss.
tdpd_status pass(tdpd_mlp *m, float lr, double *loss)
{
    static bool attr = false;
    if (!attr) {
        MCU(cudaFuncSetAttribute(k_mlp_chunk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(ChunkSmem)));
        attr = true;
    }
    const int nch = (m->n + CH - 1) / CH;
    k_mlp_chunk<<<dim3(nch, m->members), CH, sizeof(ChunkSmem), m->st>>>(m->params, m->X, m->T, m->n, m->gpart,
                                                                          m->loss_part);
    const int total = m->members * NP;
    float bc1 = 1.0f, bc2 = 1.0f;
    if (lr > 0.0f) {
        ++m->t;
        bc1 = (float)(1.0 - std::pow(0.9, (double)m->t));
        bc2 = (float)(1.0 - std::pow(0.999, (double)m->t));
    }
    k_mlp_reduce<<<(total + TPB - 1) / TPB, TPB, 0, m->st>>>(m->gpart, nch, total, m->grad, lr > 0.0f ? 1 : 0,
                                                             m->params, m->m, m->v, lr, 0.9f, 0.999f, 1e-8f, bc1,
                                                             bc2);
    MCU(cudaGetLastError());
    if (loss) {
        std::vector<float> part((size_t)m->members * nch);
        MCU(cudaMemcpyAsync(part.data(), m->loss_part, part.size() * sizeof(float), cudaMemcpyDeviceToHost, m->st));
        MCU(cudaStreamSynchronize(m->st));
        for (int k = 0; k < m->members; ++k) {
            double sum = 0.0;
            for (int c = 0; c < nch; ++c) sum += part[(size_t)k * nch + c];
            loss[k] = sum / ((double)m->n * OUT);
        }
    }
    return TDPD_OK;
}

}  // namespace

extern "C" {

tdpd_status tdpd_mlp_create(tdpd_mlp **out, int members)
{
    if (!out || members < 1 || members > 64) return mfail(TDPD_EINVAL, "tdpd_mlp_create: 1..64 members");
    *out = nullptr;
    tdpd_mlp *m = new (std::nothrow) tdpd_mlp;
    if (!m) return mfail(TDPD_ENOMEM, "host allocation failed");
    m->members = members;
    const size_t bytes = (size_t)members * NP * sizeof(float);
    void *p[4] = {};
    for (int k = 0; k < 4; ++k)
        if (cudaMalloc(&p[k], bytes) != cudaSuccess) {
            for (int j = 0; j < k; ++j) cudaFree(p[j]);
            delete m;
            return mfail(TDPD_ENOMEM, "tdpd_mlp_create: device allocation failed");
        }
    m->params = (float *)p[0];
    m->m = (float *)p[1];
    m->v = (float *)p[2];
    m->grad = (float *)p[3];
    if (cudaStreamCreateWithFlags(&m->st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMemset(m->params, 0, bytes) != cudaSuccess || cudaMemset(m->m, 0, bytes) != cudaSuccess ||
        cudaMemset(m->v, 0, bytes) != cudaSuccess) {
        for (int k = 0; k < 4; ++k) cudaFree(p[k]);
        delete m;
        return mfail(TDPD_ECUDA, "tdpd_mlp_create: stream or memset failed");
    }
    *out = m;
    return TDPD_OK;
}

tdpd_status tdpd_mlp_set_params(tdpd_mlp *m, const float *params)
{
    if (!m || !params) return mfail(TDPD_EINVAL, "null argument");
    const size_t bytes = (size_t)m->members * NP * sizeof(float);
    MCU(cudaMemcpyAsync(m->params, params, bytes, cudaMemcpyHostToDevice, m->st));
    MCU(cudaMemsetAsync(m->m, 0, bytes, m->st));
    MCU(cudaMemsetAsync(m->v, 0, bytes, m->st));
    MCU(cudaStreamSynchronize(m->st));
    m->t = 0;
    return TDPD_OK;
}

tdpd_status tdpd_mlp_get_params(tdpd_mlp *m, float *params)
{
    if (!m || !params) return mfail(TDPD_EINVAL, "null argument");
    MCU(cudaMemcpyAsync(params, m->params, (size_t)m->members * NP * sizeof(float), cudaMemcpyDeviceToHost, m->st));
    MCU(cudaStreamSynchronize(m->st));
    return TDPD_OK;
}

tdpd_status tdpd_mlp_set_data(tdpd_mlp *m, int n, const float *X, const float *Y)
{
    if (!m || n < 2 || !X || !Y) return mfail(TDPD_EINVAL, "tdpd_mlp_set_data: need n >= 2 samples");
    tdpd_status rc = alloc_data(m, n);
    if (rc) return rc;
    // standardisation: mean and population deviation of each column
    for (int k = 0; k < IN + OUT; ++k) {
        const float *src = k < IN ? X : Y;
        const int w = k < IN ? IN : OUT, c = k < IN ? k : k - IN;
        double s = 0.0, s2 = 0.0;
        for (int i = 0; i < n; ++i) s += src[(size_t)i * w + c];
        const double mean = s / n;
        for (int i = 0; i < n; ++i) {
            const double d = src[(size_t)i * w + c] - mean;
            s2 += d * d;
        }
        const double sd = std::sqrt(s2 / n) + 1e-12;
        if (k < IN) { m->mx[c] = mean; m->sx[c] = sd; }
        else { m->my[c] = mean; m->sy[c] = sd; }
    }
    std::vector<float> xs((size_t)n * IN), ys((size_t)n * OUT);
    for (int i = 0; i < n; ++i) {
        for (int c = 0; c < IN; ++c) xs[(size_t)i * IN + c] = (float)((X[(size_t)i * IN + c] - m->mx[c]) / m->sx[c]);
        for (int c = 0; c < OUT; ++c) ys[(size_t)i * OUT + c] = (float)((Y[(size_t)i * OUT + c] - m->my[c]) / m->sy[c]);
    }
    MCU(cudaMemcpyAsync(m->X, xs.data(), xs.size() * sizeof(float), cudaMemcpyHostToDevice, m->st));
    MCU(cudaMemcpyAsync(m->T, ys.data(), ys.size() * sizeof(float), cudaMemcpyHostToDevice, m->st));
    MCU(cudaStreamSynchronize(m->st));
    m->n = n;
    m->have_data = true;
    return TDPD_OK;
}

tdpd_status tdpd_mlp_loss_grad(tdpd_mlp *m, double *loss, float *grad)
{
    if (!m || !m->have_data) return mfail(TDPD_ESTATE, "tdpd_mlp_loss_grad: no data set");
    tdpd_status rc = pass(m, 0.0f, loss);
    if (rc) return rc;
    if (grad) {
        MCU(cudaMemcpyAsync(grad, m->grad, (size_t)m->members * NP * sizeof(float), cudaMemcpyDeviceToHost, m->st));
        MCU(cudaStreamSynchronize(m->st));
    }
    return TDPD_OK;
}

tdpd_status tdpd_mlp_train(tdpd_mlp *m, int steps, float lr, double *loss)
{
    if (!m || !m->have_data) return mfail(TDPD_ESTATE, "tdpd_mlp_train: no data set");
    if (steps < 0 || !(lr > 0)) return mfail(TDPD_EINVAL, "tdpd_mlp_train: steps >= 0, lr > 0");
    for (int k = 0; k < steps; ++k) {
        tdpd_status rc = pass(m, lr, nullptr);
        if (rc) return rc;
    }
    if (loss) return pass(m, 0.0f, loss);
    MCU(cudaStreamSynchronize(m->st));
    return TDPD_OK;
}

tdpd_status tdpd_mlp_predict(tdpd_mlp *m, int n, const float *X, float *mean, float *rel_spread, float *member_out)
{
    if (!m || n < 1 || !X || !mean) return mfail(TDPD_EINVAL, "tdpd_mlp_predict: bad arguments");
    if (!m->have_data) return mfail(TDPD_ESTATE, "tdpd_mlp_predict: no standardisation (set data first)");
    // prediction buffers: reuse the training buffers when large enough
    float *dX = nullptr, *dY = nullptr;
    MCU(cudaMallocAsync((void **)&dX, (size_t)n * IN * sizeof(float), m->st));
    MCU(cudaMallocAsync((void **)&dY, (size_t)m->members * n * OUT * sizeof(float), m->st));
    std::vector<float> xs((size_t)n * IN), ys((size_t)m->members * n * OUT);
    for (int i = 0; i < n; ++i)
        for (int c = 0; c < IN; ++c) xs[(size_t)i * IN + c] = (float)((X[(size_t)i * IN + c] - m->mx[c]) / m->sx[c]);
    MCU(cudaMemcpyAsync(dX, xs.data(), xs.size() * sizeof(float), cudaMemcpyHostToDevice, m->st));
    k_mlp_fwd<<<dim3((n + TPB - 1) / TPB, m->members), TPB, 0, m->st>>>(m->params, dX, n, dY);
    MCU(cudaGetLastError());
    MCU(cudaMemcpyAsync(ys.data(), dY, ys.size() * sizeof(float), cudaMemcpyDeviceToHost, m->st));
    MCU(cudaFreeAsync(dX, m->st));
    MCU(cudaFreeAsync(dY, m->st));
    MCU(cudaStreamSynchronize(m->st));
    const int M = m->members;
    for (int i = 0; i < n; ++i)
        for (int c = 0; c < OUT; ++c) {
            double s = 0.0, s2 = 0.0;
            for (int k = 0; k < M; ++k) {
                const double y = ys[((size_t)k * n + i) * OUT + c] * m->sy[c] + m->my[c];
                if (member_out) member_out[((size_t)k * n + i) * OUT + c] = (float)y;
                s += y;
                s2 += y * y;
            }
            const double mu = s / M;
            const double var = M > 1 ? std::max(0.0, (s2 - M * mu * mu) / (M - 1)) : 0.0;
            mean[(size_t)i * OUT + c] = (float)mu;
            if (rel_spread) rel_spread[(size_t)i * OUT + c] = (float)(std::sqrt(var) / std::max(std::fabs(mu), 1e-30));
        }
    return TDPD_OK;
}

void tdpd_mlp_destroy(tdpd_mlp *m)
{
    if (!m) return;
    cudaStreamSynchronize(m->st);
    free_data(m);
    cudaFree(m->params);
    cudaFree(m->m);
    cudaFree(m->v);
    cudaFree(m->grad);
    cudaStreamDestroy(m->st);
    delete m;
}

}  // extern "C"
