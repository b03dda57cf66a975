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

// Forward pass of one sample per thread. With TRAIN, keeps the pre- and
// post-activations, the output error signal dL/dy and per-block loss sums.
template <bool TRAIN>
__global__ void __launch_bounds__(TPB) k_mlp_fwd(const float *__restrict__ params, const float *__restrict__ X,
                                                 const float *__restrict__ T, int n, float *Z1, float *H1,
                                                 float *Z2, float *H2, float *D3, float *Y, float *loss_part)
{
    __shared__ float w[NP];
    __shared__ float red[TPB / 32];
    const int mbr = blockIdx.y;
    load_weights(w, params + (size_t)mbr * NP);
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    float err2 = 0.0f;
    if (s < n) {
        float x[IN];
#pragma unroll
        for (int i = 0; i < IN; ++i) x[i] = X[(size_t)s * IN + i];
        const size_t base = ((size_t)mbr * n + s) * HID;
        float h1[HID];
#pragma unroll
        for (int o = 0; o < HID; ++o) {
            float z = w[OB1 + o];
#pragma unroll
            for (int i = 0; i < IN; ++i) z = fmaf(w[OW1 + o * IN + i], x[i], z);
            h1[o] = gelu(z);
            if (TRAIN) {
                Z1[base + o] = z;
                H1[base + o] = h1[o];
            }
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
                const int o = o0 + q;
                const float h = gelu(z[q]);
                if (TRAIN) {
                    Z2[base + o] = z[q];
                    H2[base + o] = h;
                }
                y0 = fmaf(w[OW3 + o], h, y0);
                y1 = fmaf(w[OW3 + HID + o], h, y1);
            }
        }
        const size_t yo = ((size_t)mbr * n + s) * OUT;
        Y[yo] = y0;
        Y[yo + 1] = y1;
        if (TRAIN) {
            const float e0 = y0 - T[(size_t)s * OUT], e1 = y1 - T[(size_t)s * OUT + 1];
            const float sc = 2.0f / (float)(n * OUT);
            D3[yo] = sc * e0;
            D3[yo + 1] = sc * e1;
            err2 = e0 * e0 + e1 * e1;
        }
    }
    if (TRAIN) {
        for (int o = 16; o > 0; o >>= 1) err2 += __shfl_down_sync(0xffffffffu, err2, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = err2;
        __syncthreads();
        if (threadIdx.x == 0) {
            float t = 0.0f;
            for (int k = 0; k < TPB / 32; ++k) t += red[k];
            loss_part[(size_t)mbr * gridDim.x + blockIdx.x] = t;
        }
    }
}

// Back-propagated error signals of the two hidden layers, one sample per thread.
__global__ void __launch_bounds__(TPB) k_mlp_delta(const float *__restrict__ params, const float *__restrict__ Z1,
                                                   const float *__restrict__ Z2, const float *__restrict__ D3,
                                                   int n, float *D2, float *D1)
{
    __shared__ float w[NP];
    const int mbr = blockIdx.y;
    load_weights(w, params + (size_t)mbr * NP);
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const size_t base = ((size_t)mbr * n + s) * HID;
    const size_t yo = ((size_t)mbr * n + s) * OUT;
    const float d30 = D3[yo], d31 = D3[yo + 1];
    float d2[HID];
#pragma unroll
    for (int o = 0; o < HID; ++o) {
        const float g = fmaf(d30, w[OW3 + o], d31 * w[OW3 + HID + o]);
        d2[o] = g * gelu_grad(Z2[base + o]);
        D2[base + o] = d2[o];
    }
    for (int i0 = 0; i0 < HID; i0 += 4) {
        float a[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int o = 0; o < HID; ++o)
#pragma unroll
            for (int q = 0; q < 4; ++q) a[q] = fmaf(d2[o], w[OW2 + o * HID + i0 + q], a[q]);
#pragma unroll
        for (int q = 0; q < 4; ++q) D1[base + i0 + q] = a[q] * gelu_grad(Z1[base + i0 + q]);
    }
}

// Gradient of one parameter per thread, in two passes: each CTA row c sums
// the samples [c GCH, (c+1) GCH) in sample order (float-float compensated,
// the loads of several samples in flight), then k_mlp_grad_sum adds the
// chunks' partial sums in chunk order. The order is fixed, so the gradient
// is deterministic.
constexpr int GCH = 128;

__global__ void __launch_bounds__(TPB) k_mlp_grad_part(const float *__restrict__ X, const float *__restrict__ H1,
                                                       const float *__restrict__ H2, const float *__restrict__ D1,
                                                       const float *__restrict__ D2, const float *__restrict__ D3,
                                                       int n, float2 *part)
{
    const int mbr = blockIdx.z, c = blockIdx.y;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NP) return;
    const float *A = nullptr, *Bv = nullptr;   // gradient = sum_s A[s][ra] * Bv[s][rb] (Bv null: 1)
    int ra = 0, rb = 0, wa = HID, wb = HID;
    size_t oa = (size_t)mbr * n * HID, ob = (size_t)mbr * n * HID;
    if (p < OB1) { A = D1; ra = (p - OW1) / IN; Bv = X; rb = (p - OW1) % IN; wb = IN; ob = 0; }
    else if (p < OW2) { A = D1; ra = p - OB1; }
    else if (p < OB2) { A = D2; ra = (p - OW2) / HID; Bv = H1; rb = (p - OW2) % HID; }
    else if (p < OW3) { A = D2; ra = p - OB2; }
    else if (p < OB3) { A = D3; wa = OUT; oa = (size_t)mbr * n * OUT; ra = (p - OW3) / HID; Bv = H2; rb = (p - OW3) % HID; }
    else { A = D3; wa = OUT; oa = (size_t)mbr * n * OUT; ra = p - OB3; }
    const int s0 = c * GCH, s1 = min(n, s0 + GCH);
    FF acc{0.0f, 0.0f};
    if (Bv) {
#pragma unroll 8
        for (int s = s0; s < s1; ++s)
            acc = ff_add(acc, A[oa + (size_t)s * wa + ra] * Bv[ob + (size_t)s * wb + rb]);
    } else {
#pragma unroll 8
        for (int s = s0; s < s1; ++s) acc = ff_add(acc, A[oa + (size_t)s * wa + ra]);
    }
    part[((size_t)mbr * gridDim.y + c) * NP + p] = make_float2(acc.hi, acc.lo);
}

__global__ void __launch_bounds__(TPB) k_mlp_grad_sum(const float2 *__restrict__ part, int nch, float *grad)
{
    const int mbr = blockIdx.y;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NP) return;
    FF acc{0.0f, 0.0f};
    for (int c = 0; c < nch; ++c) {
        const float2 q = part[((size_t)mbr * nch + c) * NP + p];
        acc = ff_add(acc, FF{q.x, q.y});
    }
    grad[(size_t)mbr * NP + p] = acc.hi + acc.lo;
}

// Adam (Kingma & Ba) on the float master weights; bc1, bc2 are the bias
// corrections 1 - beta^t.
__global__ void k_mlp_adam(float *params, const float *__restrict__ grad, float *m, float *v, int total, float lr,
                           float beta1, float beta2, float eps, float bc1, float bc2)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= total) return;
    const float g = grad[k];
    const float mk = fmaf(beta1, m[k], (1.0f - beta1) * g);
    const float vk = fmaf(beta2, v[k], (1.0f - beta2) * g * g);
    m[k] = mk;
    v[k] = vk;
    params[k] -= lr * (mk / bc1) / (sqrtf(vk / bc2) + eps);
}

}  // namespace

struct tdpd_mlp {
    int members = 0, n = 0, cap = 0;
    int64_t t = 0;
    float *params = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
    float *X = nullptr, *T = nullptr, *Z1 = nullptr, *H1 = nullptr, *Z2 = nullptr, *H2 = nullptr;
    float *D1 = nullptr, *D2 = nullptr, *D3 = nullptr, *Y = nullptr, *loss_part = nullptr;
    float *gpart = nullptr;     // [members][chunks][NP] float-float partial gradients
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
    const size_t M = m->members;
    float **bufs[] = {&m->X, &m->T, &m->Z1, &m->H1, &m->Z2, &m->H2, &m->D1, &m->D2, &m->D3, &m->Y, &m->loss_part,
                      &m->gpart};
    const size_t sizes[] = {(size_t)n * IN, (size_t)n * OUT, M * n * HID, M * n * HID, M * n * HID, M * n * HID,
                            M * n * HID, M * n * HID, M * n * OUT, M * n * OUT, M * ((n + TPB - 1) / TPB),
                            2 * M * ((n + GCH - 1) / GCH) * NP};
    for (int k = 0; k < 12; ++k) {
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

tdpd_status forward_backward(tdpd_mlp *m, double *loss)
{
    const dim3 gs((m->n + TPB - 1) / TPB, m->members);
    k_mlp_fwd<true><<<gs, TPB, 0, m->st>>>(m->params, m->X, m->T, m->n, m->Z1, m->H1, m->Z2, m->H2, m->D3, m->Y,
                                           m->loss_part);
    k_mlp_delta<<<gs, TPB, 0, m->st>>>(m->params, m->Z1, m->Z2, m->D3, m->n, m->D2, m->D1);
    const int nch = (m->n + GCH - 1) / GCH;
    k_mlp_grad_part<<<dim3((NP + TPB - 1) / TPB, nch, m->members), TPB, 0, m->st>>>(
        m->X, m->H1, m->H2, m->D1, m->D2, m->D3, m->n, reinterpret_cast<float2 *>(m->gpart));
    k_mlp_grad_sum<<<dim3((NP + TPB - 1) / TPB, m->members), TPB, 0, m->st>>>(
        reinterpret_cast<const float2 *>(m->gpart), nch, m->grad);
    MCU(cudaGetLastError());
    if (loss) {
        const int nb = (m->n + TPB - 1) / TPB;
        std::vector<float> part((size_t)m->members * nb);
        MCU(cudaMemcpyAsync(part.data(), m->loss_part, part.size() * sizeof(float), cudaMemcpyDeviceToHost, m->st));
        MCU(cudaStreamSynchronize(m->st));
        for (int k = 0; k < m->members; ++k) {
            double s = 0.0;
            for (int b = 0; b < nb; ++b) s += part[(size_t)k * nb + b];
            loss[k] = s / ((double)m->n * OUT);
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
    tdpd_status rc = forward_backward(m, loss);
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
    const float beta1 = 0.9f, beta2 = 0.999f, eps = 1e-8f;
    const int total = m->members * NP;
    for (int k = 0; k < steps; ++k) {
        tdpd_status rc = forward_backward(m, nullptr);
        if (rc) return rc;
        ++m->t;
        const float bc1 = (float)(1.0 - std::pow(0.9, (double)m->t));
        const float bc2 = (float)(1.0 - std::pow(0.999, (double)m->t));
        k_mlp_adam<<<(total + 255) / 256, 256, 0, m->st>>>(m->params, m->grad, m->m, m->v, total, lr, beta1, beta2,
                                                           eps, bc1, bc2);
    }
    MCU(cudaGetLastError());
    if (loss) return forward_backward(m, loss);
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
    k_mlp_fwd<false><<<dim3((n + TPB - 1) / TPB, m->members), TPB, 0, m->st>>>(
        m->params, dX, nullptr, n, nullptr, nullptr, nullptr, nullptr, nullptr, dY, nullptr);
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
