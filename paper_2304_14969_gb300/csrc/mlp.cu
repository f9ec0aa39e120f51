// Proposal network for the approximate mode: nfeat -> H -> H -> 1 logit,
// ReLU, binary cross-entropy on "this check rounds" labels.
//
// Not part of arXiv 2304.14969 itself: it ranks which qubits of a
// subsystem are worth a Bloch reduction (Sec. III.A step 1) before the
// exhaustive check. FP32 master weights; inference reads BF16 copies with
// FP32 accumulation. Training is one fused forward+backward kernel that
// writes per-CTA gradient partials, then one kernel that sums them in FP32,
// reports the mean loss and applies Adam.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>

#include "qsim_internal.h"

struct qsim_mlp {
    int nf = 0, H = 0;
    int64_t np = 0;
    float *w = nullptr;        // master parameters (device)
    __nv_bfloat16 *wb = nullptr;  // BF16 copies (device)
    float *m = nullptr, *v = nullptr;  // Adam moments
    float *partial = nullptr;  // [kMlpBlocks][np + 1]
    float *dx = nullptr, *dy = nullptr, *dout = nullptr;
    size_t xcap = 0;
    int64_t step = 0;
};

namespace qs {

static const int kMlpBlocks = 64;
static const int kMlpThreads = 128;
static const int kMaxH = 64;
static const int kMaxF = 32;

struct MlpLayout {
    int nf, H;
    int w1, b1, w2, b2, w3, b3, np;
};

__host__ __device__ inline MlpLayout mlp_layout(int nf, int H)
{
    MlpLayout L;
    L.nf = nf;
    L.H = H;
    L.w1 = 0;
    L.b1 = L.w1 + H * nf;
    L.w2 = L.b1 + H;
    L.b2 = L.w2 + H * H;
    L.w3 = L.b2 + H;
    L.b3 = L.w3 + H;
    L.np = L.b3 + 1;
    return L;
}

// Inference: one thread per row, weights read from global (L1-resident).
template <bool BF16>
__global__ void k_mlp_infer(const float *__restrict__ w, const __nv_bfloat16 *__restrict__ wb, int nf, int H,
                            const float *__restrict__ x, int rows, float *__restrict__ out)
{
    MlpLayout L = mlp_layout(nf, H);
    auto W = [&](int i) -> float { return BF16 ? __bfloat162float(wb[i]) : w[i]; };
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += gridDim.x * blockDim.x) {
        float h1[kMaxH], h2[kMaxH];
        const float *xr = x + (size_t)r * nf;
        for (int j = 0; j < H; j++) {
            float s = W(L.b1 + j);
            for (int i = 0; i < nf; i++) s = fmaf(W(L.w1 + j * nf + i), xr[i], s);
            h1[j] = fmaxf(s, 0.f);
        }
        for (int j = 0; j < H; j++) {
            float s = W(L.b2 + j);
            for (int i = 0; i < H; i++) s = fmaf(W(L.w2 + j * H + i), h1[i], s);
            h2[j] = fmaxf(s, 0.f);
        }
        float z = W(L.b3);
        for (int i = 0; i < H; i++) z = fmaf(W(L.w3 + i), h2[i], z);
        out[r] = z;
    }
}

// Forward + backward of the mean BCE-with-logits loss. CTA b accumulates
// the gradient of its rows in shared memory and writes partial[b][0..np)
// plus its loss sum at partial[b][np].
__global__ void k_mlp_grad(const float *__restrict__ w, int nf, int H, const float *__restrict__ x,
                           const float *__restrict__ y, int rows, float *__restrict__ partial)
{
    MlpLayout L = mlp_layout(nf, H);
    extern __shared__ float g[];   // np + 1
    for (int i = threadIdx.x; i < L.np + 1; i += blockDim.x) g[i] = 0.f;
    __syncthreads();
    const float inv = 1.0f / (float)rows;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += gridDim.x * blockDim.x) {
        float a1[kMaxH], a2[kMaxH], d2[kMaxH];
        const float *xr = x + (size_t)r * nf;
        for (int j = 0; j < H; j++) {
            float s = w[L.b1 + j];
            for (int i = 0; i < nf; i++) s = fmaf(w[L.w1 + j * nf + i], xr[i], s);
            a1[j] = fmaxf(s, 0.f);
        }
        for (int j = 0; j < H; j++) {
            float s = w[L.b2 + j];
            for (int i = 0; i < H; i++) s = fmaf(w[L.w2 + j * H + i], a1[i], s);
            a2[j] = fmaxf(s, 0.f);
        }
        float z = w[L.b3];
        for (int i = 0; i < H; i++) z = fmaf(w[L.w3 + i], a2[i], z);
        // BCE with logits: softplus(z) - y z; d/dz = sigmoid(z) - y
        float yr = y[r];
        float loss = fmaxf(z, 0.f) - z * yr + log1pf(expf(-fabsf(z)));
        float dz = (1.0f / (1.0f + expf(-z)) - yr) * inv;
        atomicAdd(&g[L.np], loss);
        atomicAdd(&g[L.b3], dz);
        for (int i = 0; i < H; i++) {
            atomicAdd(&g[L.w3 + i], dz * a2[i]);
            d2[i] = a2[i] > 0.f ? dz * w[L.w3 + i] : 0.f;
        }
        for (int j = 0; j < H; j++) {
            if (d2[j] == 0.f) continue;
            atomicAdd(&g[L.b2 + j], d2[j]);
            for (int i = 0; i < H; i++) atomicAdd(&g[L.w2 + j * H + i], d2[j] * a1[i]);
        }
        for (int i = 0; i < H; i++) {
            if (a1[i] <= 0.f) continue;
            float d1 = 0.f;
            for (int j = 0; j < H; j++) d1 = fmaf(d2[j], w[L.w2 + j * H + i], d1);
            atomicAdd(&g[L.b1 + i], d1);
            for (int k = 0; k < nf; k++) atomicAdd(&g[L.w1 + i * nf + k], d1 * xr[k]);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < L.np + 1; i += blockDim.x) partial[(size_t)blockIdx.x * (L.np + 1) + i] = g[i];
}

// Sums the partials; mode 0 writes the gradient and loss, mode 1 applies
// an Adam step (beta1 0.9, beta2 0.999, eps 1e-8) and refreshes the BF16
// copies.
__global__ void k_mlp_reduce(const float *__restrict__ partial, int blocks, int np, float *__restrict__ grad_out,
                             float *__restrict__ loss_out, int rows, int mode, float *__restrict__ w,
                             __nv_bfloat16 *__restrict__ wb, float *__restrict__ m, float *__restrict__ v, float lr,
                             float c1, float c2)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= np; i += gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int b = 0; b < blocks; b++) s += partial[(size_t)b * (np + 1) + i];
        if (i == np) {
            *loss_out = s / (float)rows;
            continue;
        }
        if (mode == 0) {
            grad_out[i] = s;
            continue;
        }
        float mi = 0.9f * m[i] + 0.1f * s;
        float vi = 0.999f * v[i] + 0.001f * s * s;
        m[i] = mi;
        v[i] = vi;
        float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
        w[i] = wi;
        wb[i] = __float2bfloat16(wi);
    }
}

__global__ void k_to_bf16(const float *__restrict__ w, __nv_bfloat16 *__restrict__ wb, int np)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += gridDim.x * blockDim.x) wb[i] = __float2bfloat16(w[i]);
}

static qsim_status ensure_io(qsim_mlp *m, int rows)
{
    size_t need = (size_t)rows;
    if (need <= m->xcap) return QSIM_OK;
    if (m->dx) cudaFree(m->dx);
    if (m->dy) cudaFree(m->dy);
    if (m->dout) cudaFree(m->dout);
    m->dx = m->dy = m->dout = nullptr;
    size_t cap = std::max<size_t>(need, 1024);
    QS_CUDA(cudaMalloc(&m->dx, cap * m->nf * sizeof(float)));
    QS_CUDA(cudaMalloc(&m->dy, cap * sizeof(float)));
    QS_CUDA(cudaMalloc(&m->dout, (cap + m->np + 1) * sizeof(float)));
    m->xcap = cap;
    return QSIM_OK;
}

// Device inference on device features (used by the approximate mode).
qsim_status mlp_infer_device(const qsim_mlp *m, const float *d_x, int rows, float *d_out, cudaStream_t st)
{
    int grid = std::max(1, std::min(64, (rows + 127) / 128));
    k_mlp_infer<true><<<grid, 128, 0, st>>>(m->w, m->wb, m->nf, m->H, d_x, rows, d_out);
    QS_CUDA(cudaGetLastError());
    return QSIM_OK;
}

int mlp_nfeat(const qsim_mlp *m) { return m->nf; }

}  // namespace qs

using namespace qs;

extern "C" {

qsim_status qsim_mlp_create(int nfeat, int hidden, uint64_t seed, qsim_mlp **out)
{
    clear_error();
    if (!out) return fail(QSIM_E_INVAL, "out is NULL");
    *out = nullptr;
    if (nfeat < 1 || nfeat > kMaxF) return fail(QSIM_E_INVAL, "nfeat %d outside [1, %d]", nfeat, kMaxF);
    if (hidden < 1 || hidden > kMaxH) return fail(QSIM_E_INVAL, "hidden %d outside [1, %d]", hidden, kMaxH);
    qsim_mlp *m = new qsim_mlp();
    m->nf = nfeat;
    m->H = hidden;
    MlpLayout L = mlp_layout(nfeat, hidden);
    m->np = L.np;
    // He-uniform initialisation from a seeded host generator, biases zero
    std::vector<float> h(L.np, 0.f);
    std::mt19937_64 rng(seed);
    auto fill = [&](int off, int count, int fan_in) {
        float a = std::sqrt(6.0f / (float)fan_in);
        std::uniform_real_distribution<float> U(-a, a);
        for (int i = 0; i < count; i++) h[off + i] = U(rng);
    };
    fill(L.w1, hidden * nfeat, nfeat);
    fill(L.w2, hidden * hidden, hidden);
    fill(L.w3, hidden, hidden);
    cudaError_t e = cudaMalloc(&m->w, L.np * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&m->wb, L.np * sizeof(__nv_bfloat16));
    if (e == cudaSuccess) e = cudaMalloc(&m->m, L.np * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&m->v, L.np * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&m->partial, (size_t)kMlpBlocks * (L.np + 1) * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(m->m, 0, L.np * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(m->v, 0, L.np * sizeof(float));
    if (e != cudaSuccess) {
        qsim_mlp_destroy(m);
        return cuda_fail(e, "mlp alloc");
    }
    *out = m;
    return qsim_mlp_set_params(m, h.data());
}

qsim_status qsim_mlp_destroy(qsim_mlp *m)
{
    if (!m) return QSIM_OK;
    cudaDeviceSynchronize();
    for (void *p : {(void *)m->w, (void *)m->wb, (void *)m->m, (void *)m->v, (void *)m->partial, (void *)m->dx,
                    (void *)m->dy, (void *)m->dout})
        if (p) cudaFree(p);
    delete m;
    return QSIM_OK;
}

qsim_status qsim_mlp_num_params(const qsim_mlp *m, int64_t *count)
{
    clear_error();
    if (!m || !count) return fail(QSIM_E_INVAL, "NULL argument");
    *count = m->np;
    return QSIM_OK;
}

qsim_status qsim_mlp_get_params(const qsim_mlp *m, float *host)
{
    clear_error();
    if (!m || !host) return fail(QSIM_E_INVAL, "NULL argument");
    QS_CUDA(cudaMemcpy(host, m->w, m->np * sizeof(float), cudaMemcpyDeviceToHost));
    return QSIM_OK;
}

qsim_status qsim_mlp_set_params(qsim_mlp *m, const float *host)
{
    clear_error();
    if (!m || !host) return fail(QSIM_E_INVAL, "NULL argument");
    QS_CUDA(cudaMemcpy(m->w, host, m->np * sizeof(float), cudaMemcpyHostToDevice));
    k_to_bf16<<<4, 256>>>(m->w, m->wb, (int)m->np);
    QS_CUDA(cudaGetLastError());
    QS_CUDA(cudaDeviceSynchronize());
    return QSIM_OK;
}

qsim_status qsim_mlp_infer(qsim_mlp *m, const float *host_x, int rows, int bf16, float *host_logits)
{
    clear_error();
    if (!m || !host_x || !host_logits || rows < 0) return fail(QSIM_E_INVAL, "bad argument");
    if (rows == 0) return QSIM_OK;
    QS_TRY(ensure_io(m, rows));
    QS_CUDA(cudaMemcpy(m->dx, host_x, (size_t)rows * m->nf * sizeof(float), cudaMemcpyHostToDevice));
    int grid = std::max(1, std::min(64, (rows + 127) / 128));
    if (bf16) k_mlp_infer<true><<<grid, 128>>>(m->w, m->wb, m->nf, m->H, m->dx, rows, m->dout);
    else k_mlp_infer<false><<<grid, 128>>>(m->w, m->wb, m->nf, m->H, m->dx, rows, m->dout);
    QS_CUDA(cudaGetLastError());
    QS_CUDA(cudaMemcpy(host_logits, m->dout, rows * sizeof(float), cudaMemcpyDeviceToHost));
    return QSIM_OK;
}

static qsim_status mlp_pass(qsim_mlp *m, const float *host_x, const float *host_y, int rows, int mode, float lr,
                            float *loss, float *host_grad)
{
    if (!m || !host_x || !host_y || rows < 1) return fail(QSIM_E_INVAL, "bad argument");
    QS_TRY(ensure_io(m, rows));
    QS_CUDA(cudaMemcpy(m->dx, host_x, (size_t)rows * m->nf * sizeof(float), cudaMemcpyHostToDevice));
    QS_CUDA(cudaMemcpy(m->dy, host_y, rows * sizeof(float), cudaMemcpyHostToDevice));
    int blocks = std::max(1, std::min(kMlpBlocks, (rows + kMlpThreads - 1) / kMlpThreads));
    size_t smem = (m->np + 1) * sizeof(float);
    k_mlp_grad<<<blocks, kMlpThreads, smem>>>(m->w, m->nf, m->H, m->dx, m->dy, rows, m->partial);
    QS_CUDA(cudaGetLastError());
    float c1 = 1.f, c2 = 1.f;
    if (mode == 1) {
        m->step++;
        c1 = 1.f - std::pow(0.9f, (float)m->step);
        c2 = 1.f - std::pow(0.999f, (float)m->step);
    }
    float *gout = m->dout, *lout = m->dout + m->np;
    k_mlp_reduce<<<8, 256>>>(m->partial, blocks, (int)m->np, gout, lout, rows, mode, m->w, m->wb, m->m, m->v, lr,
                             c1, c2);
    QS_CUDA(cudaGetLastError());
    if (loss) QS_CUDA(cudaMemcpy(loss, lout, sizeof(float), cudaMemcpyDeviceToHost));
    if (host_grad) QS_CUDA(cudaMemcpy(host_grad, gout, m->np * sizeof(float), cudaMemcpyDeviceToHost));
    QS_CUDA(cudaDeviceSynchronize());
    return QSIM_OK;
}

qsim_status qsim_mlp_loss_grad(qsim_mlp *m, const float *host_x, const float *host_y, int rows, float *loss,
                               float *host_grad)
{
    clear_error();
    if (!host_grad) return fail(QSIM_E_INVAL, "host_grad is NULL");
    return mlp_pass(m, host_x, host_y, rows, 0, 0.f, loss, host_grad);
}

qsim_status qsim_mlp_train_step(qsim_mlp *m, const float *host_x, const float *host_y, int rows, float lr,
                                float *loss)
{
    clear_error();
    if (!(lr > 0)) return fail(QSIM_E_INVAL, "lr must be positive");
    return mlp_pass(m, host_x, host_y, rows, 1, lr, loss, nullptr);
}

}  // extern "C"
