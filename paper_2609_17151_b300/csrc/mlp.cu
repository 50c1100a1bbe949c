// mlp.cu -- the learned warm start's network: a 3-layer MLP trained and run on
// the GPU with BF16 tensor-core products and FP32 accumulation.
//
// Layers: n_in -> h (GELU) -> h (GELU) -> n_out (linear).  FP32 master
// weights; every product takes BF16-rounded operands through the warp-level
// tensor-core MMA (m16n8k16, FP32 accumulators).  The matrices are small
// (at most a few hundred rows), so each warp owns one 16 x 16 output tile and
// streams its operands straight from global memory (L1/L2-resident).
// Inputs are scaled to [-1, 1] by their ranges, outputs standardised by the
// training set's mean and deviation; both transforms run on the device.
#include "pic1d3v.h"

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

namespace pic {
void set_last_error(const std::string &msg);
}

namespace {

pic_status mlp_fail(pic_status s, const std::string &m)
{
    pic::set_last_error(m);
    return s;
}

#define MCU(call)                                                                                   \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess) return mlp_fail(PIC_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

// C = alpha * A B (+ C if accumulate), A(i,k) = A[i*ar + k*ac], B(k,j) = B[k*br + j*bc],
// C(i,j) = C[i*ldc + j]; one warp per 16x16 tile of C, K in steps of 16.
__global__ void k_gemm_bf16(const float *__restrict__ A, int ar, int ac, const float *__restrict__ B, int br, int bc,
                            float *__restrict__ C, int ldc, int M, int N, int K, float alpha, int accumulate)
{
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int tiles_n = (N + 15) / 16;
    const int tm = warp / tiles_n, tn = warp % tiles_n;
    if (tm * 16 >= M) return;
    const int g = lane >> 2, t = lane & 3;
    auto a_at = [&](int i, int k) -> float { return (i < M && k < K) ? A[(size_t)i * ar + (size_t)k * ac] : 0.0f; };
    auto b_at = [&](int k, int j) -> float { return (k < K && j < N) ? B[(size_t)k * br + (size_t)j * bc] : 0.0f; };
    float acc[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
    const int i0 = tm * 16, j0 = tn * 16;
    for (int k0 = 0; k0 < K; k0 += 16) {
        const uint32_t a0 = pack_bf16(a_at(i0 + g, k0 + 2 * t), a_at(i0 + g, k0 + 2 * t + 1));
        const uint32_t a1 = pack_bf16(a_at(i0 + g + 8, k0 + 2 * t), a_at(i0 + g + 8, k0 + 2 * t + 1));
        const uint32_t a2 = pack_bf16(a_at(i0 + g, k0 + 2 * t + 8), a_at(i0 + g, k0 + 2 * t + 9));
        const uint32_t a3 = pack_bf16(a_at(i0 + g + 8, k0 + 2 * t + 8), a_at(i0 + g + 8, k0 + 2 * t + 9));
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int jn = j0 + 8 * h + g;
            const uint32_t b0 = pack_bf16(b_at(k0 + 2 * t, jn), b_at(k0 + 2 * t + 1, jn));
            const uint32_t b1 = pack_bf16(b_at(k0 + 2 * t + 8, jn), b_at(k0 + 2 * t + 9, jn));
            asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
                         "{%8,%9}, {%0,%1,%2,%3};\n"
                         : "+f"(acc[h][0]), "+f"(acc[h][1]), "+f"(acc[h][2]), "+f"(acc[h][3])
                         : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
        }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = i0 + g + (q >= 2 ? 8 : 0);
            const int j = j0 + 8 * h + 2 * t + (q & 1);
            if (i < M && j < N) {
                float *c = C + (size_t)i * ldc + j;
                *c = accumulate ? *c + alpha * acc[h][q] : alpha * acc[h][q];
            }
        }
}

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x)
{
    return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

// Z += bias (per column); H = GELU(Z) if act, else H = Z
__global__ void k_bias_act(float *Z, float *H, const float *bias, int M, int N, int act)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= M * N) return;
    const float z = Z[idx] + bias[idx % N];
    Z[idx] = z;
    H[idx] = act ? gelu(z) : z;
}

// dZ = dH * GELU'(Z)
__global__ void k_act_grad(const float *Z, const float *dH, float *dZ, int n)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < n) dZ[idx] = dH[idx] * gelu_grad(Z[idx]);
}

// column sums: db[j] = sum_i dZ[i, j]
__global__ void k_colsum(const float *dZ, float *db, int M, int N)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    float s = 0.0f;
    for (int i = 0; i < M; ++i) s += dZ[(size_t)i * N + j];
    db[j] = s;
}

// dY = 2 (Y - T) / (M N); per-block partial sums of (Y - T)^2
__global__ void k_mse(const float *Y, const float *T, float *dY, float *part, int n, float scale)
{
    __shared__ float red[256];
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    float e = 0.0f;
    if (idx < n) {
        const float d = Y[idx] - T[idx];
        dY[idx] = 2.0f * d * scale;
        e = d * d;
    }
    red[threadIdx.x] = e;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// Adam (Kingma & Ba): m, v moving moments of the gradient, bias-corrected step
__global__ void k_adam(float *w, const float *g, float *m, float *v, int n, float lr, float b1, float b2, float eps,
                       float c1, float c2)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    const float gi = g[idx];
    const float mi = b1 * m[idx] + (1.0f - b1) * gi;
    const float vi = b2 * v[idx] + (1.0f - b2) * gi * gi;
    m[idx] = mi;
    v[idx] = vi;
    w[idx] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
}

// X_n = 2 (X - lo) / (hi - lo) - 1 (per column)
__global__ void k_norm_in(const float *X, float *Xn, const float *lo, const float *hi, int M, int N)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= M * N) return;
    const int j = idx % N;
    Xn[idx] = 2.0f * (X[idx] - lo[j]) / (hi[j] - lo[j]) - 1.0f;
}

// Y_n = (Y - mean) / std  (forward = 1) or Y = Y_n std + mean (forward = 0)
__global__ void k_norm_out(const float *in, float *out, const float *mean, const float *sd, int M, int N, int forward)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= M * N) return;
    const int j = idx % N;
    out[idx] = forward ? (in[idx] - mean[j]) / sd[j] : in[idx] * sd[j] + mean[j];
}

// Deterministic initialisation: uniform(-s, s) from a 64-bit counter hash
// (SplitMix64), s = sqrt(6 / (fan_in + fan_out)) (Glorot).
__global__ void k_init(float *w, int n, float s, uint64_t seed)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    uint64_t z = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(idx + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const float u = (float)(z >> 40) * (1.0f / 16777216.0f);
    w[idx] = s * (2.0f * u - 1.0f);
}

int blocks(long long n, int t = 256) { return (int)((n + t - 1) / t); }

} // namespace

struct pic_mlp {
    int n_in = 0, h = 0, n_out = 0;
    cudaStream_t stream = nullptr;
    // parameters, packed W1 b1 W2 b2 W3 b3 (FP32); gradient and Adam moments alike
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
    size_t n_par = 0;
    size_t off[6] = {};
    long long adam_t = 0;
    float *in_lo = nullptr, *in_hi = nullptr, *out_mean = nullptr, *out_sd = nullptr;
    // activations for a batch of up to cap rows
    int cap = 0;
    float *X = nullptr, *Xn = nullptr, *Z1 = nullptr, *H1 = nullptr, *Z2 = nullptr, *H2 = nullptr, *Y = nullptr,
          *T = nullptr, *dY = nullptr, *dH = nullptr, *dZ = nullptr, *part = nullptr;
};

namespace {

float *W(pic_mlp *m, int l) { return m->p + m->off[2 * l]; }
float *Bv(pic_mlp *m, int l) { return m->p + m->off[2 * l + 1]; }
float *dW(pic_mlp *m, int l) { return m->g + m->off[2 * l]; }
float *dB(pic_mlp *m, int l) { return m->g + m->off[2 * l + 1]; }

void gemm(pic_mlp *m, const float *A, int ar, int ac, const float *B, int br, int bc, float *C, int ldc, int M, int N,
          int K, float alpha, int acc)
{
    const int tiles = ((M + 15) / 16) * ((N + 15) / 16);
    k_gemm_bf16<<<(tiles + 7) / 8, 256, 0, m->stream>>>(A, ar, ac, B, br, bc, C, ldc, M, N, K, alpha, acc);
}

pic_status ensure_batch(pic_mlp *m, int n)
{
    if (n <= m->cap) return PIC_OK;
    float **bufs[] = {&m->X, &m->Xn, &m->Z1, &m->H1, &m->Z2, &m->H2, &m->Y, &m->T, &m->dY, &m->dH, &m->dZ, &m->part};
    for (float **b : bufs) {
        if (*b) cudaFree(*b);
        *b = nullptr;
    }
    const size_t w = (size_t)std::max(std::max(m->n_in, m->h), m->n_out);
    for (float **b : bufs) MCU(cudaMalloc(b, sizeof(float) * (size_t)n * w + 1024 * sizeof(float)));
    m->cap = n;
    return PIC_OK;
}

// forward pass on Xn (n rows, already normalised) -> Y (normalised outputs)
void forward(pic_mlp *m, int n)
{
    const int h = m->h;
    gemm(m, m->Xn, m->n_in, 1, W(m, 0), h, 1, m->Z1, h, n, h, m->n_in, 1.0f, 0);
    k_bias_act<<<blocks((long long)n * h), 256, 0, m->stream>>>(m->Z1, m->H1, Bv(m, 0), n, h, 1);
    gemm(m, m->H1, h, 1, W(m, 1), h, 1, m->Z2, h, n, h, h, 1.0f, 0);
    k_bias_act<<<blocks((long long)n * h), 256, 0, m->stream>>>(m->Z2, m->H2, Bv(m, 1), n, h, 1);
    gemm(m, m->H2, h, 1, W(m, 2), m->n_out, 1, m->Y, m->n_out, n, m->n_out, h, 1.0f, 0);
    k_bias_act<<<blocks((long long)n * m->n_out), 256, 0, m->stream>>>(m->Y, m->Y, Bv(m, 2), n, m->n_out, 0);
}

// gradient of the mean squared error against T (normalised targets) into m->g
void backward(pic_mlp *m, int n)
{
    const int h = m->h, no = m->n_out, ni = m->n_in;
    const int tot = n * no;
    k_mse<<<blocks(tot), 256, 0, m->stream>>>(m->Y, m->T, m->dY, m->part, tot, 1.0f / (float)tot);
    // layer 3
    gemm(m, m->H2, 1, h, m->dY, no, 1, dW(m, 2), no, h, no, n, 1.0f, 0);        // H2^T dY
    k_colsum<<<blocks(no), 256, 0, m->stream>>>(m->dY, dB(m, 2), n, no);
    gemm(m, m->dY, no, 1, W(m, 2), 1, no, m->dH, h, n, h, no, 1.0f, 0);          // dY W3^T
    k_act_grad<<<blocks((long long)n * h), 256, 0, m->stream>>>(m->Z2, m->dH, m->dZ, n * h);
    // layer 2
    gemm(m, m->H1, 1, h, m->dZ, h, 1, dW(m, 1), h, h, h, n, 1.0f, 0);           // H1^T dZ2
    k_colsum<<<blocks(h), 256, 0, m->stream>>>(m->dZ, dB(m, 1), n, h);
    gemm(m, m->dZ, h, 1, W(m, 1), 1, h, m->dH, h, n, h, h, 1.0f, 0);            // dZ2 W2^T
    k_act_grad<<<blocks((long long)n * h), 256, 0, m->stream>>>(m->Z1, m->dH, m->dZ, n * h);
    // layer 1
    gemm(m, m->Xn, 1, ni, m->dZ, h, 1, dW(m, 0), h, ni, h, n, 1.0f, 0);         // Xn^T dZ1
    k_colsum<<<blocks(h), 256, 0, m->stream>>>(m->dZ, dB(m, 0), n, h);
}

pic_status read_loss(pic_mlp *m, int n, float *loss)
{
    const int tot = n * m->n_out;
    const int nb = blocks(tot);
    std::vector<float> part((size_t)nb);
    MCU(cudaMemcpyAsync(part.data(), m->part, nb * sizeof(float), cudaMemcpyDeviceToHost, m->stream));
    MCU(cudaStreamSynchronize(m->stream));
    double s = 0;
    for (float p : part) s += p;
    *loss = (float)(s / tot);
    return PIC_OK;
}

pic_status upload_batch(pic_mlp *m, const float *X, const float *Tgt, int n)
{
    pic_status st = ensure_batch(m, n);
    if (st != PIC_OK) return st;
    MCU(cudaMemcpyAsync(m->X, X, sizeof(float) * (size_t)n * m->n_in, cudaMemcpyHostToDevice, m->stream));
    k_norm_in<<<blocks((long long)n * m->n_in), 256, 0, m->stream>>>(m->X, m->Xn, m->in_lo, m->in_hi, n, m->n_in);
    if (Tgt) {
        MCU(cudaMemcpyAsync(m->dH, Tgt, sizeof(float) * (size_t)n * m->n_out, cudaMemcpyHostToDevice, m->stream));
        k_norm_out<<<blocks((long long)n * m->n_out), 256, 0, m->stream>>>(m->dH, m->T, m->out_mean, m->out_sd, n,
                                                                          m->n_out, 1);
    }
    MCU(cudaGetLastError());
    return PIC_OK;
}

} // namespace

extern "C" {

pic_status pic_mlp_create(int n_in, int n_hidden, int n_out, uint64_t seed, pic_mlp **out)
{
    if (!out || n_in < 1 || n_hidden < 1 || n_out < 1 || n_in > 4096 || n_hidden > 4096 || n_out > 4096)
        return mlp_fail(PIC_EINVAL, "bad MLP sizes");
    pic_mlp *m = new pic_mlp();
    m->n_in = n_in; m->h = n_hidden; m->n_out = n_out;
    const size_t sizes[6] = {(size_t)n_in * n_hidden, (size_t)n_hidden, (size_t)n_hidden * n_hidden, (size_t)n_hidden,
                             (size_t)n_hidden * n_out, (size_t)n_out};
    size_t o = 0;
    for (int i = 0; i < 6; ++i) { m->off[i] = o; o += sizes[i]; }
    m->n_par = o;
    auto cleanup = [&](pic_status s, const char *msg) { pic_mlp_destroy(m); return mlp_fail(s, msg); };
    if (cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking) != cudaSuccess) return cleanup(PIC_ECUDA, "stream");
    float **bufs[] = {&m->p, &m->g, &m->m, &m->v};
    for (float **b : bufs)
        if (cudaMalloc(b, sizeof(float) * m->n_par) != cudaSuccess) return cleanup(PIC_ENOMEM, "MLP parameters");
    if (cudaMalloc(&m->in_lo, sizeof(float) * n_in) != cudaSuccess || cudaMalloc(&m->in_hi, sizeof(float) * n_in) != cudaSuccess ||
        cudaMalloc(&m->out_mean, sizeof(float) * n_out) != cudaSuccess || cudaMalloc(&m->out_sd, sizeof(float) * n_out) != cudaSuccess)
        return cleanup(PIC_ENOMEM, "MLP normalisation");
    cudaMemsetAsync(m->p, 0, sizeof(float) * m->n_par, m->stream);
    cudaMemsetAsync(m->g, 0, sizeof(float) * m->n_par, m->stream);
    cudaMemsetAsync(m->m, 0, sizeof(float) * m->n_par, m->stream);
    cudaMemsetAsync(m->v, 0, sizeof(float) * m->n_par, m->stream);
    const int fan[3][2] = {{n_in, n_hidden}, {n_hidden, n_hidden}, {n_hidden, n_out}};
    for (int l = 0; l < 3; ++l) {
        const int n = fan[l][0] * fan[l][1];
        k_init<<<blocks(n), 256, 0, m->stream>>>(m->p + m->off[2 * l], n, std::sqrt(6.0f / (fan[l][0] + fan[l][1])),
                                                 seed + 0x1000ull * (uint64_t)l);
    }
    std::vector<float> lo(n_in, -1.0f), hi(n_in, 1.0f), mean(n_out, 0.0f), sd(n_out, 1.0f);
    cudaMemcpyAsync(m->in_lo, lo.data(), sizeof(float) * n_in, cudaMemcpyHostToDevice, m->stream);
    cudaMemcpyAsync(m->in_hi, hi.data(), sizeof(float) * n_in, cudaMemcpyHostToDevice, m->stream);
    cudaMemcpyAsync(m->out_mean, mean.data(), sizeof(float) * n_out, cudaMemcpyHostToDevice, m->stream);
    cudaMemcpyAsync(m->out_sd, sd.data(), sizeof(float) * n_out, cudaMemcpyHostToDevice, m->stream);
    if (cudaStreamSynchronize(m->stream) != cudaSuccess || cudaGetLastError() != cudaSuccess)
        return cleanup(PIC_ECUDA, "MLP initialisation");
    *out = m;
    return PIC_OK;
}

pic_status pic_mlp_set_normalization(pic_mlp *m, const float *in_lo, const float *in_hi, const float *out_mean,
                                     const float *out_sd)
{
    if (!m || !in_lo || !in_hi || !out_mean || !out_sd) return mlp_fail(PIC_EINVAL, "null normalisation");
    for (int j = 0; j < m->n_in; ++j)
        if (!(in_hi[j] > in_lo[j])) return mlp_fail(PIC_EINVAL, "input range must have hi > lo");
    for (int j = 0; j < m->n_out; ++j)
        if (!(out_sd[j] > 0)) return mlp_fail(PIC_EINVAL, "output deviation must be positive");
    MCU(cudaMemcpyAsync(m->in_lo, in_lo, sizeof(float) * m->n_in, cudaMemcpyHostToDevice, m->stream));
    MCU(cudaMemcpyAsync(m->in_hi, in_hi, sizeof(float) * m->n_in, cudaMemcpyHostToDevice, m->stream));
    MCU(cudaMemcpyAsync(m->out_mean, out_mean, sizeof(float) * m->n_out, cudaMemcpyHostToDevice, m->stream));
    MCU(cudaMemcpyAsync(m->out_sd, out_sd, sizeof(float) * m->n_out, cudaMemcpyHostToDevice, m->stream));
    MCU(cudaStreamSynchronize(m->stream));
    return PIC_OK;
}

int64_t pic_mlp_param_count(const pic_mlp *m) { return m ? (int64_t)m->n_par : 0; }

pic_status pic_mlp_get_params(pic_mlp *m, float *params)
{
    if (!m || !params) return mlp_fail(PIC_EINVAL, "null argument");
    MCU(cudaMemcpyAsync(params, m->p, sizeof(float) * m->n_par, cudaMemcpyDeviceToHost, m->stream));
    MCU(cudaStreamSynchronize(m->stream));
    return PIC_OK;
}

pic_status pic_mlp_set_params(pic_mlp *m, const float *params)
{
    if (!m || !params) return mlp_fail(PIC_EINVAL, "null argument");
    MCU(cudaMemcpyAsync(m->p, params, sizeof(float) * m->n_par, cudaMemcpyHostToDevice, m->stream));
    MCU(cudaMemsetAsync(m->m, 0, sizeof(float) * m->n_par, m->stream));
    MCU(cudaMemsetAsync(m->v, 0, sizeof(float) * m->n_par, m->stream));
    m->adam_t = 0;
    MCU(cudaStreamSynchronize(m->stream));
    return PIC_OK;
}

pic_status pic_mlp_gradients(pic_mlp *m, const float *X, const float *Y, int n, float *grads, float *loss)
{
    if (!m || !X || !Y || n < 1) return mlp_fail(PIC_EINVAL, "bad gradient arguments");
    pic_status st = upload_batch(m, X, Y, n);
    if (st != PIC_OK) return st;
    forward(m, n);
    backward(m, n);
    MCU(cudaGetLastError());
    if (grads) MCU(cudaMemcpyAsync(grads, m->g, sizeof(float) * m->n_par, cudaMemcpyDeviceToHost, m->stream));
    float l = 0;
    st = read_loss(m, n, &l);
    if (loss) *loss = l;
    return st;
}

pic_status pic_mlp_train(pic_mlp *m, const float *X, const float *Y, int n, int epochs, float lr, float *loss_curve)
{
    if (!m || !X || !Y || n < 1 || epochs < 0 || !(lr > 0)) return mlp_fail(PIC_EINVAL, "bad training arguments");
    pic_status st = upload_batch(m, X, Y, n);
    if (st != PIC_OK) return st;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int e = 0; e < epochs; ++e) {
        forward(m, n);
        backward(m, n);
        m->adam_t++;
        const float c1 = 1.0f / (1.0f - std::pow(b1, (float)m->adam_t));
        const float c2 = 1.0f / (1.0f - std::pow(b2, (float)m->adam_t));
        k_adam<<<blocks((long long)m->n_par), 256, 0, m->stream>>>(m->p, m->g, m->m, m->v, (int)m->n_par, lr, b1, b2,
                                                                    eps, c1, c2);
        if (loss_curve) {
            st = read_loss(m, n, &loss_curve[e]);
            if (st != PIC_OK) return st;
        }
    }
    MCU(cudaGetLastError());
    MCU(cudaStreamSynchronize(m->stream));
    return PIC_OK;
}

pic_status pic_mlp_adam_step(pic_mlp *m, const float *grads, float lr)
{
    if (!m || !grads || !(lr > 0)) return mlp_fail(PIC_EINVAL, "bad Adam arguments");
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    MCU(cudaMemcpyAsync(m->g, grads, sizeof(float) * m->n_par, cudaMemcpyHostToDevice, m->stream));
    m->adam_t++;
    const float c1 = 1.0f / (1.0f - std::pow(b1, (float)m->adam_t));
    const float c2 = 1.0f / (1.0f - std::pow(b2, (float)m->adam_t));
    k_adam<<<blocks((long long)m->n_par), 256, 0, m->stream>>>(m->p, m->g, m->m, m->v, (int)m->n_par, lr, b1, b2, eps,
                                                                c1, c2);
    MCU(cudaGetLastError());
    MCU(cudaStreamSynchronize(m->stream));
    return PIC_OK;
}

pic_status pic_warmstart_train(pic_mlp *m, const double *params, const double *ne, const double *ni, const double *te,
                               int n_cases, int n_params, int n_points, const double *in_lo, const double *in_hi,
                               int epochs, float lr, float *loss_curve)
{
    if (!m || !params || !ne || !ni || !te || !in_lo || !in_hi || n_cases < 1 || n_params != m->n_in ||
        n_points < 2 || 3 * n_points != m->n_out || epochs < 0 || !(lr > 0))
        return mlp_fail(PIC_EINVAL, "bad warm-start training arguments");
    const int no = m->n_out;
    std::vector<float> X((size_t)n_cases * n_params), Y((size_t)n_cases * no);
    for (size_t k = 0; k < X.size(); ++k) X[k] = (float)params[k];
    for (int i = 0; i < n_cases; ++i)
        for (int j = 0; j < n_points; ++j) {
            const size_t a = (size_t)i * n_points + j, r = (size_t)i * no;
            if (!(ne[a] >= 0) || !(ni[a] >= 0) || !std::isfinite(te[a]))
                return mlp_fail(PIC_EINVAL, "negative or non-finite training profile");
            Y[r + j] = (float)std::log10(std::max(ne[a], 1e6));
            Y[r + n_points + j] = (float)std::log10(std::max(ni[a], 1e6));
            Y[r + 2 * n_points + j] = (float)te[a];
        }
    std::vector<float> lo(n_params), hi(n_params), mean(no, 0.0f), sd(no, 0.0f);
    for (int k = 0; k < n_params; ++k) {
        lo[k] = (float)in_lo[k];
        hi[k] = (float)in_hi[k];
        if (!(hi[k] > lo[k])) return mlp_fail(PIC_EINVAL, "input range must have in_hi > in_lo");
    }
    for (int j = 0; j < no; ++j) {                   // per output: mean and deviation over the cases
        double s = 0, s2 = 0;
        for (int i = 0; i < n_cases; ++i) s += Y[(size_t)i * no + j];
        const double mu = s / n_cases;
        for (int i = 0; i < n_cases; ++i) s2 += (Y[(size_t)i * no + j] - mu) * (Y[(size_t)i * no + j] - mu);
        mean[j] = (float)mu;
        sd[j] = (float)(std::sqrt(s2 / n_cases) + 1e-3);
    }
    pic_status st = pic_mlp_set_normalization(m, lo.data(), hi.data(), mean.data(), sd.data());
    if (st != PIC_OK) return st;
    return pic_mlp_train(m, X.data(), Y.data(), n_cases, epochs, lr, loss_curve);
}

pic_status pic_mlp_predict(pic_mlp *m, const float *X, int n, float *Y)
{
    if (!m || !X || !Y || n < 1) return mlp_fail(PIC_EINVAL, "bad predict arguments");
    pic_status st = upload_batch(m, X, nullptr, n);
    if (st != PIC_OK) return st;
    forward(m, n);
    k_norm_out<<<blocks((long long)n * m->n_out), 256, 0, m->stream>>>(m->Y, m->dH, m->out_mean, m->out_sd, n, m->n_out, 0);
    MCU(cudaGetLastError());
    MCU(cudaMemcpyAsync(Y, m->dH, sizeof(float) * (size_t)n * m->n_out, cudaMemcpyDeviceToHost, m->stream));
    MCU(cudaStreamSynchronize(m->stream));
    return PIC_OK;
}

pic_status pic_mlp_destroy(pic_mlp *m)
{
    if (!m) return PIC_OK;
    if (m->stream) cudaStreamSynchronize(m->stream);
    float *bufs[] = {m->p, m->g, m->m, m->v, m->in_lo, m->in_hi, m->out_mean, m->out_sd, m->X, m->Xn, m->Z1, m->H1,
                     m->Z2, m->H2, m->Y, m->T, m->dY, m->dH, m->dZ, m->part};
    for (float *b : bufs)
        if (b) cudaFree(b);
    if (m->stream) cudaStreamDestroy(m->stream);
    delete m;
    return PIC_OK;
}

pic_status pic_gemm_bf16(const float *A, int ar, int ac, const float *B, int br, int bc, float *C, int ldc, int M, int N,
                         int K, void *stream)
{
    if (!A || !B || !C || M < 1 || N < 1 || K < 1) return mlp_fail(PIC_EINVAL, "bad GEMM arguments");
    const int tiles = ((M + 15) / 16) * ((N + 15) / 16);
    k_gemm_bf16<<<(tiles + 7) / 8, 256, 0, (cudaStream_t)stream>>>(A, ar, ac, B, br, bc, C, ldc, M, N, K, 1.0f, 0);
    MCU(cudaGetLastError());
    return PIC_OK;
}

} // extern "C"
