// Learned boundary gate: weight layout, training kernels (forward, backward,
// Adam) and the trainer entry points of include/sn_gate.h.
//
// Network (per pixel p, see include/sn_gate.h): features f(p) (8 channels:
// FP32 steps of the FP32 log2 of the codes to the right and down, validity,
// 5 zeros), a 3x3
// convolution 8 -> 16 with ReLU, a 3x3 convolution 16 -> 16 with ReLU, a
// 1x1 layer 16 -> 1 and a sigmoid.  Training works on 6x6 patches of
// integer disparity codes (centre at [2][2]).  Every contraction is a BF16
// tensor-core GEMM with FP32 accumulation (mma.sync m16n8k16); the master
// weights and the optimiser state are FP32.
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <new>

#include "sn_device.cuh"
#include "sn_gate_internal.h"

namespace sn {

// ------------------------------------------------------------------ GEMM
// C[M][N] (fp32, ldc) = sum_k A(m, k) B(k, n); A(m, k) = A[m sam + k sak],
// B(k, n) = B[k sbk + n sbn] (bf16 element strides).  Block tile 64 x 16,
// 4 warps, each warp 16 rows x 16 columns (two m16n8k16 products per k-step).
namespace {

constexpr int kGM = 64, kGN = 16, kGK = 16, kLd = 24;  // smem row stride (bf16), conflict-free ldmatrix

__global__ void __launch_bounds__(128) k_gemm(int M, int N, int K, const __nv_bfloat16* __restrict__ A, long long sam,
                                              long long sak, const __nv_bfloat16* __restrict__ B, long long sbk,
                                              long long sbn, float* __restrict__ C, long long ldc) {
    __shared__ __align__(16) __nv_bfloat16 As[kGM][kLd];
    __shared__ __align__(16) __nv_bfloat16 Bs[kGN][kLd];  // [n][k]
    const int m0 = blockIdx.x * kGM, n0 = blockIdx.y * kGN;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    float acc0[4] = {0, 0, 0, 0}, acc1[4] = {0, 0, 0, 0};
    const __nv_bfloat16 zero = __float2bfloat16(0.0f);
    for (int k0 = 0; k0 < K; k0 += kGK) {
        for (int i = tid; i < kGM * kGK; i += 128) {
            const int r = i / kGK, k = i % kGK;
            const int m = m0 + r, kk = k0 + k;
            As[r][k] = (m < M && kk < K) ? A[(long long)m * sam + (long long)kk * sak] : zero;
        }
        for (int i = tid; i < kGN * kGK; i += 128) {
            const int c = i / kGK, k = i % kGK;
            const int n = n0 + c, kk = k0 + k;
            Bs[c][k] = (n < N && kk < K) ? B[(long long)kk * sbk + (long long)n * sbn] : zero;
        }
        __syncthreads();
        unsigned a[4], b[4];
        ldsm_x4(a, &As[warp * 16 + (lane & 15)][(lane >> 4) * 8]);
        ldsm_x4(b, &Bs[(lane & 7) + ((lane >> 4) << 3)][((lane >> 3) & 1) * 8]);
        mma_bf16(acc0, a, b[0], b[1]);
        mma_bf16(acc1, a, b[2], b[3]);
        __syncthreads();
    }
    const int g = lane >> 2, t = lane & 3;
    const int r0 = m0 + warp * 16 + g;
    for (int h = 0; h < 2; h++) {
        const int r = r0 + 8 * h;
        if (r >= M) continue;
        const int c0 = n0 + 2 * t, c1 = n0 + 8 + 2 * t;
        if (c0 < N) C[(long long)r * ldc + c0] = acc0[2 * h];
        if (c0 + 1 < N) C[(long long)r * ldc + c0 + 1] = acc0[2 * h + 1];
        if (c1 < N) C[(long long)r * ldc + c1] = acc1[2 * h];
        if (c1 + 1 < N) C[(long long)r * ldc + c1 + 1] = acc1[2 * h + 1];
    }
}

}  // namespace

cudaError_t gemm_bf16(int M, int N, int K, const __nv_bfloat16* A, long long sam, long long sak,
                      const __nv_bfloat16* B, long long sbk, long long sbn, float* C, long long ldc,
                      cudaStream_t s) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    const dim3 grid((M + kGM - 1) / kGM, (N + kGN - 1) / kGN);
    k_gemm<<<grid, 128, 0, s>>>(M, N, K, A, sam, sak, B, sbk, sbn, C, ldc);
    return cudaGetLastError();
}

namespace {

// Dp [B][36] -> F [B][25][8] (bf16): features at the 5x5 patch positions.
__global__ void k_features(int B, const int* __restrict__ Dp, const float* __restrict__ tab,
                           __nv_bfloat16* __restrict__ F) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)B * 25) return;
    const int b = (int)(i / 25), pos = (int)(i % 25), r = pos / 5, c = pos % 5;
    const int* d = Dp + (long long)b * 36;
    float f[3];
    gate_feature(tab, d[r * 6 + c], d[r * 6 + c + 1], d[(r + 1) * 6 + c], f);
    __nv_bfloat16* o = F + i * 8;
    o[0] = __float2bfloat16(f[0]);
    o[1] = __float2bfloat16(f[1]);
    o[2] = __float2bfloat16(f[2]);
    for (int k = 3; k < 8; k++) o[k] = __float2bfloat16(0.0f);
}

// F -> A1 [B*9][80]: row (b, q) for the layer-1 output at patch position
// (1 + q/3, 1 + q%3); k = tap * 8 + channel, taps 0..8, then 8 zeros.
__global__ void k_im2col1(int B, const __nv_bfloat16* __restrict__ F, __nv_bfloat16* __restrict__ A1) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)B * 9 * 80) return;
    const long long row = i / 80;
    const int k = (int)(i % 80);
    const int b = (int)(row / 9), q = (int)(row % 9);
    __nv_bfloat16 v = __float2bfloat16(0.0f);
    if (k < 72) {
        const int tap = k / 8, ch = k % 8;
        const int r = 1 + q / 3 + tap / 3 - 1, c = 1 + q % 3 + tap % 3 - 1;
        v = F[((long long)b * 25 + r * 5 + c) * 8 + ch];
    }
    A1[i] = v;
}

// h1 = relu(C1 + b1) -> A2 (bf16, [B][144] == [B*9][16]); C1 keeps the pre-activation.
__global__ void k_act1(long long n, const float* __restrict__ C1, const float* __restrict__ b1,
                       __nv_bfloat16* __restrict__ A2) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    A2[i] = __float2bfloat16(fmaxf(C1[i] + b1[i % 16], 0.0f));
}

// Head: a2 = C2 + b2, z = relu(a2), logit = z . W3 + b3, q = sigmoid;
// loss (mean BCE), d logit = (q - y) / B, dZ = d logit W3 [a2 > 0] (bf16),
// and the gradients of W3, b3, b2 (accumulated with atomics).
__global__ void k_head(int B, const float* __restrict__ C2, const float* __restrict__ b2,
                       const float* __restrict__ W3, const float* __restrict__ b3, const float* __restrict__ y,
                       float* __restrict__ q_out, __nv_bfloat16* __restrict__ dZ, float* __restrict__ gW3,
                       float* __restrict__ gb2, float* __restrict__ gb3, float* __restrict__ loss) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    float a2[16], logit = b3[0];
    for (int c = 0; c < 16; c++) {
        a2[c] = C2[(long long)b * 16 + c] + b2[c];
        logit += fmaxf(a2[c], 0.0f) * W3[c];
    }
    const float q = 1.0f / (1.0f + expf(-logit));
    if (q_out) q_out[b] = q;
    if (!y) return;
    const float yb = y[b];
    const float qc = fminf(fmaxf(q, 1e-7f), 1.0f - 1e-7f);
    atomicAdd(loss, -(yb * logf(qc) + (1.0f - yb) * logf(1.0f - qc)) / B);
    const float dl = (q - yb) / B;
    atomicAdd(gb3, dl);
    for (int c = 0; c < 16; c++) {
        const float z = fmaxf(a2[c], 0.0f);
        atomicAdd(&gW3[c], z * dl);
        const float dz = a2[c] > 0.0f ? dl * W3[c] : 0.0f;
        atomicAdd(&gb2[c], dz);
        dZ[(long long)b * 16 + c] = __float2bfloat16(dz);
    }
}

// dH1 = dA2 [C1 + b1 > 0] (bf16) and the gradient of b1.
__global__ void k_act1_bwd(long long n, const float* __restrict__ dA2, const float* __restrict__ C1,
                           const float* __restrict__ b1, __nv_bfloat16* __restrict__ dH1, float* __restrict__ gb1) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = (int)(i % 16);
    const float d = C1[i] + b1[c] > 0.0f ? dA2[i] : 0.0f;
    dH1[i] = __float2bfloat16(d);
    if (d != 0.0f) atomicAdd(&gb1[c], d);
}

// Gradient vector in the flat parameter order from the GEMM outputs:
// dW1g [16][80] -> W1 [16][9][8]; dW2g [16][144] -> W2 [16][9][16].
__global__ void k_pack_grad(const float* __restrict__ dW1g, const float* __restrict__ dW2g, float* __restrict__ g) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kW1N) {
        const int o = i / 72, k = i % 72;
        g[kOffW1 + i] = dW1g[o * 80 + k];
    } else if (i < kW1N + kW2N) {
        const int j = i - kW1N;
        g[kOffW2 + j] = dW2g[j];
    }
}

// Adam on the FP32 master weights, then the BF16 GEMM copies.
__global__ void k_adam(int n, float* __restrict__ theta, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, float lr, float b1c, float b2c) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = 0.9f * m[i] + 0.1f * gi;
    const float vi = 0.999f * v[i] + 0.001f * gi * gi;
    m[i] = mi;
    v[i] = vi;
    theta[i] -= lr * (mi / b1c) / (sqrtf(vi / b2c) + 1e-8f);
}

}  // namespace

// Writes the kernel-side weights: W1g [16][80] (bf16, k = tap * 8 + ch, pad
// zero), W2g [16][144] (bf16, k = tap * 16 + ch), b1, b2, W3, b3 (fp32).
__global__ void k_gate_layout(const float* __restrict__ theta, GateDev w) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 16 * 80) {
        const int o = i / 80, k = i % 80;
        w.W1g[i] = __float2bfloat16(k < 72 ? theta[kOffW1 + o * 72 + k] : 0.0f);
    }
    if (i < 16 * 144) w.W2g[i] = __float2bfloat16(theta[kOffW2 + i]);
    if (i < 16) {
        w.b1[i] = theta[kOffB1 + i];
        w.b2[i] = theta[kOffB2 + i];
        w.W3[i] = theta[kOffW3 + i];
    }
    if (i == 0) w.b3[0] = theta[kOffB3];
}

// BF16 rounding (to nearest, ties to even) of a finite float, as a float
static float bf16_round(float x) {
    uint32_t u;
    memcpy(&u, &x, 4);
    u = (u + 0x7FFFu + ((u >> 16) & 1u)) & 0xFFFF0000u;
    float r;
    memcpy(&r, &u, 4);
    return r;
}

void gate_constants(const float* theta, GateView* gv) {
    float c3 = theta[kOffB3];
    for (int c = 0; c < 16; c++) {
        gv->k.b1[c] = theta[kOffB1 + c];
        gv->k.nb2[c] = -theta[kOffB2 + c];
        gv->k.w3[c] = bf16_round(theta[kOffW3 + c]);
        c3 = fmaf(gv->k.w3[c], theta[kOffB2 + c], c3);
    }
    gv->k.c3 = c3;
}

cudaError_t gate_layout(const float* theta, const GateDev& w, cudaStream_t s) {
    k_gate_layout<<<(16 * 144 + 255) / 256, 256, 0, s>>>(theta, w);
    return cudaGetLastError();
}

}  // namespace sn

// ------------------------------------------------------------------ trainer
struct sn_gate_trainer {
    int max_batch = 0;
    long long step = 0;
    float *theta = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr, *loss = nullptr;
    sn::GateDev w{};
    __nv_bfloat16 *F = nullptr, *A1 = nullptr, *A2 = nullptr, *dZ = nullptr, *dH1 = nullptr;
    float *C1 = nullptr, *C2 = nullptr, *dA2 = nullptr, *dW1g = nullptr, *dW2g = nullptr;
    const float* log2tab = nullptr;  // FP32 log2 of every code (the library's table)
};

namespace {

unsigned blocks(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// forward (+ backward when y != nullptr) of one batch; gradient into t->grad
cudaError_t gate_pass(sn_gate_trainer* t, const int* Dp, const float* y, int B, float* q_out, cudaStream_t s) {
    using namespace sn;
    cudaError_t e;
    k_features<<<blocks((long long)B * 25), 256, 0, s>>>(B, Dp, t->log2tab, t->F);
    k_im2col1<<<blocks((long long)B * 9 * 80), 256, 0, s>>>(B, t->F, t->A1);
    // C1 [B*9][16] = A1 [B*9][80] x W1g^T
    if ((e = gemm_bf16(B * 9, 16, 80, t->A1, 80, 1, t->w.W1g, 1, 80, t->C1, 16, s)) != cudaSuccess) return e;
    k_act1<<<blocks((long long)B * 144), 256, 0, s>>>((long long)B * 144, t->C1, t->w.b1, t->A2);
    // C2 [B][16] = A2 [B][144] x W2g^T
    if ((e = gemm_bf16(B, 16, 144, t->A2, 144, 1, t->w.W2g, 1, 144, t->C2, 16, s)) != cudaSuccess) return e;
    if (y) {
        cudaMemsetAsync(t->grad, 0, sizeof(float) * kGateParams, s);
        cudaMemsetAsync(t->loss, 0, sizeof(float), s);
    }
    k_head<<<blocks(B, 128), 128, 0, s>>>(B, t->C2, t->w.b2, t->w.W3, t->w.b3, y, q_out, t->dZ,
                                         t->grad + kOffW3, t->grad + kOffB2, t->grad + kOffB3, t->loss);
    if (!y) return cudaGetLastError();
    // dW2g [16][144] = dZ^T [16][B] x A2 [B][144]
    if ((e = gemm_bf16(16, 144, B, t->dZ, 1, 16, t->A2, 144, 1, t->dW2g, 144, s)) != cudaSuccess) return e;
    // dA2 [B][144] = dZ [B][16] x W2g [16][144]
    if ((e = gemm_bf16(B, 144, 16, t->dZ, 16, 1, t->w.W2g, 144, 1, t->dA2, 144, s)) != cudaSuccess) return e;
    k_act1_bwd<<<blocks((long long)B * 144), 256, 0, s>>>((long long)B * 144, t->dA2, t->C1, t->w.b1, t->dH1,
                                                          t->grad + kOffB1);
    // dW1g [16][80] = dH1^T [16][B*9] x A1 [B*9][80]
    if ((e = gemm_bf16(16, 80, B * 9, t->dH1, 1, 16, t->A1, 80, 1, t->dW1g, 80, s)) != cudaSuccess) return e;
    k_pack_grad<<<blocks(kW1N + kW2N), 256, 0, s>>>(t->dW1g, t->dW2g, t->grad);
    return cudaGetLastError();
}

template <class T>
cudaError_t alloc(T** p, size_t n) {
    return cudaMalloc((void**)p, sizeof(T) * (n ? n : 1));
}

}  // namespace

extern "C" {

int sn_gate_param_count(void) { return sn::kGateParams; }

sn_status sn_gate_trainer_create(int max_batch, const float* theta0, sn_gate_trainer** out) {
    if (!out || max_batch < 1 || max_batch > (1 << 20) || !theta0) return SN_EINVAL;
    *out = nullptr;
    auto* t = new (std::nothrow) sn_gate_trainer();
    if (!t) return SN_ENOMEM;
    t->max_batch = max_batch;
    const size_t B = max_batch;
    cudaError_t e = cudaSuccess;
    const int P = sn::kGateParams;
    if (e == cudaSuccess) e = sn::log2_table(&t->log2tab);
    if (e == cudaSuccess) e = alloc(&t->theta, P);
    if (e == cudaSuccess) e = alloc(&t->m, P);
    if (e == cudaSuccess) e = alloc(&t->v, P);
    if (e == cudaSuccess) e = alloc(&t->grad, P);
    if (e == cudaSuccess) e = alloc(&t->loss, 1);
    if (e == cudaSuccess) e = sn::gate_alloc(t->w);
    if (e == cudaSuccess) e = alloc(&t->F, B * 25 * 8);
    if (e == cudaSuccess) e = alloc(&t->A1, B * 9 * 80);
    if (e == cudaSuccess) e = alloc(&t->A2, B * 144);
    if (e == cudaSuccess) e = alloc(&t->dZ, B * 16);
    if (e == cudaSuccess) e = alloc(&t->dH1, B * 144);
    if (e == cudaSuccess) e = alloc(&t->C1, B * 144);
    if (e == cudaSuccess) e = alloc(&t->C2, B * 16);
    if (e == cudaSuccess) e = alloc(&t->dA2, B * 144);
    if (e == cudaSuccess) e = alloc(&t->dW1g, 16 * 80);
    if (e == cudaSuccess) e = alloc(&t->dW2g, 16 * 144);
    if (e == cudaSuccess) e = cudaMemcpy(t->theta, theta0, sizeof(float) * P, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(t->m, 0, sizeof(float) * P);
    if (e == cudaSuccess) e = cudaMemset(t->v, 0, sizeof(float) * P);
    if (e == cudaSuccess) e = sn::gate_layout(t->theta, t->w, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cudaGetLastError();
        sn_gate_trainer_destroy(t);
        return SN_ENOMEM;
    }
    *out = t;
    return SN_OK;
}

sn_status sn_gate_trainer_destroy(sn_gate_trainer* t) {
    if (!t) return SN_OK;
    cudaFree(t->theta);
    cudaFree(t->m);
    cudaFree(t->v);
    cudaFree(t->grad);
    cudaFree(t->loss);
    sn::gate_free(t->w);
    cudaFree(t->F);
    cudaFree(t->A1);
    cudaFree(t->A2);
    cudaFree(t->dZ);
    cudaFree(t->dH1);
    cudaFree(t->C1);
    cudaFree(t->C2);
    cudaFree(t->dA2);
    cudaFree(t->dW1g);
    cudaFree(t->dW2g);
    delete t;
    return SN_OK;
}

sn_status sn_gate_trainer_grad(sn_gate_trainer* t, const int32_t* patches, const float* y, int B, float* grad,
                               float* q, float* loss, sn_stream s) {
    if (!t || !patches || B < 1 || B > t->max_batch) return SN_EINVAL;
    cudaError_t e = gate_pass(t, patches, y, B, q, s);
    if (e == cudaSuccess && y && grad)
        e = cudaMemcpyAsync(grad, t->grad, sizeof(float) * sn::kGateParams, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && y && loss) e = cudaMemcpyAsync(loss, t->loss, sizeof(float), cudaMemcpyDeviceToDevice, s);
    return e == cudaSuccess ? SN_OK : SN_ECUDA;
}

sn_status sn_gate_trainer_step(sn_gate_trainer* t, const int32_t* patches, const float* y, int B, float lr,
                               float* loss, sn_stream s) {
    if (!t || !patches || !y || B < 1 || B > t->max_batch || !(lr > 0)) return SN_EINVAL;
    cudaError_t e = gate_pass(t, patches, y, B, nullptr, s);
    if (e != cudaSuccess) return SN_ECUDA;
    t->step++;
    const float b1c = 1.0f - powf(0.9f, (float)t->step), b2c = 1.0f - powf(0.999f, (float)t->step);
    sn::k_adam_launch(sn::kGateParams, t->theta, t->m, t->v, t->grad, lr, b1c, b2c, s);
    e = sn::gate_layout(t->theta, t->w, s);
    if (e == cudaSuccess && loss) e = cudaMemcpyAsync(loss, t->loss, sizeof(float), cudaMemcpyDeviceToDevice, s);
    return e == cudaSuccess ? SN_OK : SN_ECUDA;
}

sn_status sn_gate_trainer_state(sn_gate_trainer* t, float* theta, float* m, float* v, long long* step) {
    if (!t) return SN_EINVAL;
    cudaError_t e = cudaDeviceSynchronize();
    const size_t b = sizeof(float) * sn::kGateParams;
    if (e == cudaSuccess && theta) e = cudaMemcpy(theta, t->theta, b, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && m) e = cudaMemcpy(m, t->m, b, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && v) e = cudaMemcpy(v, t->v, b, cudaMemcpyDeviceToHost);
    if (step) *step = t->step;
    return e == cudaSuccess ? SN_OK : SN_ECUDA;
}

sn_status sn_gate_trainer_resume(sn_gate_trainer* t, const float* theta, const float* m, const float* v,
                                 long long step) {
    if (!t || !theta || !m || !v || step < 0) return SN_EINVAL;
    const size_t b = sizeof(float) * sn::kGateParams;
    cudaError_t e = cudaMemcpy(t->theta, theta, b, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(t->m, m, b, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(t->v, v, b, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = sn::gate_layout(t->theta, t->w, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    t->step = step;
    return e == cudaSuccess ? SN_OK : SN_ECUDA;
}

}  // extern "C"

namespace sn {
void k_adam_launch(int n, float* theta, float* m, float* v, const float* g, float lr, float b1c, float b2c,
                   cudaStream_t s) {
    k_adam<<<(n + 255) / 256, 256, 0, s>>>(n, theta, m, v, g, lr, b1c, b2c);
}

cudaError_t gate_alloc(GateDev& w) {
    cudaError_t e = cudaMalloc((void**)&w.W1g, sizeof(__nv_bfloat16) * 16 * 80);
    if (e == cudaSuccess) e = cudaMalloc((void**)&w.W2g, sizeof(__nv_bfloat16) * 16 * 144);
    if (e == cudaSuccess) e = cudaMalloc((void**)&w.b1, sizeof(float) * 64);
    if (e == cudaSuccess) {
        w.b2 = w.b1 + 16;
        w.W3 = w.b1 + 32;
        w.b3 = w.b1 + 48;
    }
    return e;
}

void gate_free(GateDev& w) {
    cudaFree(w.W1g);
    cudaFree(w.W2g);
    cudaFree(w.b1);
    w = GateDev{};
}
}  // namespace sn
