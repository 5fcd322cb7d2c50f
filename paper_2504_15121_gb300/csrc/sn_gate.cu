// Learned boundary gate: weight layout, training kernels (forward, backward,
// Adam) and the trainer entry points of include/sn_gate.h.
//
// Network (per pixel p, see include/sn_gate.h): features f(p) (8 channels:
// FP32 steps of the FP32 log2 of the codes to the right and down, validity,
// 5 zeros), a 3x3
// convolution 8 -> 16 with ReLU, a 3x3 convolution 16 -> 16 with ReLU, a
// 1x1 layer 16 -> 1 and a sigmoid.  Training works on 6x6 patches of
// integer disparity codes (centre at [2][2]).  Every contraction is a BF16
// tcgen05 GEMM with FP32 accumulation in tensor memory; the master weights
// and the optimiser state are FP32.
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <new>

#include "sn_device.cuh"
#include "sn_gate_internal.h"
#include "sn_umma.cuh"

namespace sn {

// ------------------------------------------------------------------ GEMM
// C (FP32; element (m, n) at C[m scm + n scn]) = sum_k A(m, k) B(k, n), with
// A(m, k) = A[m sam + k sak] and B(k, n) = B[k sbk + n sbn] (BF16, element
// strides).  One CTA of 128 threads per 128 x 16 tile of C.  Per K-step of
// 16 the threads gather the A tile (128 x 16) and the B tile (16 x 16) into
// shared memory in the tensor core's K-major layout (core matrices of 8 rows
// x 16 bytes; the two K halves kTM or kTN rows apart), one thread issues a
// tcgen05.mma (M = 128, N = 16, K = 16, accumulator in 32 TMEM columns) and
// commits it to an mbarrier, and one thread waits for it (bounded) before
// the next step overwrites the tiles.  The accumulator comes back by
// tcgen05.ld: warp w holds rows 32 w .. 32 w + 31.
namespace {

constexpr int kTM = 128, kTN = 16;
constexpr uint32_t kGemmIdesc = umma::idesc_bf16<kTM, kTN>();

__device__ __forceinline__ uint4 pack8(const unsigned short (&v)[16], int h) {
    return make_uint4(v[8 * h] | ((unsigned)v[8 * h + 1] << 16), v[8 * h + 2] | ((unsigned)v[8 * h + 3] << 16),
                      v[8 * h + 4] | ((unsigned)v[8 * h + 5] << 16), v[8 * h + 6] | ((unsigned)v[8 * h + 7] << 16));
}

__global__ void __launch_bounds__(128) k_gemm(int M, int N, int K, const __nv_bfloat16* __restrict__ A, long long sam,
                                              long long sak, const __nv_bfloat16* __restrict__ B, long long sbk,
                                              long long sbn, float* __restrict__ C, long long scm, long long scn,
                                              int* err) {
    __shared__ __align__(128) uint4 As[2 * kTM];  // [k half][row]: 8 BF16 each
    __shared__ __align__(128) uint4 Bs[2 * kTN];  // [k half][n]
    __shared__ uint64_t bar;
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * kTM, n0 = blockIdx.y * kTN;
    const unsigned short* Au = reinterpret_cast<const unsigned short*>(A);
    const unsigned short* Bu = reinterpret_cast<const unsigned short*>(B);
    if (warp == 0) umma::tmem_alloc(&tslot, 32);
    if (tid == 0) umma::mbar_init(&bar, 1);
    umma::fence_before();
    __syncthreads();
    umma::fence_after();
    const uint32_t tmem = tslot;
    bool ok = true;
    int steps = 0;
    for (int k0 = 0; k0 < K; k0 += 16, steps++) {
        unsigned short v[16];
        const int m = m0 + tid;
#pragma unroll
        for (int k = 0; k < 16; k++) {
            const int kk = k0 + k;
            v[k] = (m < M && kk < K) ? Au[(long long)m * sam + (long long)kk * sak] : (unsigned short)0;
        }
        As[tid] = pack8(v, 0);
        As[kTM + tid] = pack8(v, 1);
        if (tid < kTN) {
            const int n = n0 + tid;
#pragma unroll
            for (int k = 0; k < 16; k++) {
                const int kk = k0 + k;
                v[k] = (n < N && kk < K) ? Bu[(long long)kk * sbk + (long long)n * sbn] : (unsigned short)0;
            }
            Bs[tid] = pack8(v, 0);
            Bs[kTN + tid] = pack8(v, 1);
        }
        umma::fence_proxy_async();  // the tiles, written by the generic proxy, are read by the tensor core
        umma::fence_before();
        __syncthreads();
        umma::fence_after();
        if (tid == 0) {
            const uint64_t ad = umma::desc(umma::smem_addr(As), kTM * 16, 128);
            const uint64_t bd = umma::desc(umma::smem_addr(Bs), kTN * 16, 128);
            umma::mma<kGemmIdesc>(tmem, ad, bd, k0 > 0);
            umma::commit(&bar);
            ok = umma::mbar_wait_ns(&bar, steps & 1, umma::kWaitNs);
            if (!ok) {
                // gave up: report, and drain the MMA before the tiles or the
                // TMEM are given back
                atomicOr(err, 1);
                umma::mbar_wait_ns(&bar, steps & 1, umma::kDrainNs);
            }
        }
        ok = __syncthreads_and(ok);
        umma::fence_after();
        if (!ok) break;
    }
    if (ok) {
        float c[16];
        if (K > 0) {
            uint32_t r[16];
            umma::ld16(tmem + ((uint32_t)(warp * 32) << 16), r);
            umma::wait_ld();
#pragma unroll
            for (int j = 0; j < 16; j++) c[j] = __uint_as_float(r[j]);
        } else {
#pragma unroll
            for (int j = 0; j < 16; j++) c[j] = 0.0f;
        }
        const int m = m0 + warp * 32 + lane;
        if (m < M) {
#pragma unroll
            for (int j = 0; j < 16; j++)
                if (n0 + j < N) C[(long long)m * scm + (long long)(n0 + j) * scn] = c[j];
        }
    }
    umma::fence_before();
    __syncthreads();
    if (warp == 0) {
        umma::fence_after();
        umma::tmem_dealloc(tmem, 32);
    }
}

}  // namespace

cudaError_t gemm_bf16(int M, int N, int K, const __nv_bfloat16* A, long long sam, long long sak,
                      const __nv_bfloat16* B, long long sbk, long long sbn, float* C, long long ldc, int* err,
                      cudaStream_t s) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    // the tensor core's M is 128: a narrow product (M < 64) is computed as
    // its transpose, C^T = B^T A^T
    if (M < 64 && N > M) {
        const dim3 grid((N + kTM - 1) / kTM, (M + kTN - 1) / kTN);
        k_gemm<<<grid, 128, 0, s>>>(N, M, K, B, sbn, sbk, A, sak, sam, C, 1, ldc, err);
    } else {
        const dim3 grid((M + kTM - 1) / kTM, (N + kTN - 1) / kTN);
        k_gemm<<<grid, 128, 0, s>>>(M, N, K, A, sam, sak, B, sbk, sbn, C, ldc, 1, err);
    }
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
    int* err = nullptr;              // device error word: a GEMM's bounded MMA wait gave up
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
    if ((e = gemm_bf16(B * 9, 16, 80, t->A1, 80, 1, t->w.W1g, 1, 80, t->C1, 16, t->err, s)) != cudaSuccess) return e;
    k_act1<<<blocks((long long)B * 144), 256, 0, s>>>((long long)B * 144, t->C1, t->w.b1, t->A2);
    // C2 [B][16] = A2 [B][144] x W2g^T
    if ((e = gemm_bf16(B, 16, 144, t->A2, 144, 1, t->w.W2g, 1, 144, t->C2, 16, t->err, s)) != cudaSuccess) return e;
    if (y) {
        cudaMemsetAsync(t->grad, 0, sizeof(float) * kGateParams, s);
        cudaMemsetAsync(t->loss, 0, sizeof(float), s);
    }
    k_head<<<blocks(B, 128), 128, 0, s>>>(B, t->C2, t->w.b2, t->w.W3, t->w.b3, y, q_out, t->dZ,
                                         t->grad + kOffW3, t->grad + kOffB2, t->grad + kOffB3, t->loss);
    if (!y) return cudaGetLastError();
    // dW2g [16][144] = dZ^T [16][B] x A2 [B][144]
    if ((e = gemm_bf16(16, 144, B, t->dZ, 1, 16, t->A2, 144, 1, t->dW2g, 144, t->err, s)) != cudaSuccess) return e;
    // dA2 [B][144] = dZ [B][16] x W2g [16][144]
    if ((e = gemm_bf16(B, 144, 16, t->dZ, 16, 1, t->w.W2g, 144, 1, t->dA2, 144, t->err, s)) != cudaSuccess) return e;
    k_act1_bwd<<<blocks((long long)B * 144), 256, 0, s>>>((long long)B * 144, t->dA2, t->C1, t->w.b1, t->dH1,
                                                          t->grad + kOffB1);
    // dW1g [16][80] = dH1^T [16][B*9] x A1 [B*9][80]
    if ((e = gemm_bf16(16, 80, B * 9, t->dH1, 1, 16, t->A1, 80, 1, t->dW1g, 80, t->err, s)) != cudaSuccess) return e;
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
    if (e == cudaSuccess) e = alloc(&t->err, 1);
    if (e == cudaSuccess) e = cudaMemset(t->err, 0, sizeof(int));
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
    cudaFree(t->err);
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

sn_status sn_gate_trainer_check_device(sn_gate_trainer* t, sn_stream stream) {
    if (!t) return SN_EINVAL;
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, t->err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && h) e = cudaMemsetAsync(t->err, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return SN_ECUDA;
    return h ? SN_ETIMEOUT : SN_OK;
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
