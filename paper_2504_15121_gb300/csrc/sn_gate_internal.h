// Internal declarations of the learned gate (weights layout, GEMM, kernels).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "sn_gate.h"
#include "sn_internal.h"

namespace sn {

// flat parameter vector: W1 [16][9][8], b1 [16], W2 [16][9][16], b2 [16], W3 [16], b3
constexpr int kW1N = 16 * 9 * 8;
constexpr int kW2N = 16 * 9 * 16;
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kW1N;
constexpr int kOffW2 = kOffB1 + 16;
constexpr int kOffB2 = kOffW2 + kW2N;
constexpr int kOffW3 = kOffB2 + 16;
constexpr int kOffB3 = kOffW3 + 16;
constexpr int kGateParams = kOffB3 + 1;

// Kernel-side weights: GEMM copies in BF16 (rows = output channel, k =
// tap * channels + channel; W1g padded to k = 80), the rest FP32.
struct GateDev {
    __nv_bfloat16* W1g;  // [16][80]
    __nv_bfloat16* W2g;  // [16][144]
    float* b1;           // [16]
    float* b2;           // [16]
    float* W3;           // [16]
    float* b3;           // [1]
};

cudaError_t gate_alloc(GateDev& w);
void gate_free(GateDev& w);
cudaError_t gate_layout(const float* theta, const GateDev& w, cudaStream_t s);
// C [M][N] (FP32, rows ldc apart) = A B with A(m, k) = A[m sam + k sak],
// B(k, n) = B[k sbk + n sbn] on the tcgen05 tensor cores; err: device word
// that a kernel whose bounded MMA wait gave up sets (its C is undefined).
cudaError_t gemm_bf16(int M, int N, int K, const __nv_bfloat16* A, long long sam, long long sak,
                      const __nv_bfloat16* B, long long sbk, long long sbn, float* C, long long ldc, int* err,
                      cudaStream_t s);
void k_adam_launch(int n, float* theta, float* m, float* v, const float* g, float lr, float b1c, float b2c,
                   cudaStream_t s);

}  // namespace sn
