// Internal declarations shared by the C-ABI layer and the kernels.
#pragma once

#include <cuda.h>  // CUtensorMap
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "sn.h"  // include/ is on the include path

namespace sn {

constexpr int kDMax = 131071;       // largest integer disparity code (d < 512 px)
constexpr int kMaxDirs = 16;
constexpr int kMaxSteps = 30;
constexpr int kMaxStar = kMaxDirs * kMaxSteps;
constexpr int kMaxShared = 64;      // offsets reached by more than one ray
constexpr int kCclTile = 32;        // CCL tiles are 32 x 32 pixels

// error bits written to the context's device error word
constexpr int kErrFindLimit = 1;    // a union-find walk exceeded its bound
constexpr int kWalkLimitDefault = 1 << 22;  // > any parent chain of a 16384^2 frame
constexpr int kErrUnionLimit = 2;   // a union retry loop exceeded its bound
constexpr int kErrBarrier = 4;      // a grid barrier wait exceeded its bound
constexpr int kErrMmaWait = 8;      // a tensor-core or TMA completion wait exceeded its bound

// Per-context constants read by every kernel (passed by value).
struct Geo {
    int W, H;
    int in_dtype;
    int r_d, r_a, support, dirs, steps;
    int K_cd, K_pair, K_range;
    // relative guard band of the FP32 covered-depth test (1 + e, 1 - e)
    float cd_hi, cd_lo;
    int normal_fmt;
    float fx, fy, cx, cy, B;
    float fy_over_fx, inv_fx, B_fx_over_fy, fxB;
    double dfx, dfy, dcx, dcy, dB;
    // ST stop: depth z = st_F / D (metres); edge iff |Laplacian of z| > st_t
    double st_F, st_t;
    float st_Ff, st_tf;
    int walk_limit;  // parent steps of one union-find walk in the component passes
    // ceil(2^64 / W) for W >= 2: for any 0 <= i < 2^32 the quotient i / W is
    // the high word of the 128-bit product i w_rcp (the rounding error
    // i (w_rcp W - 2^64) / (W 2^64) stays below i / 2^64 < 1 / W); 0 for W = 1
    unsigned long long w_rcp;
    // Moments of each star ray's prefixes (device, may be null): entry
    // (j (steps + 1) + k) 6 + q holds, over the entries of ray j before step
    // k that only this ray reaches, the sum of 1, u, v, u^2, u v, v^2 (q = 0..5)
    const int* star_pm;
    int* err;        // device error word
};

// Star-fill table.  cls: 0 = repeats the previous step of its ray (never
// stops the ray, adds nothing), 1 = offset reached by this ray only
// (accumulated when reached), 2 = offset reached by several rays (sets bit
// `bit`; accumulated once after all rays).
struct StarTable {
    int n;
    int nshared;
    int8_t ou[kMaxStar];
    int8_t ov[kMaxStar];
    uint8_t cls[kMaxStar];
    uint8_t bit[kMaxStar];
    int8_t sou[kMaxShared];
    int8_t sov[kMaxShared];
};

struct Workspace {
    int* err = nullptr;        // device error word
    float* den = nullptr;      // W x H floats, used by run_frame when the caller passes no den
    size_t den_pitch = 0;
    int32_t* count = nullptr;  // component counter when the caller passes none
};

// Counts kernel launches and, when `ev` is set, records one event after
// each stage slot (a slot whose kernel is not needed still gets its event).
struct Marks {
    cudaEvent_t* ev = nullptr;
    int n = 0;
    unsigned long long launches = 0;
    void after(cudaStream_t s, bool launched = true) {
        if (launched) launches++;
        if (ev) cudaEventRecord(ev[n++], s);
    }
};

// Guard band factors (1 + e, 1 - e) of the FP32 reciprocal covered-depth test
// for K = rint(2^16 k).
void cd_band(int K, float* hi, float* lo);

// ceil(2^64 / W) (UINT64_MAX / W + 1 equals it whether or not W divides
// 2^64), 0 for W < 2.
inline unsigned long long w_reciprocal(int W) { return W < 2 ? 0ull : ~0ull / (unsigned long long)W + 1ull; }

// The FP32 reciprocal of every code 0..kDMax as the kernels compute it,
// copied to host memory (kDMax + 1 floats).
cudaError_t rcp_codes(float* host_out);

// Checks camera, size and parameters and fills the kernel constants without
// touching the device.
sn_status prepare_constants(const sn_camera* cam, int W, int H, const sn_params* p, Geo* g, StarTable* t);

// Launchers (return cudaGetLastError() of their launches).
cudaError_t launch_denoise(const Geo& g, const void* disp, size_t dp, float* den, size_t denp,
                           uint8_t* mask, size_t mp, cudaStream_t s, Marks& mk);
cudaError_t launch_affine(const Geo& g, const StarTable& t, const void* disp, size_t dp,
                          const float* den, size_t denp, void* nrm, size_t np, uint8_t* mask,
                          size_t mp, bool mask_or, cudaStream_t s, Marks& mk);
cudaError_t launch_points(const Geo& g, const float* den, size_t denp, const uint8_t* mask,
                          size_t mp, float* pts, size_t pp, cudaStream_t s, Marks& mk);
// three stage slots: tile-local union-find, border merge, flatten
cudaError_t launch_components(const Geo& g, const void* disp, size_t dp, int32_t* labels,
                              size_t lp, int32_t* count, cudaStream_t s, Marks& mk);
// stage kernels on the fused kernel's fast paths (5x5 denoise; M = 8, s = 10 star)
cudaError_t launch_denoise5(const Geo& g, const void* disp, size_t dp, float* den, size_t denp, uint8_t* mask,
                            size_t mp, cudaStream_t s);
cudaError_t launch_affine_star8(const Geo& g, const void* disp, size_t dp, const float* den, size_t denp, void* nrm,
                                size_t np, uint8_t* mask, size_t mp, bool mask_or, cudaStream_t s);
// comparison estimators (one stage slot each)
cudaError_t launch_cross(const Geo& g, const void* disp, size_t dp, void* nrm, size_t np, uint8_t* mask,
                         size_t mp, cudaStream_t s, Marks& mk);
cudaError_t launch_pca(const Geo& g, const void* disp, size_t dp, int r, void* nrm, size_t np, uint8_t* mask,
                       size_t mp, cudaStream_t s, Marks& mk);
// two stage slots: border merge between tw x th tiles, flatten
cudaError_t launch_ccl_merge_flatten(const Geo& g, const void* disp, size_t dp, int32_t* labels,
                                     size_t lp, int32_t* count, int tw, int th, cudaStream_t s,
                                     Marks& mk);

// Outputs of sn_run_frame.  The fused frame kernel writes den (when given),
// normals, points and mask; the component passes write labels and count.
// Star-fill with M = 8, s = 10 uses compile-time rays when `star8` is set
// (the host checks that the context's table is exactly that ray set).
struct FrameOut {
    float* den;  // may be null
    size_t denp;
    void* nrm;
    size_t np;
    float* pts;
    size_t pp;
    int32_t* labels;
    size_t lp;
    uint8_t* mask;
    size_t mp;
    int32_t* count;
};
constexpr int kFrameTW = 32;
constexpr int kFrameTH = 16;
// Learned gate weights as the frame kernel reads them (device pointers).
struct GateView {
    const __nv_bfloat16* W1g;  // [16][80]
    const __nv_bfloat16* W2g;  // [16][144]
    const float* b1;
    const float* b2;
    const float* W3;
    const float* b3;
    float tau;
    // The B operands of the two convolutions as the gate kernel's shared
    // memory holds them (kNetImageBytes, written by launch_net_image), in
    // tcgen05 core-matrix layout: 3 and 9 K-steps of 512 bytes.
    const void* net;
    const float* log2tab;  // log2_table()
    // The epilogue constants (kernel parameters, read from the constant
    // bank): b1, -b2, W3 rounded to BF16 as every weight of the network, and
    // c3 = b3 + sum W3 b2 (FP32 multiply-adds in channel order), so that
    // W3 . relu(acc + b2) + b3 = W3 . max(acc, -b2) + c3.
    struct {
        float b1[16], nb2[16], w3[16], c3;
    } k;
};
constexpr int kNetImageBytes = 3 * 512 + 9 * 512;
// Fills gv->k from the FP32 parameter vector (host).
void gate_constants(const float* theta, GateView* gv);
// Builds the image `net` from the other GateView fields.
cudaError_t launch_net_image(const GateView& gv, void* img, cudaStream_t s);
// Device address of the table of log2 of every disparity code (FP32,
// correctly rounded; NaN for code 0) on the current device, filled by the
// first call on that device (synchronously; not under stream capture).
cudaError_t log2_table(const float** out);
// The learned form: the gate kernel (network on the tensor cores, gate bits
// into o.mask), then the chain kernel (certified pixels on the full window,
// the others on the plain chain).  q != nullptr: only the gate kernel,
// writing q at the pixels with both coordinates even and NaN at the others
// (W x H floats, rows qp bytes apart).
cudaError_t launch_learned(const Geo& g, const void* disp, size_t dp, const FrameOut& o, const GateView& gv, float* q,
                           size_t qp, cudaStream_t s);
// The fused frame kernel alone (denoise, support, fit, normal, point, mask;
// not the labels).  gv == nullptr: plain chain; otherwise the learned
// kernel (star M = 8, s = 10, r_d = 2).
cudaError_t launch_frame(const Geo& g, const StarTable& t, bool star8, const void* disp, size_t dp,
                         const FrameOut& o, const GateView* gv, cudaStream_t s, Marks& mk);
// The fixed (2 r_a + 1)^2 window with the 5 x 5 denoise (2 <= r_a <= 7,
// r_d = 2; window_supported) in its convolution form: one fused kernel like
// launch_frame's.
bool window_supported(const Geo& g);
cudaError_t launch_window(const Geo& g, const void* disp, size_t dp, const FrameOut& o, cudaStream_t s);
bool star_is_m8(const StarTable& t, int dirs, int steps);
// Host: the prefix moments of the table's rays (dirs (steps + 1) 6 ints; see
// Geo::star_pm).
void star_prefix_moments(const StarTable& t, int dirs, int steps, int* pm);
// Tensor map of a disparity image (the context's input type) for TMA tile
// loads: W x H elements, rows `pitch` bytes apart (16-byte aligned base and
// pitch), box bw x bh elements, zero outside the image.
cudaError_t encode_disp_map(CUtensorMap* m, const void* disp, size_t pitch, int W, int H, int in_dtype, int bw,
                            int bh);

}  // namespace sn
