// Fused frame kernel: one pass over 32 x 8 (compile-time star) or 32 x 16
// pixel tiles computes the denoised disparity, the support (fixed window or
// star-fill), the affine fit, the normal, the point and the mask.  The
// component labels come from the separate run-based passes (k_ccl_local,
// k_ccl_merge, k_ccl_flatten), which need only the ingested codes and run
// beside this kernel on a side stream.  The tile and its halo are staged
// once in shared memory (by one TMA copy where the halo is fixed at compile
// time) as (D, 1/D) pairs: D is the exact integer disparity code used by
// every sum and decision, 1/D (FP32, within 1 ulp; +inf for invalid)
// carries the covered-depth test, which in reciprocal form reads
// 1/Dmin - 1/Dmax > K / (2^16 Dc).
#include <atomic>

#include <cuda.h>  // CUtensorMap (the encoder is reached through the runtime's driver entry point)
#include <cuda_bf16.h>
#include <cudaTypedefs.h>
#include <mutex>

#include "sn_pixel.cuh"

namespace sn {

namespace {

// tile (D, 1/D) (+ one ST edge byte per tile entry) of a 32 x TH tile
__host__ __device__ constexpr size_t frame_smem(int Rr, bool st = false, int TH = kTH) {
    return sizeof(int2) * (size_t)(kTW + 2 * Rr) * (TH + 2 * Rr) + (st ? (size_t)(kTW + 2 * Rr) * (TH + 2 * Rr) : 0);
}

constexpr bool frame_tma(int VAR, int R) { return R > 0 && (VAR == 0 || VAR == 2 || VAR == 5); }
// Offset and size of the raw box (then its 8-byte mbarrier) after the
// variant's other shared memory.
template <int IN, int VAR, int R>
__host__ __device__ constexpr size_t tma_raw_off() {
    return align128z(frame_smem(R, false, frame_th(VAR)));
}
template <int IN, int VAR, int R>
__host__ __device__ constexpr int tma_raw_bytes() {
    return tma_bw<IN, R, kTW + 2 * R>() * (frame_th(VAR) + 2 * R) * tma_esize<IN>();
}

// VAR: 0 fixed window of a runtime radius (radii 2..7 with the 5x5 denoise
// have their own kernel, k_window), 1 star table, 2 compile-time M = 8,
// s = 10 star, 4 star table with the ST stop, 5 = 2 with the ST stop instead
// of the covered-depth test (the learned form has its own kernels, k_gate and
// k_learned).  R: halo radius at compile time (0 = runtime).
// RD: denoise radius (0 = runtime).
template <int IN, int VAR, int R, int RD>
__global__ void __launch_bounds__(kTW* frame_th(VAR), 1024 / (kTW * frame_th(VAR)))
    k_frame(const Geo g, const __grid_constant__ StarTable T, const char* __restrict__ disp, size_t dp,
            const FrameOut o, const __grid_constant__ CUtensorMap dmap) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int TH = frame_th(VAR), NT = kTW * TH;
    // ST needs the edge bit of every pixel a ray can reach: one more halo row
    const int Rr = R > 0 ? R : max(g.r_d, VAR == 0 ? g.r_a : (VAR == 4 ? g.steps + 1 : g.steps));
    const int TWR = kTW + 2 * Rr, THR = TH + 2 * Rr;
    int2* tile = reinterpret_cast<int2*>(smem);
    uint8_t* Est = reinterpret_cast<uint8_t*>(smem + sizeof(int2) * (size_t)TWR * THR);  // ST edge bytes (VAR 4)
    const int x0 = blockIdx.x * kTW, y0 = blockIdx.y * TH;
    const int tid = threadIdx.y * kTW + threadIdx.x;

    // ---- stage the tile and its halo: (D, 1/D)
    const int n = TWR * THR;
    if constexpr (frame_tma(VAR, R)) {
        stage_tile<IN, R, TH, NT>(tile, smem + tma_raw_off<IN, VAR, R>(), &dmap, true, disp, dp, x0, y0, g, kStageRcp);
    } else {
        for (int i = tid; i < n; i += NT) {
            const int ly = i / TWR;
            const int lx = i - ly * TWR;
            const int D = load_code<IN>(disp, dp, x0 - Rr + lx, y0 - Rr + ly, g.W, g.H);
            const float w = D > 0 ? rcp_approx((float)D) : __int_as_float(0x7f800000);
            tile[i] = make_int2(D, __float_as_int(w));
        }
        __syncthreads();
    }
    if constexpr (VAR == 5) {
        // ST edges folded into the tile: 1/D = +inf for every pixel that stops
        // a ray (invalid, or |depth Laplacian| > t; the outer ring, which no
        // ray reaches, too).  Only the .y words change, the edge tests read .x.
        for (int i = tid; i < n; i += NT) {
            const int ly = i / TWR, lx = i - ly * TWR;
            bool e = true;
            if (lx > 0 && lx < TWR - 1 && ly > 0 && ly < THR - 1)
                e = st_edge(g, tile[i].x, tile[i - 1].x, tile[i + 1].x, tile[i - TWR].x, tile[i + TWR].x);
            if (e) tile[i].y = 0x7f800000;
        }
        __syncthreads();
    }
    if constexpr (VAR == 4) {
        for (int i = tid; i < n; i += NT) {
            const int ly = i / TWR, lx = i - ly * TWR;
            bool e = true;  // the outer ring is never reached by a ray
            if (lx > 0 && lx < TWR - 1 && ly > 0 && ly < THR - 1)
                e = st_edge(g, tile[i].x, tile[i - 1].x, tile[i + 1].x, tile[i - TWR].x, tile[i + TWR].x);
            Est[i] = e;
        }
        __syncthreads();
    }

    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    const bool inside = x < g.W && y < g.H;
    const int2* c = tile + (threadIdx.y + Rr) * TWR + threadIdx.x + Rr;
    const int Dc = c[0].x;  // 0 outside the image

    if (inside) {
        PixOut r;
        plain_pixel<VAR, R, RD>(g, &T, c, TWR, x, y, r, Est + (c - tile));
        emit(g, o, x, y, r);
    }
}

template <int IN, int VAR, int R, int RD>
cudaError_t launch_in(const Geo& g, const StarTable& t, const char* d, size_t dp, const FrameOut& o,
                      cudaStream_t s) {
    constexpr int Rmax = R > 0 ? R : (VAR == 0 ? 15 : (VAR == 4 ? kMaxSteps + 1 : kMaxSteps));
    const int Rr = R > 0 ? R : max(g.r_d, VAR == 0 ? g.r_a : (VAR == 4 ? g.steps + 1 : g.steps));
    constexpr int TH = frame_th(VAR);
    constexpr bool kTma = frame_tma(VAR, R);
    const size_t bytes = kTma ? tma_raw_off<IN, VAR, R>() + tma_raw_bytes<IN, VAR, R>() + 16
                              : frame_smem(Rr, VAR == 4, TH);
    const size_t bytes_max = kTma ? bytes : frame_smem(Rmax, VAR == 4, TH);
    CUtensorMap dmap{};
    if constexpr (kTma) {
        const cudaError_t me = encode_disp_map(&dmap, d, dp, g.W, g.H, IN, tma_bw<IN, R, kTW + 2 * R>(), TH + 2 * R);
        if (me != cudaSuccess) return me;
    }
    const dim3 grid((g.W + kTW - 1) / kTW, (g.H + TH - 1) / TH), block(kTW, TH);
    static std::atomic<unsigned long long> done{0};
    const cudaError_t e = smem_limit_once(k_frame<IN, VAR, R, RD>, bytes_max, done);
    if (e != cudaSuccess) return e;
    k_frame<IN, VAR, R, RD><<<grid, block, bytes, s>>>(g, t, d, dp, o, dmap);
    return cudaGetLastError();
}

template <int VAR, int R, int RD>
cudaError_t launch_var(const Geo& g, const StarTable& t, const void* disp, size_t dp, const FrameOut& o,
                       cudaStream_t s) {
    const char* d = static_cast<const char*>(disp);
    switch (g.in_dtype) {
        case SN_IN_F32: return launch_in<SN_IN_F32, VAR, R, RD>(g, t, d, dp, o, s);
        case SN_IN_F16: return launch_in<SN_IN_F16, VAR, R, RD>(g, t, d, dp, o, s);
        default: return launch_in<SN_IN_U16X256, VAR, R, RD>(g, t, d, dp, o, s);
    }
}

// ---------------------------------------------------------------- stage kernels on the fast paths
// sn_denoise with the 5x5 window and sn_affine_normals with the M = 8, s = 10
// star, on the fused kernel's code: the popcount denoise and the branch-free
// compile-time rays over a (D, 1/D) tile.  32 x 8 tiles, 4 CTAs per SM.
constexpr int kSTH = 8;

template <int IN>
__global__ void __launch_bounds__(kTW* kSTH, 4)
    k_denoise5(const Geo g, const char* __restrict__ disp, size_t dp, float* __restrict__ den, size_t denp,
               uint8_t* __restrict__ mask, size_t mp) {
    // plain loads: for the 2-pixel halo a TMA box measured slower
    constexpr int R = 2, TW = kTW + 2 * R, N = TW * (kSTH + 2 * R);
    __shared__ int2 tile[N];
    const int x0 = blockIdx.x * kTW, y0 = blockIdx.y * kSTH;
    for (int i = threadIdx.y * kTW + threadIdx.x; i < N; i += kTW * kSTH) {
        const int ly = i / TW, lx = i - ly * TW;
        tile[i] = make_int2(load_code<IN>(disp, dp, x0 - R + lx, y0 - R + ly, g.W, g.H), 0);
    }
    __syncthreads();
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    if (x >= g.W || y >= g.H) return;
    const int2* c = tile + (threadIdx.y + R) * TW + threadIdx.x + R;
    const int Dc = c[0].x;
    float out = 0.0f;
    uint8_t m = 0;
    if (Dc > 0) {
        long long num, det;
        const bool fit = denoise_exact<2>(c, TW, 2, Dc, g.K_range, num, det);
        const float dcf = fit ? i64_to_f32(num) / (float)(int)det : 0.0f;  // 5x5: det below 2^24
        out = ((float)Dc + dcf) * (1.0f / 256.0f);
        m = SN_MASK_VALID | (fit ? SN_MASK_DENOISED : 0);
    }
    reinterpret_cast<float*>(reinterpret_cast<char*>(den) + (size_t)y * denp)[x] = out;
    mask[(size_t)y * mp + x] = m;
}

template <int IN>
__global__ void __launch_bounds__(kTW* kSTH, 4)
    k_affine_star8(const Geo g, const char* __restrict__ disp, size_t dp, const float* __restrict__ den,
                   size_t denp, char* __restrict__ nrm, size_t np, uint8_t* __restrict__ mask, size_t mp,
                   int mask_or, const __grid_constant__ CUtensorMap dmap, int use_tma) {
    constexpr int R = 10, TW = kTW + 2 * R;
    __shared__ int2 tile[TW * (kSTH + 2 * R)];
    __shared__ __align__(128) unsigned char raw[tma_bw<IN, R, TW>() * (kSTH + 2 * R) * tma_esize<IN>() + 16];
    const int x0 = blockIdx.x * kTW, y0 = blockIdx.y * kSTH;
    stage_tile<IN, R, kSTH, kTW * kSTH>(tile, raw, &dmap, use_tma, disp, dp, x0, y0, g, kStageRcp);
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    if (x >= g.W || y >= g.H) return;
    const int2* c = tile + (threadIdx.y + R) * TW + threadIdx.x + R;
    const int Dc = c[0].x;
    float n[3] = {0.0f, 0.0f, 0.0f};
    uint8_t m = 0;
    if (Dc > 0) {
        m = SN_MASK_VALID;
        const float dtil =
            __ldg(reinterpret_cast<const float*>(reinterpret_cast<const char*>(den) + (size_t)y * denp) + x);
        AffSums s;
        star8<10, TW>(c, Dc, __int_as_float(c[0].y), make_thr(g, Dc), s);
        bool fp64;
        if (solve_normal<true>(s, Dc, dtil, x, y, g, n, fp64)) m |= SN_MASK_NORMAL | (fp64 ? SN_MASK_FP64 : 0);
    }
    if (g.normal_fmt == SN_NORMALS_F32X3) {
        const size_t plane = (size_t)g.H * np;
        float* p0 = reinterpret_cast<float*>(nrm + (size_t)y * np) + x;
        p0[0] = n[0];
        *reinterpret_cast<float*>(reinterpret_cast<char*>(p0) + plane) = n[1];
        *reinterpret_cast<float*>(reinterpret_cast<char*>(p0) + 2 * plane) = n[2];
    } else {
        short4 q;
        q.x = snorm16(n[0]);
        q.y = snorm16(n[1]);
        q.z = snorm16(n[2]);
        q.w = 0;
        reinterpret_cast<short4*>(nrm + (size_t)y * np)[x] = q;
    }
    uint8_t* mo = mask + (size_t)y * mp + x;
    *mo = mask_or ? (uint8_t)(*mo | m) : m;
}

}  // namespace

// Tensor map of a disparity image for the TMA tile staging: W x H elements
// of the input type, rows `pitch` bytes apart (16-byte aligned base and
// pitch, checked by the C-ABI layer), box bw x bh, zero outside the image.
cudaError_t encode_disp_map(CUtensorMap* m, const void* disp, size_t pitch, int W, int H, int in_dtype, int bw,
                            int bh) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
    if (!encode) return cudaErrorNotSupported;
    const CUtensorMapDataType type = in_dtype == SN_IN_F32   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                     : in_dtype == SN_IN_F16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                             : CU_TENSOR_MAP_DATA_TYPE_UINT16;
    const cuuint64_t dims[2] = {(cuuint64_t)W, (cuuint64_t)H};
    const cuuint64_t strides[1] = {(cuuint64_t)pitch};
    const cuuint32_t box[2] = {(cuuint32_t)bw, (cuuint32_t)bh};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = encode(m, type, 2, const_cast<void*>(disp), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}


void star_prefix_moments(const StarTable& t, int dirs, int steps, int* pm) {
    for (int j = 0; j < dirs; j++) {
        int acc[6] = {0, 0, 0, 0, 0, 0};
        for (int k = 0; k <= steps; k++) {
            int* q = pm + (j * (steps + 1) + k) * 6;
            for (int i = 0; i < 6; i++) q[i] = acc[i];
            if (k == steps) break;
            const int e = j * steps + k;
            if (t.cls[e] != 1) continue;
            const int u = t.ou[e], v = t.ov[e];
            acc[0] += 1;
            acc[1] += u;
            acc[2] += v;
            acc[3] += u * u;
            acc[4] += u * v;
            acc[5] += v * v;
        }
    }
}

bool star_is_m8(const StarTable& t, int dirs, int steps) {
    if (dirs != 8 || steps != 10) return false;
    const int su[8] = {1, 1, 0, -1, -1, -1, 0, 1};
    const int sv[8] = {0, 1, 1, 1, 0, -1, -1, -1};
    const int len[8] = {10, diag_len(10), 10, diag_len(10), 10, diag_len(10), 10, diag_len(10)};
    for (int j = 0; j < 8; j++) {
        int tpos = 0;
        for (int k = 0; k < steps; k++) {
            const int e = j * steps + k;
            if (t.cls[e] == 0) continue;
            if (t.cls[e] != 1) return false;
            tpos++;
            if (t.ou[e] != su[j] * tpos || t.ov[e] != sv[j] * tpos) return false;
        }
        if (tpos != len[j]) return false;
    }
    return true;
}

cudaError_t launch_frame(const Geo& g, const StarTable& t, bool star8, const void* disp, size_t dp,
                         const FrameOut& o, const GateView* gv, cudaStream_t s, Marks& mk) {
    cudaError_t e;
    if (gv && star8 && g.r_d == 2) {
        e = launch_learned(g, disp, dp, o, *gv, nullptr, 0, s);  // the gate kernel, then the chain kernel
        mk.launches++;
    }
    else if (g.support == SN_SUPPORT_STARFILL_CD && star8)
        e = g.r_d == 2 ? launch_var<2, 10, 2>(g, t, disp, dp, o, s) : launch_var<2, 10, 0>(g, t, disp, dp, o, s);
    else if (g.support == SN_SUPPORT_STARFILL_CD)
        e = launch_var<1, 0, 0>(g, t, disp, dp, o, s);
    else if (g.support == SN_SUPPORT_STARFILL_ST && star8)
        e = g.r_d == 2 ? launch_var<5, 11, 2>(g, t, disp, dp, o, s) : launch_var<5, 11, 0>(g, t, disp, dp, o, s);
    else if (g.support == SN_SUPPORT_STARFILL_ST)
        e = launch_var<4, 0, 0>(g, t, disp, dp, o, s);
    else if (window_supported(g))
        e = launch_window(g, disp, dp, o, s);  // fixed windows up to 15x15 with the 5x5 denoise, convolution form
    else
        e = launch_var<0, 0, 0>(g, t, disp, dp, o, s);
    mk.after(s);
    return e;
}


// Tensor map of the stage kernels' TMA box (halo R, kSTH rows); use_tma is
// 0 if it cannot be made (the kernels then use plain loads).
template <int IN, int R>
int stage_map(const Geo& g, const void* disp, size_t dp, CUtensorMap* m) {
    return encode_disp_map(m, disp, dp, g.W, g.H, IN, tma_bw<IN, R, kTW + 2 * R>(), kSTH + 2 * R) == cudaSuccess;
}

cudaError_t launch_denoise5(const Geo& g, const void* disp, size_t dp, float* den, size_t denp, uint8_t* mask,
                            size_t mp, cudaStream_t s) {
    const dim3 grid((g.W + kTW - 1) / kTW, (g.H + kSTH - 1) / kSTH), block(kTW, kSTH);
    const char* d = static_cast<const char*>(disp);
    switch (g.in_dtype) {
        case SN_IN_F32: k_denoise5<SN_IN_F32><<<grid, block, 0, s>>>(g, d, dp, den, denp, mask, mp); break;
        case SN_IN_F16: k_denoise5<SN_IN_F16><<<grid, block, 0, s>>>(g, d, dp, den, denp, mask, mp); break;
        default: k_denoise5<SN_IN_U16X256><<<grid, block, 0, s>>>(g, d, dp, den, denp, mask, mp); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_affine_star8(const Geo& g, const void* disp, size_t dp, const float* den, size_t denp, void* nrm,
                                size_t np, uint8_t* mask, size_t mp, bool mask_or, cudaStream_t s) {
    const dim3 grid((g.W + kTW - 1) / kTW, (g.H + kSTH - 1) / kSTH), block(kTW, kSTH);
    const char* d = static_cast<const char*>(disp);
    char* n = static_cast<char*>(nrm);
    const int mo = mask_or ? 1 : 0;
    CUtensorMap m{};
    int t;
    switch (g.in_dtype) {
        case SN_IN_F32:
            t = stage_map<SN_IN_F32, 10>(g, disp, dp, &m);
            k_affine_star8<SN_IN_F32><<<grid, block, 0, s>>>(g, d, dp, den, denp, n, np, mask, mp, mo, m, t);
            break;
        case SN_IN_F16:
            t = stage_map<SN_IN_F16, 10>(g, disp, dp, &m);
            k_affine_star8<SN_IN_F16><<<grid, block, 0, s>>>(g, d, dp, den, denp, n, np, mask, mp, mo, m, t);
            break;
        default:
            t = stage_map<SN_IN_U16X256, 10>(g, disp, dp, &m);
            k_affine_star8<SN_IN_U16X256><<<grid, block, 0, s>>>(g, d, dp, den, denp, n, np, mask, mp, mo, m, t);
            break;
    }
    return cudaGetLastError();
}

}  // namespace sn
