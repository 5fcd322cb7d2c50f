// The fixed (2R + 1)^2 window (r_a = R, 2 <= R <= 7) with the 5 x 5
// range-gated denoise, in the convolution form of Sec. III-C: every sum the
// two fits need over a square window is a separable sum of per-sample terms
// (1, u, u^2, D, u D along a row; then weights 1, v, v^2 along the column),
// so a row pass over the staged tile and a column pass over the row sums
// give every pixel's sums at a cost per pixel that grows with the window's
// side, not its area.
//
// Denoise: where every valid sample of a pixel's 5 x 5 window passes the
// range gate (the usual case: one surface), the gated fit takes exactly the
// valid samples, whose sums the separable passes give.  The test needs the
// window's smallest and largest valid code (also separable).  The other
// valid pixels take the gated fit sample by sample (denoise_exact) in
// place: compacting them onto a list measured slower, its block barrier
// costing more than the divergence it saves.  Both routes give the same
// integers as the direct fits, hence the same outputs bit for bit.
#include <atomic>

#include <cuda.h>  // CUtensorMap
#include <cudaTypedefs.h>

#include "sn_pixel.cuh"

namespace sn {

namespace {

constexpr int kWTH = 16;       // tile rows; 32 x 8 threads, two pixels each (rows ty, ty + 8)
constexpr int kWNT = kTW * 8;  // threads per CTA

// Geometry and shared-memory layout of the kernel for window radius R.
template <int R>
struct Win {
    static_assert(R >= 2 && R <= 7, "window radius 2..7");
    static constexpr int HR = R;                  // halo (>= 2, the denoise's)
    static constexpr int TW = kTW + 2 * HR;       // staged columns
    static constexpr int THR = kWTH + 2 * HR;     // staged rows
    static constexpr int RS = THR * kTW;          // row sums: every staged row, the tile's 32 columns
    static constexpr int ROUNDS = (RS + kWNT - 1) / kWNT;
    static constexpr size_t OFF_TILE = 0;
    static constexpr size_t OFF_RSA = align128z(sizeof(int2) * TW * THR);  // the full window's row sums
    static constexpr size_t OFF_RS5 = OFF_RSA + sizeof(int4) * RS;
    static constexpr size_t OFF_MM = OFF_RS5 + sizeof(int4) * RS;
    static constexpr size_t SMEM = align128z(OFF_MM + sizeof(int2) * RS);
    // sums of u^2 E stay packed up to R = 5 (sum u^2 D <= 110 * 2^17 < 2^24)
    static constexpr bool PACKED_UU = R <= 5;
    // moments bounded as for the M = 8, s = 10 star (1024 alpha gamma < 2^31)
    // up to R = 5: the 32-bit solve
    static constexpr bool SOLVE32 = R <= 5;
};
static_assert(tma_bw<SN_IN_F32, 7, Win<7>::TW>() * Win<7>::THR * 4 + 8 <= sizeof(int4) * Win<7>::RS,
              "raw box inside the row sums");
static_assert(4 * (Win<7>::SMEM + 1024) <= 228 * 1024, "four CTAs per SM");

// Row sums of one staged entry, from the packed words E = D + 2^24 [D > 0]
// (D < 2^17) over |u| <= R <= 7 (at most 15 samples): sum E = sum D +
// 2^24 n with sum D < 15 * 2^17 < 2^24; sum u E = sum u D + 2^24 sum u with
// |sum u D| <= 56 * 2^17 < 2^23; sum u^2 E = sum u^2 D + 2^24 sum u^2 where
// that packs (R <= 5), else sum u^2 directly.  Unpacked into
// (n + 2^16 sum u, sum u^2, sum D, sum u D).
__device__ __forceinline__ int4 unpack_row(int Q0, int Q1, int Suu) {
    const int n = Q0 >> 24, SD = Q0 & 0xFFFFFF;
    const int Su = (Q1 + (1 << 23)) >> 24;
    const int SuD = Q1 - Su * (1 << 24);
    return make_int4(n + Su * 65536, Suu, SD, SuD);
}

// Column pass over rows j = -H .. H of the row sums (A = n + 2^16 sum u per
// row, B = sum u^2, sum D, sum u D): sum A = n + 2^16 Su, sum j A = Sv +
// 2^16 Suv, sum j^2 A = Svv + 2^16 (sum v^2 u), each low field within its
// 16 bits (n <= 225, |Sv| <= 840, Svv <= 4200 for H <= 7).
template <int H>
__device__ __forceinline__ WinSums column_sums(const int4* rs, int e0) {
    int SA = 0, SAv = 0, SAv2 = 0, SB = 0, SQ0 = 0, SQ0v = 0, SQ1 = 0;
#pragma unroll
    for (int j = -H; j <= H; j++) {
        const int4 a = rs[e0 + j * kTW];
        SA += a.x;
        SAv += j * a.x;
        SAv2 += (j * j) * a.x;
        SB += a.y;
        SQ0 += a.z;
        SQ0v += j * a.z;
        SQ1 += a.w;
    }
    WinSums w;
    w.n = SA & 0xFFFF;
    w.Su = (SA - w.n) >> 16;
    w.Sv = (int)(short)(SAv & 0xFFFF);
    w.Suv = (SAv - w.Sv) >> 16;
    w.Svv = SAv2 & 0xFFFF;
    w.Suu = SB;
    w.SD = SQ0;
    w.SuD = SQ1;
    w.SvD = SQ0v;
    return w;
}

// The affine fit over the window's valid samples except the centre (sums
// wa include the centre, which adds only to n and SD), anchored at the
// denoised centre; normal, point and mask.
template <bool SOLVE32>
__device__ __forceinline__ void window_affine(const Geo& g, int Dc, bool fit, long long num, long long det,
                                              const WinSums& wa, int x, int y, PixOut& r) {
    pix_zero(r);
    r.m = SN_MASK_VALID;
    const float dcf = fit ? i64_to_f32(num) * rcp_approx((float)(int)det) : 0.0f;  // 5x5: det below 2^24
    if (fit) r.m |= SN_MASK_DENOISED;
    r.dtil = ((float)Dc + dcf) * (1.0f / 256.0f);
    AffSums s;
    s.N = wa.n - 1;
    s.Su = wa.Su;
    s.Sv = wa.Sv;
    s.Suu = wa.Suu;
    s.Suv = wa.Suv;
    s.Svv = wa.Svv;
    s.Bu = wa.SuD - Dc * wa.Su;
    s.Bv = wa.SvD - Dc * wa.Sv;
    bool fp64;
    if (solve_normal_dc<SOLVE32>(s, Dc, dcf, [=] { return fit ? (double)num / (double)det : 0.0; }, r.dtil, x, y,
                                 g, r.n, fp64))
        r.m |= SN_MASK_NORMAL | (fp64 ? SN_MASK_FP64 : 0);
    pix_points(g, x, y, r);
}

template <int IN, int R>
__global__ void __launch_bounds__(kWNT, 4)
    k_window(const Geo g, const char* __restrict__ disp, size_t dp, const FrameOut o,
             const __grid_constant__ CUtensorMap dmap) {
    using L = Win<R>;
    extern __shared__ __align__(128) unsigned char smem[];
    int2* tile = reinterpret_cast<int2*>(smem + L::OFF_TILE);
    int4* rsa = reinterpret_cast<int4*>(smem + L::OFF_RSA);
    int4* rs5 = reinterpret_cast<int4*>(smem + L::OFF_RS5);
    int2* mm5 = reinterpret_cast<int2*>(smem + L::OFF_MM);
    const int lane = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * kTW + lane;
    const int x0 = blockIdx.x * kTW, y0 = blockIdx.y * kWTH;
    // the raw TMA box (and its mbarrier) lies where the full window's row sums go
    stage_tile<IN, L::HR, kWTH, kWNT>(tile, smem + L::OFF_RSA, &dmap, true, disp, dp, x0, y0, g, kStagePacked);

    // ---- row pass: every staged row, the tile's columns; |u| <= 2 first
    // (with the smallest valid code minus 1, as unsigned, and the largest
    // code), then |u| <= R
#pragma unroll
    for (int k = 0; k < L::ROUNDS; k++) {
        const int e = tid + k * kWNT;
        if (L::RS % kWNT != 0 && e >= L::RS) break;
        const int2* p = tile + (e / kTW) * L::TW + e % kTW + L::HR;
        int Q0 = 0, Q1 = 0, Q2 = 0, B = 0, mx = 0;
        unsigned mn = 0xFFFFFFFFu;
#pragma unroll
        for (int u = -2; u <= 2; u++) {
            const int2 t = p[u];
            Q0 += t.y;
            Q1 += u * t.y;
            Q2 += (u * u) * t.y;
            mn = min(mn, (unsigned)(t.x - 1));
            mx = max(mx, t.x);
        }
        rs5[e] = unpack_row(Q0, Q1, Q2 >> 24);
        mm5[e] = make_int2((int)mn, mx);
        if constexpr (!L::PACKED_UU) B = Q2 >> 24;
#pragma unroll
        for (int a = 3; a <= R; a++) {
#pragma unroll
            for (int sgn = -1; sgn <= 1; sgn += 2) {
                const int u = sgn * a;
                const int E = p[u].y;
                Q0 += E;
                Q1 += u * E;
                if constexpr (L::PACKED_UU)
                    Q2 += (u * u) * E;
                else
                    B += (u * u) * (E >> 24);
            }
        }
        rsa[e] = unpack_row(Q0, Q1, L::PACKED_UU ? Q2 >> 24 : B);
    }
    __syncthreads();

    // ---- each thread's two pixels: the window sums where the 5x5 gate
    // passes every valid sample, else the gate sample by sample
#pragma unroll
    for (int k = 0; k < 2; k++) {
        const int row = ty + 8 * k, x = x0 + lane, y = y0 + row;
        const int e0 = (row + L::HR) * kTW + lane;
        const int Dc = tile[(row + L::HR) * L::TW + lane + L::HR].x;  // 0 outside the image
        if (x >= g.W || y >= g.H) continue;
        PixOut r;
        if (Dc <= 0) {
            pix_zero(r);
            emit(g, o, x, y, r);
            continue;
        }
        // the gate: -lo <= D - Dc <= thr, lo = min(thr, Dc - 1)
        const int thr = (int)(((unsigned long long)(unsigned)g.K_range * (unsigned)Dc) >> 16);
        const int lo = min(thr, Dc - 1);
        unsigned mn = 0xFFFFFFFFu;
        int mx = 0;
#pragma unroll
        for (int j = -2; j <= 2; j++) {
            const int2 m = mm5[e0 + j * kTW];
            mn = min(mn, (unsigned)m.x);
            mx = max(mx, m.y);
        }
        // the centre is valid, so mn + 1 is the window's smallest valid code
        long long num, det;
        bool fit;
        if ((int)mn + 1 < Dc - lo || mx > Dc + thr)
            fit = denoise_exact<2>(tile + (row + L::HR) * L::TW + lane + L::HR, L::TW, 2, Dc, g.K_range, num, det);
        else
            fit = denoise_from_sums(column_sums<2>(rs5, e0), Dc, num, det);
        window_affine<L::SOLVE32>(g, Dc, fit, num, det, column_sums<R>(rsa, e0), x, y, r);
        emit(g, o, x, y, r);
    }

}

template <int IN, int R>
cudaError_t launch_window_in(const Geo& g, const void* disp, size_t dp, const FrameOut& o, cudaStream_t s) {
    using L = Win<R>;
    CUtensorMap dmap{};
    const cudaError_t me = encode_disp_map(&dmap, disp, dp, g.W, g.H, IN, tma_bw<IN, L::HR, L::TW>(), L::THR);
    if (me != cudaSuccess) return me;
    static std::atomic<unsigned long long> done{0};
    const cudaError_t e = smem_limit_once(k_window<IN, R>, L::SMEM, done);
    if (e != cudaSuccess) return e;
    const dim3 grid((g.W + kTW - 1) / kTW, (g.H + kWTH - 1) / kWTH), block(kTW, 8);
    k_window<IN, R><<<grid, block, L::SMEM, s>>>(g, static_cast<const char*>(disp), dp, o, dmap);
    return cudaGetLastError();
}

template <int R>
cudaError_t launch_window_r(const Geo& g, const void* disp, size_t dp, const FrameOut& o, cudaStream_t s) {
    switch (g.in_dtype) {
        case SN_IN_F32: return launch_window_in<SN_IN_F32, R>(g, disp, dp, o, s);
        case SN_IN_F16: return launch_window_in<SN_IN_F16, R>(g, disp, dp, o, s);
        default: return launch_window_in<SN_IN_U16X256, R>(g, disp, dp, o, s);
    }
}

}  // namespace

bool window_supported(const Geo& g) {
    return g.support == SN_SUPPORT_FIXED && g.r_d == 2 && g.r_a >= 2 && g.r_a <= 7;
}

cudaError_t launch_window(const Geo& g, const void* disp, size_t dp, const FrameOut& o, cudaStream_t s) {
    switch (g.r_a) {
        case 2: return launch_window_r<2>(g, disp, dp, o, s);
        case 3: return launch_window_r<3>(g, disp, dp, o, s);
        case 4: return launch_window_r<4>(g, disp, dp, o, s);
        case 5: return launch_window_r<5>(g, disp, dp, o, s);
        case 6: return launch_window_r<6>(g, disp, dp, o, s);
        case 7: return launch_window_r<7>(g, disp, dp, o, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sn
