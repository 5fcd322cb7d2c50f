// The fixed 9 x 9 window (r_a = 4) with the 5 x 5 range-gated denoise, in
// the convolution form of Sec. III-C: every sum the two fits need over a
// square window is a separable sum of per-sample terms (1, u, u^2, D, u D
// along a row; then weights 1, v, v^2 along the column), so a row pass
// over the staged tile and a column pass over the row sums give every
// pixel's sums at a cost per pixel that no longer grows with the window's
// area.
//
// Denoise: where every valid sample of a pixel's 5 x 5 window passes the
// range gate (the usual case: one surface), the gated fit takes exactly the
// valid samples, whose sums the separable passes give.  The test needs the
// window's smallest and largest valid code (also separable).  The other
// valid pixels are compacted into a list and take the gated fit sample by
// sample (denoise_exact), then the same window sums for the affine fit.
// Both routes give the same integers as the direct fits, hence the same
// outputs bit for bit.
#include <atomic>

#include <cuda.h>  // CUtensorMap
#include <cudaTypedefs.h>

#include "sn_pixel.cuh"

namespace sn {

namespace {

constexpr int kWR = 4;                     // the window's radius r_a
constexpr int kWTH = 16;                   // tile rows; 32 x 8 threads, two pixels each (rows ty, ty + 8)
constexpr int kWNT = kTW * 8;              // threads per CTA
constexpr int kWTW = kTW + 2 * kWR;        // 40 staged columns
constexpr int kWTHR = kWTH + 2 * kWR;      // 24 staged rows
constexpr int kWRS = kWTHR * kTW;          // row sums: every staged row, the tile's 32 columns
static_assert(kWRS % kWNT == 0, "whole row-pass rounds");
constexpr size_t kWOffTile = 0;
constexpr size_t kWOffRS9 = align128z(sizeof(int2) * kWTW * kWTHR);
constexpr size_t kWOffRS5 = kWOffRS9 + sizeof(int4) * kWRS;
constexpr size_t kWOffMM = kWOffRS5 + sizeof(int4) * kWRS;
constexpr size_t kWOffList = kWOffMM + sizeof(int2) * kWRS;
constexpr size_t kWOffCnt = kWOffList + sizeof(int) * kTW * kWTH;
constexpr size_t kWSmem = align128z(kWOffCnt + 16);
// the raw TMA box (and its mbarrier) lies where the 9-wide row sums go
static_assert(tma_bw<SN_IN_F32, kWR, kWTW>() * kWTHR * 4 + 8 <= sizeof(int4) * kWRS, "raw box inside the row sums");

// Row sums of one staged entry over |u| <= h, from the packed words
// E = D + 2^23 [D > 0] (D < 2^17).  Over at most 9 samples with |u| <= 4:
// sum E = sum D + 2^23 n with sum D < 9 * 2^17 < 2^23; sum u E = sum u D +
// 2^23 sum u with |sum u D| <= 20 * 2^17 < 2^22; sum u^2 E = sum u^2 D +
// 2^23 sum u^2 with sum u^2 D <= 60 * 2^17 < 2^23.  Unpacked into
// (n + 2^16 sum u, sum u^2, sum D, sum u D).
__device__ __forceinline__ int4 unpack_row(int Q0, int Q1, int Q2) {
    const int n = Q0 >> 23, SD = Q0 & 0x7FFFFF;
    const int Su = (Q1 + (1 << 22)) >> 23;
    const int SuD = Q1 - Su * (1 << 23);
    return make_int4(n + Su * 65536, Q2 >> 23, SD, SuD);
}

// Column pass over rows j = -H .. H of the row sums (A = n + 2^16 sum u per
// row, B = sum u^2, sum D, sum u D): sum A = n + 2^16 Su, sum j A = Sv +
// 2^16 Suv, sum j^2 A = Svv + 2^16 (sum v^2 u), each low field within its
// 16 bits (n <= 81, |Sv| <= 180, Svv <= 540).
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

// The affine fit over the 9 x 9 window's valid samples except the centre
// (sums wa include the centre, which adds only to n and SD), anchored at
// the denoised centre; normal, point and mask.  The window bounds the
// moments like the M = 8, s = 10 star (alpha gamma <= 540^2), so the 32-bit
// solve applies.
__device__ __forceinline__ void window_affine(const Geo& g, int Dc, bool fit, long long num, long long det,
                                              const WinSums& wa, int x, int y, PixOut& r) {
    pix_zero(r);
    r.m = SN_MASK_VALID;
    const float dcf = fit ? i64_to_f32(num) / (float)(int)det : 0.0f;  // 5x5: det below 2^24
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
    if (solve_normal_dc<true>(s, Dc, dcf, [=] { return fit ? (double)num / (double)det : 0.0; }, r.dtil, x, y, g,
                              r.n, fp64))
        r.m |= SN_MASK_NORMAL | (fp64 ? SN_MASK_FP64 : 0);
    pix_points(g, x, y, r);
}

template <int IN>
__global__ void __launch_bounds__(kWNT, 4)
    k_window(const Geo g, const char* __restrict__ disp, size_t dp, const FrameOut o,
             const __grid_constant__ CUtensorMap dmap) {
    extern __shared__ __align__(128) unsigned char smem[];
    int2* tile = reinterpret_cast<int2*>(smem + kWOffTile);
    int4* rs9 = reinterpret_cast<int4*>(smem + kWOffRS9);
    int4* rs5 = reinterpret_cast<int4*>(smem + kWOffRS5);
    int2* mm5 = reinterpret_cast<int2*>(smem + kWOffMM);
    int* list = reinterpret_cast<int*>(smem + kWOffList);
    int* cnt = reinterpret_cast<int*>(smem + kWOffCnt);
    const int lane = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * kTW + lane;
    const int x0 = blockIdx.x * kTW, y0 = blockIdx.y * kWTH;
    if (tid == 0) *cnt = 0;
    stage_tile<IN, kWR, kWTH, kWNT>(tile, smem + kWOffRS9, &dmap, true, disp, dp, x0, y0, g, kStagePacked);

    // ---- row pass: every staged row, the tile's columns; |u| <= 2 first
    // (with the smallest valid code minus 1, as unsigned, and the largest
    // code), then |u| <= 4
#pragma unroll
    for (int k = 0; k < kWRS / kWNT; k++) {
        const int e = tid + k * kWNT;
        const int2* p = tile + (e / kTW) * kWTW + e % kTW + kWR;
        int Q0 = 0, Q1 = 0, Q2 = 0, mx = 0;
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
        rs5[e] = unpack_row(Q0, Q1, Q2);
        mm5[e] = make_int2((int)mn, mx);
#pragma unroll
        for (int a = 3; a <= kWR; a++) {
#pragma unroll
            for (int sgn = -1; sgn <= 1; sgn += 2) {
                const int u = sgn * a;
                const int E = p[u].y;
                Q0 += E;
                Q1 += u * E;
                Q2 += (u * u) * E;
            }
        }
        rs9[e] = unpack_row(Q0, Q1, Q2);
    }
    __syncthreads();

    // ---- each thread's two pixels: the fast route where the 5x5 gate
    // passes every valid sample, else onto the list
    bool need[2];
#pragma unroll
    for (int k = 0; k < 2; k++) {
        const int row = ty + 8 * k, x = x0 + lane, y = y0 + row;
        const int e0 = (row + kWR) * kTW + lane;
        const int Dc = tile[(row + kWR) * kWTW + lane + kWR].x;  // 0 outside the image
        const bool inside = x < g.W && y < g.H;
        need[k] = false;
        if (!inside) continue;
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
        if ((int)mn + 1 < Dc - lo || mx > Dc + thr) {
            need[k] = true;
            continue;
        }
        const WinSums w2 = column_sums<2>(rs5, e0);
        long long num, det;
        const bool fit = denoise_from_sums(w2, Dc, num, det);
        window_affine(g, Dc, fit, num, det, column_sums<kWR>(rs9, e0), x, y, r);
        emit(g, o, x, y, r);
    }

    // ---- the others, compacted so that whole warps take the sample-by-sample gate
#pragma unroll
    for (int k = 0; k < 2; k++) {
        const unsigned m = __ballot_sync(0xffffffffu, need[k]);
        int base = 0;
        if (lane == 0 && m) base = atomicAdd(cnt, __popc(m));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (need[k]) list[base + __popc(m & ((1u << lane) - 1u))] = (ty + 8 * k) * kTW + lane;
    }
    __syncthreads();
    const int nl = *cnt;
    for (int i = tid; i < nl; i += kWNT) {
        const int p = list[i];
        const int px = p % kTW, py = p / kTW;
        const int2* c = tile + (py + kWR) * kWTW + px + kWR;
        const int Dc = c[0].x;
        long long num, det;
        const bool fit = denoise_exact<2>(c, kWTW, 2, Dc, g.K_range, num, det);
        PixOut r;
        window_affine(g, Dc, fit, num, det, column_sums<kWR>(rs9, (py + kWR) * kTW + px), x0 + px, y0 + py, r);
        emit(g, o, x0 + px, y0 + py, r);
    }
}

template <int IN>
cudaError_t launch_window_in(const Geo& g, const void* disp, size_t dp, const FrameOut& o, cudaStream_t s) {
    CUtensorMap dmap{};
    const cudaError_t me = encode_disp_map(&dmap, disp, dp, g.W, g.H, IN, tma_bw<IN, kWR, kWTW>(), kWTHR);
    if (me != cudaSuccess) return me;
    static std::atomic<unsigned long long> done{0};
    const cudaError_t e = smem_limit_once(k_window<IN>, kWSmem, done);
    if (e != cudaSuccess) return e;
    const dim3 grid((g.W + kTW - 1) / kTW, (g.H + kWTH - 1) / kWTH), block(kTW, 8);
    k_window<IN><<<grid, block, kWSmem, s>>>(g, static_cast<const char*>(disp), dp, o, dmap);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_window(const Geo& g, const void* disp, size_t dp, const FrameOut& o, cudaStream_t s) {
    switch (g.in_dtype) {
        case SN_IN_F32: return launch_window_in<SN_IN_F32>(g, disp, dp, o, s);
        case SN_IN_F16: return launch_window_in<SN_IN_F16>(g, disp, dp, o, s);
        default: return launch_window_in<SN_IN_U16X256>(g, disp, dp, o, s);
    }
}

}  // namespace sn
