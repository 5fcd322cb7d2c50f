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

#include "sn_device.cuh"
#include "sn_umma.cuh"

namespace sn {

namespace {

constexpr int kTW = kFrameTW, kTH = kFrameTH, kThreads = kTW * kTH;
// Tile height of each variant.  The compile-time M = 8, s = 10 star takes
// 32 x 8 tiles, 4 CTAs of 256 threads per SM (more independent CTAs hide the
// barrier and staging stalls better than 2 CTAs of 512: 130 vs 139 us per
// 2048x1024 frame); the variants with larger halos (star tables up to s = 30,
// ST) and the learned one (whose network halo is amortised over more pixels)
// keep 32 x 16.
__host__ __device__ constexpr int frame_th(int var) { return var == 2 || var == 5 ? 8 : kTH; }

// distinct pixels of an M = 8 diagonal ray of s steps: round(s / sqrt 2),
// i.e. the r with (2r - 1)^2 < 2 s^2 < (2r + 1)^2
__host__ __device__ constexpr int diag_len(int s) {
    int r = 0;
    while ((2 * r + 1) * (2 * r + 1) < 2 * s * s) r++;
    return r;
}

// Covered-depth thresholds of one centre pixel.  `hi`/`lo` bracket the exact
// threshold K / (2^16 Dc) by the worst-case rounding of the FP32 reciprocals:
// above hi the exact test surely stops the ray, below lo it surely does not,
// in between the exact integer test decides.
struct Thr {
    float hi, lo;
    int K;
};

__device__ __forceinline__ Thr make_thr(const Geo& g, int Dc) {
    Thr t;
    t.K = g.K_cd;
    if (g.K_cd == 0) {
        // any spread stops; a zero spread is left to the exact test
        t.hi = 0.0f;
        t.lo = 0.0f;
    } else {
        const float thr = __fdiv_rn((float)g.K_cd * (1.0f / 65536.0f), (float)Dc);
        t.hi = thr * g.cd_hi;
        t.lo = thr * g.cd_lo;
    }
    return t;
}

// Reciprocal with at most 1 ulp error (PTX rcp.approx); the inputs are
// integer codes 1..131071, never denormal.
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Exact decision from the two extreme reciprocals: w is within 1 ulp of 1/D
// and D < 2^17, so rint(1/w) recovers D exactly.
__device__ __noinline__ bool cd_stop_from_w(float wlo, float whi, int Dc, int K) {
    const int Dmax = __float2int_rn(rcp_approx(wlo));
    const int Dmin = __float2int_rn(rcp_approx(whi));
    return cd_stop(Dmin, Dmax, Dc, K);
}

// Continues a ray from its first unsure step n + 1 with the exact integer
// test (taken only when a spread falls inside the rounding band).
template <int SU, int SV, int L, int STRIDE>
__device__ __noinline__ void ray8_exact_tail(const int2* __restrict__ c, int Dc, int K, int* n_io, int* A_io) {
    int n = *n_io, A = *A_io;
    int dmin = Dc, dmax = Dc;
    for (int t = 1; t <= n; t++) {
        const int D = c[(SV * t) * STRIDE + SU * t].x;
        dmin = min(dmin, D);
        dmax = max(dmax, D);
    }
    for (int t = n + 1; t <= L; t++) {
        const int D = c[(SV * t) * STRIDE + SU * t].x;
        if (D <= 0) break;
        const int nmin = min(dmin, D), nmax = max(dmax, D);
        if (cd_stop(nmin, nmax, Dc, K)) break;
        dmin = nmin;
        dmax = nmax;
        A += t * D;
        n = t;
    }
    *n_io = n;
    *A_io = A;
}

// One ray of the M = 8 star with direction (SU, SV) and L distinct pixels
// t (SU, SV), t = 1..L.  All L samples are loaded first; the walk is
// branch-free: a step is taken while the spread is surely below the
// threshold.  The running extremes stop moving after the first step that is
// not taken (the spread only grows, so no later step is taken either), so
// after the walk they give the spread of that step.  Only if it lies inside
// the rounding band does the exact test decide (and possibly continue the
// ray).  The data enters as A = sum t D over the included pixels; the
// moments of the included prefix 1..n are closed forms.
template <int SU, int SV, int L, int STRIDE>
__device__ __forceinline__ void ray8(const int2* __restrict__ c, int Dc, float wc, const Thr& th, AffSums& s) {
    int2 e[L];
#pragma unroll
    for (int t = 1; t <= L; t++) e[t - 1] = c[(SV * t) * STRIDE + SU * t];
    float wlo = wc, whi = wc;
    int A = 0, n = 0;
    bool alive = true;
#pragma unroll
    for (int t = 1; t <= L; t++) {
        const float w = __int_as_float(e[t - 1].y);
        if (alive) {
            wlo = fminf(wlo, w);
            whi = fmaxf(whi, w);
        }
        alive = whi - wlo < th.lo;
        if (alive) {
            A += t * e[t - 1].x;
            n++;
        }
    }
    if (n < L && !(whi - wlo > th.hi)) ray8_exact_tail<SU, SV, L, STRIDE>(c, Dc, th.K, &n, &A);
    const int T1 = (n * (n + 1)) >> 1;
    const int T2 = (n * (n + 1) * (2 * n + 1)) / 6;
    const int Ad = A - Dc * T1;
    s.N += n;
    if (SU != 0) {
        s.Su += SU * T1;
        s.Suu += T2;
        s.Bu += SU * Ad;
    }
    if (SV != 0) {
        s.Sv += SV * T1;
        s.Svv += T2;
        s.Bv += SV * Ad;
    }
    if (SU != 0 && SV != 0) s.Suv += SU * SV * T2;
}

template <int S, int STRIDE>
__device__ __forceinline__ void star8(const int2* c, int Dc, float wc, const Thr& th, AffSums& s) {
    constexpr int LD = diag_len(S);
    aff_zero(s);
    ray8<1, 0, S, STRIDE>(c, Dc, wc, th, s);
    ray8<1, 1, LD, STRIDE>(c, Dc, wc, th, s);
    ray8<0, 1, S, STRIDE>(c, Dc, wc, th, s);
    ray8<-1, 1, LD, STRIDE>(c, Dc, wc, th, s);
    ray8<-1, 0, S, STRIDE>(c, Dc, wc, th, s);
    ray8<-1, -1, LD, STRIDE>(c, Dc, wc, th, s);
    ray8<0, -1, S, STRIDE>(c, Dc, wc, th, s);
    ray8<1, -1, LD, STRIDE>(c, Dc, wc, th, s);
}

// Any star table (union of rays, see StarTable), on the packed tile.  With
// the rays' prefix moments (pm, see Geo::star_pm) a step accumulates only the
// data sums, and each ray adds the moments of the prefix it took.
__device__ __forceinline__ void star_table(const int2* c, int stride, int Dc, float wc, const Thr& th,
                                           const StarTable& T, int dirs, int steps, const int* __restrict__ pm,
                                           AffSums& s) {
    aff_zero(s);
    unsigned long long bits = 0ull;
    for (int j = 0; j < dirs; j++) {
        float wlo = wc, whi = wc;
        const int e0 = j * steps;
        int kend = steps;  // the ray takes steps 0 .. kend - 1
        for (int k = 0; k < steps; k++) {
            const int e = e0 + k;
            const int cls = T.cls[e];
            if (cls == 0) continue;
            const int ou = T.ou[e], ov = T.ov[e];
            const int2 v = c[ov * stride + ou];
            const float w = __int_as_float(v.y);
            const float lo = fminf(wlo, w), hi = fmaxf(whi, w);
            const float diff = hi - lo;
            if (diff > th.hi || (diff >= th.lo && cd_stop_from_w(lo, hi, Dc, th.K))) {
                kend = k;
                break;
            }
            wlo = lo;
            whi = hi;
            if (cls == 1) {
                if (pm) {
                    const int dd = v.x - Dc;
                    s.Bu += ou * dd;
                    s.Bv += ov * dd;
                } else {
                    aff_add(s, ou, ov, v.x - Dc);
                }
            } else {
                bits |= 1ull << T.bit[e];
            }
        }
        if (pm) {
            const int* q = pm + (j * (steps + 1) + kend) * 6;
            s.N += __ldg(q);
            s.Su += __ldg(q + 1);
            s.Sv += __ldg(q + 2);
            s.Suu += __ldg(q + 3);
            s.Suv += __ldg(q + 4);
            s.Svv += __ldg(q + 5);
        }
    }
    for (int b = 0; b < T.nshared; b++) {
        if ((bits >> b) & 1ull) {
            const int ou = T.sou[b], ov = T.sov[b];
            aff_add(s, ou, ov, c[ov * stride + ou].x - Dc);
        }
    }
}

// Star table with the ST stop on the packed tile: a ray stops before the
// first invalid or edge pixel (ec: the centre's entry of the edge bytes,
// laid out like the tile).
__device__ __forceinline__ void star_table_st(const int2* c, const uint8_t* ec, int stride, int Dc,
                                              const StarTable& T, int dirs, int steps, AffSums& s) {
    aff_zero(s);
    unsigned long long bits = 0ull;
    for (int j = 0; j < dirs; j++) {
        const int e0 = j * steps;
        for (int k = 0; k < steps; k++) {
            const int e = e0 + k;
            const int cls = T.cls[e];
            if (cls == 0) continue;
            const int ou = T.ou[e], ov = T.ov[e];
            const int Di = c[ov * stride + ou].x;
            if (Di <= 0 || ec[ov * stride + ou]) break;
            if (cls == 1)
                aff_add(s, ou, ov, Di - Dc);
            else
                bits |= 1ull << T.bit[e];
        }
    }
    for (int b = 0; b < T.nshared; b++) {
        if ((bits >> b) & 1ull) {
            const int ou = T.sou[b], ov = T.sov[b];
            aff_add(s, ou, ov, c[ov * stride + ou].x - Dc);
        }
    }
}

// Fixed (2R + 1)^2 window on the packed tile; RA > 0 fixes the radius (and
// the row stride STRIDE) at compile time, so the window unrolls.
template <int RA = 0, int STRIDE = 0>
__device__ __forceinline__ void fixed_packed(const int2* c, int stride, int R, int Dc, AffSums& s) {
    aff_zero(s);
    if constexpr (RA > 0) {
#pragma unroll
        for (int ov = -RA; ov <= RA; ov++) {
#pragma unroll
            for (int ou = -RA; ou <= RA; ou++) {
                const int Di = c[ov * STRIDE + ou].x;
                if (Di > 0 && (ou | ov) != 0) aff_add(s, ou, ov, Di - Dc);
            }
        }
    } else {
        for (int ov = -R; ov <= R; ov++) {
            const int2* row = c + ov * stride;
            for (int ou = -R; ou <= R; ou++) {
                const int Di = row[ou].x;
                if (Di > 0 && (ou | ov) != 0) aff_add(s, ou, ov, Di - Dc);
            }
        }
    }
}

// Denoise with exact intercept: returns fit and (num, det) with
// intercept = Dc + num / det (integer codes).  RD > 0 fixes the radius at
// compile time.
// bit (ov + 2) 5 + (ou + 2) of a 5x5 pass mask is set where q(ou, ov) == val,
// q = ou (kind 0), ov (kind 1) or ou ov (kind 2)
__host__ __device__ constexpr unsigned mask5(int kind, int val) {
    unsigned m = 0;
    for (int ov = -2; ov <= 2; ov++)
        for (int ou = -2; ou <= 2; ou++) {
            const int q = kind == 0 ? ou : (kind == 1 ? ov : ou * ov);
            if (q == val) m |= 1u << ((ov + 2) * 5 + (ou + 2));
        }
    return m;
}

__device__ __forceinline__ int popc_and(unsigned m, unsigned k) { return __popc(m & k); }

template <int RD>
__device__ __forceinline__ bool denoise_exact(const int2* c, int stride, int rd_rt, int Dc, int K_range,
                                              long long& num, long long& det) {
    const int R = RD > 0 ? RD : rd_rt;
    // -lo <= dd <= thr with lo = min(thr, Dc - 1): an invalid sample
    // (D = 0, dd = -Dc) never passes, whatever K_range is
    const int thr = (int)(((unsigned long long)(unsigned)K_range * (unsigned)Dc) >> 16);
    const int lo = min(thr, Dc - 1);
    const unsigned span = (unsigned)lo + (unsigned)thr;
    int n = 0, Su = 0, Sv = 0, Suu = 0, Suv = 0, Svv = 0, b0 = 0, b1 = 0, b2 = 0;
    if constexpr (RD == 2) {
        // 5x5: record the passing samples in a bit mask and take the moments
        // from population counts of column, row and product classes
        unsigned m = 0;
#pragma unroll
        for (int ov = -2; ov <= 2; ov++) {
#pragma unroll
            for (int ou = -2; ou <= 2; ou++) {
                const int dd = c[ov * stride + ou].x - Dc;
                if ((unsigned)(dd + lo) <= span) {
                    m |= 1u << ((ov + 2) * 5 + (ou + 2));
                    b0 += dd;
                    b1 += ou * dd;
                    b2 += ov * dd;
                }
            }
        }
        n = __popc(m);
        const int um2 = popc_and(m, mask5(0, -2)), um1 = popc_and(m, mask5(0, -1));
        const int up1 = popc_and(m, mask5(0, 1)), up2 = popc_and(m, mask5(0, 2));
        const int vm2 = popc_and(m, mask5(1, -2)), vm1 = popc_and(m, mask5(1, -1));
        const int vp1 = popc_and(m, mask5(1, 1)), vp2 = popc_and(m, mask5(1, 2));
        Su = 2 * (up2 - um2) + (up1 - um1);
        Suu = 4 * (up2 + um2) + (up1 + um1);
        Sv = 2 * (vp2 - vm2) + (vp1 - vm1);
        Svv = 4 * (vp2 + vm2) + (vp1 + vm1);
        Suv = (popc_and(m, mask5(2, 1)) - popc_and(m, mask5(2, -1))) +
              2 * (popc_and(m, mask5(2, 2)) - popc_and(m, mask5(2, -2))) +
              4 * (popc_and(m, mask5(2, 4)) - popc_and(m, mask5(2, -4)));
    } else {
#pragma unroll
        for (int ov = -R; ov <= R; ov++) {
#pragma unroll
            for (int ou = -R; ou <= R; ou++) {
                const int dd = c[ov * stride + ou].x - Dc;
                if ((unsigned)(dd + lo) <= span) {
                    n++;
                    Su += ou;
                    Sv += ov;
                    Suu += ou * ou;
                    Suv += ou * ov;
                    Svv += ov * ov;
                    b0 += dd;
                    b1 += ou * dd;
                    b2 += ov * dd;
                }
            }
        }
    }
    if constexpr (RD == 2) {
        // 5x5: |Su|, |Sv| <= 30, Suu, Svv <= 50, |Suv| <= 36, so the cofactors
        // (<= 2580) and det (<= 217,300) fit in 32 bits; num needs 64
        const int M00 = Suu * Svv - Suv * Suv;
        const int M10 = Su * Svv - Sv * Suv;
        const int M20 = Su * Suv - Sv * Suu;
        det = n * M00 - Su * M10 + Sv * M20;
        num = (long long)b0 * M00 - (long long)b1 * M10 + (long long)b2 * M20;
    } else {
        const long long M00 = (long long)Suu * Svv - (long long)Suv * Suv;
        const long long M10 = (long long)Su * Svv - (long long)Sv * Suv;
        const long long M20 = (long long)Su * Suv - (long long)Sv * Suu;
        det = n * M00 - Su * M10 + Sv * M20;
        num = b0 * M00 - b1 * M10 + b2 * M20;
    }
    return det > 0 && (long long)Dc * det + num > 0;
}

// Results of one pixel before they are stored.
struct PixOut {
    float n[3];
    float P[3];
    float dtil;
    uint8_t m;
};

__device__ __forceinline__ void pix_zero(PixOut& r) {
    r.n[0] = r.n[1] = r.n[2] = 0.0f;
    r.P[0] = r.P[1] = r.P[2] = 0.0f;
    r.dtil = 0.0f;
    r.m = 0;
}

__device__ __forceinline__ void pix_points(const Geo& g, int x, int y, PixOut& r) {
    const float inv = 1.0f / r.dtil;
    r.P[0] = g.B * ((float)x - g.cx) * inv;
    r.P[1] = g.B_fx_over_fy * ((float)y - g.cy) * inv;
    r.P[2] = g.fxB * inv;
}

__device__ __forceinline__ void emit(const Geo& g, const FrameOut& o, int x, int y, const PixOut& r) {
    if (o.den) reinterpret_cast<float*>(reinterpret_cast<char*>(o.den) + (size_t)y * o.denp)[x] = r.dtil;
    if (g.normal_fmt == SN_NORMALS_F32X3) {
        char* p0 = static_cast<char*>(o.nrm) + (size_t)y * o.np + (size_t)x * 4;
        const size_t plane = (size_t)g.H * o.np;
        *reinterpret_cast<float*>(p0) = r.n[0];
        *reinterpret_cast<float*>(p0 + plane) = r.n[1];
        *reinterpret_cast<float*>(p0 + 2 * plane) = r.n[2];
    } else {
        short4 q;
        q.x = snorm16(r.n[0]);
        q.y = snorm16(r.n[1]);
        q.z = snorm16(r.n[2]);
        q.w = 0;
        reinterpret_cast<short4*>(static_cast<char*>(o.nrm) + (size_t)y * o.np)[x] = q;
    }
    char* p0 = reinterpret_cast<char*>(o.pts) + (size_t)y * o.pp + (size_t)x * 4;
    const size_t plane = (size_t)g.H * o.pp;
    *reinterpret_cast<float*>(p0) = r.P[0];
    *reinterpret_cast<float*>(p0 + plane) = r.P[1];
    *reinterpret_cast<float*>(p0 + 2 * plane) = r.P[2];
    o.mask[(size_t)y * o.mp + x] = r.m;
}

// The plain per-pixel chain: range-gated denoise, support (fixed window or
// star-fill), two-pass fit, normal, point.  c points at the pixel in the tile.
template <int VAR, int R, int RD>
__device__ __forceinline__ void plain_pixel(const Geo& g, const StarTable& T, const int2* c, int TWR, int x, int y,
                                            PixOut& r, const uint8_t* ec = nullptr) {
    pix_zero(r);
    const int2 cc = c[0];
    const int Dc = cc.x;
    if (Dc <= 0) return;
    r.m = SN_MASK_VALID;
    long long num, det;
    const bool fit = denoise_exact<RD>(c, TWR, g.r_d, Dc, g.K_range, num, det);
    // a 5x5 det is below 2^24 (exact in FP32)
    const float dcf = fit ? i64_to_f32(num) / (RD == 2 ? (float)(int)det : i64_to_f32(det)) : 0.0f;
    if (fit) r.m |= SN_MASK_DENOISED;
    r.dtil = ((float)Dc + dcf) * (1.0f / 256.0f);
    AffSums s;
    if constexpr (VAR == 4) {
        star_table_st(c, ec, TWR, Dc, T, g.dirs, g.steps, s);
    } else if constexpr (VAR == 5) {
        // ST stop on the compile-time star: invalid and edge pixels carry
        // 1/D = +inf in this tile, so a ray is alive while its spread is
        // finite (lo = +inf) and never enters the exact tail (hi = -inf)
        static_assert(R == 11, "the M = 8, s = 10 star with the ST stop needs a halo of 11");
        const Thr st{-__int_as_float(0x7f800000), __int_as_float(0x7f800000), 0};
        star8<10, kTW + 2 * R>(c, Dc, rcp_approx((float)Dc), st, s);
    } else if constexpr (VAR >= 2) {
        static_assert(R == 10, "the M = 8, s = 10 star needs a halo of 10");
        star8<10, kTW + 2 * R>(c, Dc, __int_as_float(cc.y), make_thr(g, Dc), s);
    } else if constexpr (VAR == 1) {
        star_table(c, TWR, Dc, __int_as_float(cc.y), make_thr(g, Dc), T, g.dirs, g.steps, g.star_pm, s);
    } else if constexpr (R > 0) {
        fixed_packed<R, kTW + 2 * R>(c, TWR, R, Dc, s);  // compile-time 9x9 (R = r_a = 4 >= r_d)
    } else {
        fixed_packed(c, TWR, g.r_a, Dc, s);
    }
    bool fp64;
    if (solve_normal_dc<VAR == 2 || VAR == 3 || VAR == 5>(
            s, Dc, dcf, [=] { return fit ? (double)num / (double)det : 0.0; }, r.dtil, x, y, g, r.n, fp64))
        r.m |= SN_MASK_NORMAL | (fp64 ? SN_MASK_FP64 : 0);
    pix_points(g, x, y, r);
}

// Sums over the valid samples of a square window around a pixel (offsets
// u, v): moments and the data sums of D, u D, v D.
struct WinSums {
    int n, Su, Sv, Suu, Suv, Svv, SD, SuD, SvD;
};

// The learned fast path of a certified pixel (its (2 kFastR + 1)^2 window
// shows one surface): the denoise fit takes every valid sample of the 5x5
// window (no range gate) and the affine fit every valid sample of the full
// window except the centre (no star-fill).
__device__ __forceinline__ void fast_pixel(const Geo& g, int Dc, const WinSums& w2, const WinSums& wa, int x, int y,
                                           PixOut& r) {
    pix_zero(r);
    r.m = SN_MASK_VALID | SN_MASK_LEARNED;
    // the 5x5 window bounds the moments (as in denoise_exact<2>): the
    // cofactors and det fit in 32 bits, det below 2^24
    const int b0 = w2.SD - w2.n * Dc, b1 = w2.SuD - w2.Su * Dc, b2 = w2.SvD - w2.Sv * Dc;
    const int M00 = w2.Suu * w2.Svv - w2.Suv * w2.Suv;
    const int M10 = w2.Su * w2.Svv - w2.Sv * w2.Suv;
    const int M20 = w2.Su * w2.Suv - w2.Sv * w2.Suu;
    const int det = w2.n * M00 - w2.Su * M10 + w2.Sv * M20;
    const long long num = (long long)b0 * M00 - (long long)b1 * M10 + (long long)b2 * M20;
    const bool fit = det > 0 && (long long)Dc * det + num > 0;
    const float dcf = fit ? i64_to_f32(num) / (float)det : 0.0f;
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
    if (solve_normal_dc(s, Dc, dcf, [=] { return fit ? (double)num / (double)det : 0.0; }, r.dtil, x, y, g, r.n,
                        fp64))
        r.m |= SN_MASK_NORMAL | (fp64 ? SN_MASK_FP64 : 0);
    pix_points(g, x, y, r);
}

// The learned fast path fits the full (2 kFastR + 1)^2 window; the gate
// certifies it when the 5x5 patches centred within kQM of the pixel all show
// one surface (their union is the window).
constexpr int kFastR = SN_LEARNED_RADIUS, kQM = kFastR - 2;
static_assert(kFastR >= 3 && kFastR + 2 <= 10, "the features of the q region must lie inside the halo of 10");
constexpr int kFeatW = kTW + 2 * (kQM + 2), kFeatH = kTH + 2 * (kQM + 2);  // features: tile + kQM + 2
constexpr int kH1W = kTW + 2 * (kQM + 1), kH1H = kTH + 2 * (kQM + 1);      // layer 1:  tile + kQM + 1
constexpr int kQW = kTW + 2 * kQM, kQH = kTH + 2 * kQM;                    // q:        tile + kQM
constexpr int kFeatN = kFeatW * kFeatH;
constexpr int kQN = kQW * kQH;
constexpr int kRSRows = kTH + 2 * kFastR;   // row-sum rows: tile rows -kFastR .. kTH - 1 + kFastR
constexpr int kRS = kRSRows * kTW;          // row-sum entries per quantity
// Both 3x3 convolutions run as implicit GEMMs on the tcgen05 tensor cores
// (M = 128 rows per MMA, N = 16 channels, K = 16, BF16 in, FP32 in TMEM).
// Every map is stored row-major with the same pitch kPitch: output row m of a
// layer is position (m / kPitch, m % kPitch) of its map, and tap (dy, dx) of
// it reads input row m + dy kPitch + dx, so each tap's A operand is the input
// map at a constant offset (the columns past kH1W or kQW are computed and
// dropped).  A map row is 16 bytes per 8 channels: the A operand's core
// matrices are 8 consecutive rows, 128 bytes apart in M.
constexpr int kPitch = kFeatW;
constexpr int kM1 = kH1H * kPitch, kM2 = kQH * kPitch;            // GEMM rows of the two layers
constexpr int kMT1 = (kM1 + 127) / 128, kMT2 = (kM2 + 127) / 128;  // 128-row MMA tiles
// Layer 1 runs with K = 48 (3 MMAs per tile): K-step dy reads feature row
// m + dy kPitch with its 8 channels (the position's own 4 and its right
// neighbour's) as K 0-7 and row m + dy kPitch + 2 as K 8-15, i.e. the second
// K core matrix lies 2 rows (32 bytes) after the first; the 4th position's
// weights are zero.  Layer 2 runs with K = 144: K-step = tap, its channels
// 0-7 and 8-15 in two planes of the layer-1 map.
constexpr int kFeatPos = (kMT1 * 128 + 2 * kPitch + 2 + 7) & ~7;  // feature rows layer 1 reads
constexpr int kH1Pos = ((kMT2 * 128 + 2 * kPitch + 2 > kMT1 * 128 ? kMT2 * 128 + 2 * kPitch + 2 : kMT1 * 128) + 7) & ~7;
constexpr int kTmemCols = 256;              // 16 columns per MMA tile; a power of two
static_assert(kFeatPos >= kFeatN && 16 * kMT1 <= kTmemCols && kMT2 == kMT1 && kMT1 <= kThreads / 32,
              "learned GEMM sizes: one issuing warp per tile of both layers");
constexpr uint32_t kNetIdesc = umma::idesc_bf16<128, 16>();
constexpr int kNetSpin = 1 << 22;           // polls of an MMA completion wait before giving up
constexpr size_t align16z(size_t b) { return (b + 15) & ~(size_t)15; }

// tile (D, 1/D) (+ one ST edge byte per tile entry) of a 32 x TH tile
__host__ __device__ constexpr size_t frame_smem(int Rr, bool st = false, int TH = kTH) {
    return sizeof(int2) * (size_t)(kTW + 2 * Rr) * (TH + 2 * Rr) + (st ? (size_t)(kTW + 2 * Rr) * (TH + 2 * Rr) : 0);
}

// Shared-memory layout of the learned variant (after the tile; all offsets
// 16-byte aligned): work-list counter; mbarrier and TMEM address; b1, b2,
// W3, b3; the B operands of the two layers (16 x 16 BF16 core-matrix blocks
// of 512 bytes per K-step); the feature map; the two planes of the layer-1
// map; q.
struct LearnedSmem {
    size_t cnt, bar, par, w1, w2, feat, h1, q, end;
};
__host__ __device__ constexpr LearnedSmem learned_layout(size_t base) {
    LearnedSmem L{};
    L.cnt = align16z(base);
    L.bar = align16z(L.cnt + 16);  // weights barrier, TMEM address, one MMA barrier per 128-row tile
    L.par = align16z(L.bar + 16 + 8 * kMT1);
    L.w1 = align16z(L.par + 4 * 49);
    L.w2 = align16z(L.w1 + 3 * 512);
    L.feat = align16z(L.w2 + 9 * 512);
    L.h1 = align16z(L.feat + 16 * kFeatPos);
    L.q = align16z(L.h1 + 2 * 16 * kH1Pos);
    L.end = align16z(L.q + 4 * kQN);
    return L;
}
// The q region later holds the work list (one int per tile pixel); features
// and layer 1 later hold the row sums (10 ints per entry) and layer 1 the
// row minima of q.  Two CTAs per SM at most (each holds kTmemCols of the
// SM's 512 TMEM columns): the shared memory of three would exceed the SM's.
static_assert(kQN >= kThreads, "work list");
static_assert(learned_layout(0).q - learned_layout(0).feat >= sizeof(int) * 10 * kRS, "row sums");
static_assert(2 * 16 * kH1Pos >= sizeof(float) * kQH * kTW, "row minima of q");
static_assert(3 * (learned_layout(frame_smem(10)).end + 1024) > 228 * 1024 && 2 * kTmemCols <= 512, "TMEM per SM");
// b1, b2, W3, b3 and the two B operands are one contiguous block, copied
// whole from the image launch_net_image writes
static_assert(learned_layout(0).w1 - learned_layout(0).par == 208 &&
                  learned_layout(0).feat - learned_layout(0).par == (size_t)kNetImageBytes,
              "weights image layout");

// The image: b1, b2, W3, b3 (FP32), then the B operands, element (n, k) of
// K-step s at s 512 + (k / 8) 256 + (n / 8) 128 + (n % 8) 16 + (k % 8) 2
// bytes (16 x 16 BF16 in 8 x 16-byte core matrices).  Layer 1, K-step dy:
// k 0-7 weigh the feature row of position dx = 0 (its channels 0-3) and its
// right neighbour dx = 1 (4-7), k 8-15 position dx = 2 and dx = 3 (zero).
__global__ void k_net_image(const GateView gv, unsigned char* __restrict__ img) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float* par = reinterpret_cast<float*>(img);
    unsigned char* W1s = img + 208;
    unsigned char* W2s = img + 208 + 3 * 512;
    if (i < 52) par[i] = i < 16 ? gv.b1[i] : i < 32 ? gv.b2[i - 16] : i < 48 ? gv.W3[i - 32] : i == 48 ? gv.b3[0] : 0.0f;
    if (i < 16 * 48) {
        // W1g is [16][80] with k = tap * 8 + channel (tap = 3 dy + dx)
        const int nn = i / 48, k = i % 48;
        const int dy = k / 16, kk = k % 16, dx = 2 * (kk / 8) + ((kk % 8) >= 4), ch = kk % 4;
        *reinterpret_cast<__nv_bfloat16*>(W1s + dy * 512 + (kk / 8) * 256 + (nn / 8) * 128 + (nn % 8) * 16 +
                                          (kk % 8) * 2) =
            (dx <= 2 && ch < 3) ? gv.W1g[nn * 80 + (3 * dy + dx) * 8 + ch] : __float2bfloat16(0.0f);
    }
    if (i < 16 * 144) {
        // W2g is [16][144] with k = tap * 16 + channel
        const int nn = i / 144, k = i % 144, tap = k / 16, ch = k % 16;
        *reinterpret_cast<__nv_bfloat16*>(W2s + tap * 512 + (ch / 8) * 256 + (nn / 8) * 128 + (nn % 8) * 16 +
                                          (ch % 8) * 2) = gv.W2g[i];
    }
}


// Tile staging by TMA (variants with a compile-time halo R): one 2-D tensor
// copy brings the raw disparity box into shared memory, then each thread
// converts entries to (D, 1/D).  The box starts at x0 - kTmaXPad (a 16-byte
// boundary: x0 is a multiple of 32) and is kTmaBW wide, so tile column lx
// (image column x0 - R + lx) is box column lx + kTmaXPad - R; rows y0 - R
// .. y0 + TH + R - 1.  Outside the image the box reads zero (code 0).
template <int IN> constexpr int tma_esize() { return IN == SN_IN_F32 ? 4 : 2; }
template <int IN, int R> constexpr int tma_xpad() {  // R rounded up to whole 16-byte units
    return (R + 16 / tma_esize<IN>() - 1) / (16 / tma_esize<IN>()) * (16 / tma_esize<IN>());
}
template <int IN, int R, int TWR> constexpr int tma_bw() {
    return (tma_xpad<IN, R>() - R + TWR + 16 / tma_esize<IN>() - 1) / (16 / tma_esize<IN>()) * (16 / tma_esize<IN>());
}

// Stages the (32 + 2R) x (TH + 2R) tile around (x0, y0) as (D, 1/D) pairs
// (1/D only if with_rcp): one TMA copy of the raw box into `raw` (128-byte
// aligned, tma_bw x (TH + 2R) elements, then an 8-byte mbarrier), then a
// conversion pass.  If `use_tma` is off or `raw` is not 128-byte aligned,
// the tile is loaded with plain loads instead.  Ends with a block barrier.
template <int IN, int R, int TH, int NT>
__device__ __forceinline__ void stage_tile(int2* tile, unsigned char* raw, const CUtensorMap* dmap, bool use_tma,
                                           const char* disp, size_t dp, int x0, int y0, const Geo& g, bool with_rcp) {
    constexpr int TW = kTW + 2 * R, N = TW * (TH + 2 * R), BW = tma_bw<IN, R, TW>();
    constexpr int kRawBytes = BW * (TH + 2 * R) * tma_esize<IN>();
    static_assert(kRawBytes % 16 == 0 && (BW * tma_esize<IN>()) % 16 == 0, "TMA box rows of whole 16-byte units");
    uint64_t* sbar = reinterpret_cast<uint64_t*>(raw + kRawBytes);
    const int tid = threadIdx.y * kTW + threadIdx.x;  // blocks are kTW wide, NT threads
    const bool tma = use_tma && (umma::smem_addr(raw) & 127u) == 0;
    if (tma) {
        if (tid == 0) {
            umma::mbar_init(sbar, 1);
            umma::mbar_expect_tx(sbar, kRawBytes);
            umma::tma_load_2d(raw, dmap, x0 - tma_xpad<IN, R>(), y0 - R, sbar);
        }
        __syncthreads();  // no thread polls the barrier before it is initialised
    }
    const bool ok = tma && umma::mbar_wait(sbar, 0, 1 << 22);
    if (tma && !ok) {
        // Gave up: every thread that did reports it (the polls of different
        // threads may end on either side of a late completion), converts no
        // box entry (its tile entries become invalid codes) and waits once
        // more, again bounded, for the copy still in flight, so that this
        // CTA's shared memory is not handed to another CTA while the copy may
        // still write it.  The frame's outputs are undefined after this.
        atomicOr(g.err, kErrMmaWait);
        umma::mbar_wait(sbar, 0, 1 << 24);
    }
    for (int i = tid; i < N; i += NT) {
        const int ly = i / TW, lx = i - ly * TW;
        const int b = ly * BW + lx + tma_xpad<IN, R>() - R;
        int D = 0;
        if (ok) {
            if constexpr (IN == SN_IN_F32)
                D = code_from_float(reinterpret_cast<const float*>(raw)[b]);
            else if constexpr (IN == SN_IN_F16)
                D = code_from_float(__half2float(reinterpret_cast<const __half*>(raw)[b]));
            else
                D = reinterpret_cast<const unsigned short*>(raw)[b];
        } else if (!tma) {
            D = load_code<IN>(disp, dp, x0 - R + lx, y0 - R + ly, g.W, g.H);
        }
        const float w = !with_rcp ? 0.0f : (D > 0 ? rcp_approx((float)D) : __int_as_float(0x7f800000));
        tile[i] = make_int2(D, __float_as_int(w));
    }
    __syncthreads();
}
constexpr bool frame_tma(int VAR, int R) { return R > 0 && (VAR == 0 || VAR == 2 || VAR == 3 || VAR == 5); }
constexpr size_t align128z(size_t b) { return (b + 127) & ~(size_t)127; }
// Offset and size of the raw box (then its 8-byte mbarrier) after the
// variant's other shared memory.
template <int IN, int VAR, int R>
__host__ __device__ constexpr size_t tma_raw_off() {
    return align128z(VAR == 3 ? learned_layout(frame_smem(R)).end : frame_smem(R, false, frame_th(VAR)));
}
template <int IN, int VAR, int R>
__host__ __device__ constexpr int tma_raw_bytes() {
    return tma_bw<IN, R, kTW + 2 * R>() * (frame_th(VAR) + 2 * R) * tma_esize<IN>();
}

// VAR: 0 fixed window, 1 star table, 2 compile-time M = 8, s = 10 star,
// 3 = 2 with the learned gate, 4 star table with the ST stop, 5 = 2 with the
// ST stop instead of the covered-depth test.  R: halo
// radius at compile time (0 = runtime).
// RD: denoise radius (0 = runtime).
template <int IN, int VAR, int R, int RD>
__global__ void __launch_bounds__(kTW* frame_th(VAR), 1024 / (kTW * frame_th(VAR)))
    k_frame(const Geo g, const __grid_constant__ StarTable T, const char* __restrict__ disp, size_t dp,
            const FrameOut o, const GateView gv, const __grid_constant__ CUtensorMap dmap) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int TH = frame_th(VAR), NT = kTW * TH;
    static_assert(VAR != 3 || TH == kTH, "the learned layout is laid out for kTH-row tiles");
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
        stage_tile<IN, R, TH, NT>(tile, smem + tma_raw_off<IN, VAR, R>(), &dmap, true, disp, dp, x0, y0, g, true);
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

    const int lane = threadIdx.x, row = threadIdx.y;

    if constexpr (VAR != 3) {
        if (inside) {
            PixOut r;
            plain_pixel<VAR, R, RD>(g, T, c, TWR, x, y, r, Est + (c - tile));
            emit(g, o, x, y, r);
        }
    } else {
        // ================= learned gate (tensor cores), then the two paths
        constexpr int TW = kTW + 2 * R;
        constexpr LearnedSmem L = learned_layout(frame_smem(R));  // the launch sizes it the same way
        int* cnt = reinterpret_cast<int*>(smem + L.cnt);
        uint64_t* wbar = reinterpret_cast<uint64_t*>(smem + L.bar);  // weights copy
        uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + L.bar + 8);
        // tile t's MMAs: layer 1 completes phase 0, layer 2 phase 1
        uint64_t* tbar = reinterpret_cast<uint64_t*>(smem + L.bar + 16);
        const float* par = reinterpret_cast<const float*>(smem + L.par);  // b1[16], b2[16], W3[16], b3
        const unsigned char* W1s = smem + L.w1;
        const unsigned char* W2s = smem + L.w2;
        uint4* feat = reinterpret_cast<uint4*>(smem + L.feat);
        uint4* h1p0 = reinterpret_cast<uint4*>(smem + L.h1);                 // layer 1, channels 0-7
        uint4* h1p1 = reinterpret_cast<uint4*>(smem + L.h1 + 16 * kH1Pos);  // channels 8-15
        float* qs = reinterpret_cast<float*>(smem + L.q);
        const int warp = tid >> 5;
        // TMEM for the accumulators; the barriers; the weights (biases, head
        // and both B operands) by one bulk copy, overlapped with the features
        if (warp == 0) umma::tmem_alloc(tslot, kTmemCols);
        if (tid == 0) {
            for (int t = 0; t < kMT1; t++) umma::mbar_init(tbar + t, 1);
            umma::mbar_init(wbar, 1);
            umma::mbar_expect_tx(wbar, kNetImageBytes);
            umma::bulk_g2s(smem + L.par, gv.net, kNetImageBytes, wbar);
        }
        __syncthreads();  // no thread polls a barrier before it is initialised
        // features of the tile + (kQM + 2) region: position i holds its own
        // features (channels 0-3) and its right neighbour's (4-7); rows past
        // the region (read only by dropped GEMM rows) are zero
        for (int i = tid; i < kFeatPos; i += kThreads) {
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (i < kFeatN) {
                const int fx = i % kFeatW - (kQM + 2), fy = i / kFeatW - (kQM + 2);
                const int2* p = tile + (fy + R) * TW + fx + R;
                float f[3], f1[3];
                gate_feature(p[0].x, p[1].x, p[TW].x, f);
                gate_feature(p[1].x, p[2].x, p[TW + 1].x, f1);
                const __nv_bfloat162 a = __floats2bfloat162_rn(f[0], f[1]);
                const __nv_bfloat162 b = __floats2bfloat162_rn(f[2], 0.0f);
                const __nv_bfloat162 a1 = __floats2bfloat162_rn(f1[0], f1[1]);
                const __nv_bfloat162 b1 = __floats2bfloat162_rn(f1[2], 0.0f);
                v.x = *reinterpret_cast<const unsigned*>(&a);
                v.y = *reinterpret_cast<const unsigned*>(&b);
                v.z = *reinterpret_cast<const unsigned*>(&a1);
                v.w = *reinterpret_cast<const unsigned*>(&b1);
            }
            feat[i] = v;
        }
        for (int i = kMT1 * 128 + tid; i < kH1Pos; i += kThreads) h1p0[i] = h1p1[i] = make_uint4(0u, 0u, 0u, 0u);
        if (tid == 0) *cnt = 0;
        bool net_ok = umma::mbar_wait(wbar, 0, kNetSpin);
        umma::fence_proxy_async();
        umma::fence_before();
        net_ok = __syncthreads_and(net_ok);
        umma::fence_after();
        const uint32_t tmem = *tslot;
        const uint32_t tlane = (uint32_t)((warp & 3) * 32) << 16;  // the TMEM lanes this warp may read
        // layer 1: h1 = relu(conv3x3(feat) W1 + b1).  Lane 0 of warp t issues
        // tile t's MMAs and commits them to tbar[t]; the epilogue of a tile
        // starts as soon as its own MMAs are done.  A descriptor's start
        // field counts 16-byte rows, so a tap offset is added to it directly.
        const bool issued1 = net_ok;
        if (net_ok && lane == 0 && warp < kMT1) {
            const uint64_t a0 = umma::desc(umma::smem_addr(feat + 128 * warp), 32, 128);
            const uint64_t b0 = umma::desc(umma::smem_addr(W1s), 256, 128);
#pragma unroll
            for (int dy = 0; dy < 3; dy++)
                umma::mma<kNetIdesc>(tmem + 16 * warp, a0 + dy * kPitch, b0 + 32 * dy, dy > 0);
            umma::commit(tbar + warp);
        }
        bool ok = true;
        if (net_ok) {
            for (int t = warp >> 2; t < kMT1; t += kThreads / 128) {
                ok = __all_sync(0xffffffffu, ok && umma::mbar_wait(tbar + t, 0, kNetSpin));  // warp-uniform
                umma::fence_after();
                if (!ok) break;
                uint32_t r[16];
                umma::ld16(tmem + tlane + 16 * t, r);
                umma::wait_ld();
                unsigned w[8];
#pragma unroll
                for (int c = 0; c < 8; c++) {
                    const __nv_bfloat162 v = __floats2bfloat162_rn(fmaxf(__uint_as_float(r[2 * c]) + par[2 * c], 0.0f),
                                                                   fmaxf(__uint_as_float(r[2 * c + 1]) + par[2 * c + 1], 0.0f));
                    w[c] = *reinterpret_cast<const unsigned*>(&v);
                }
                const int j = 128 * t + (warp & 3) * 32 + lane;
                h1p0[j] = make_uint4(w[0], w[1], w[2], w[3]);
                h1p1[j] = make_uint4(w[4], w[5], w[6], w[7]);
            }
            umma::fence_proxy_async();
            umma::fence_before();
            net_ok = __syncthreads_and(ok);
            umma::fence_after();
        }
        // layer 2 and head: q = sigmoid(relu(conv3x3(h1) W2 + b2) . W3 + b3)
        const bool issued2 = net_ok;
        if (net_ok && lane == 0 && warp < kMT2) {
            const uint64_t a0 = umma::desc(umma::smem_addr(h1p0 + 128 * warp), 16 * kH1Pos, 128);
            const uint64_t b0 = umma::desc(umma::smem_addr(W2s), 256, 128);
#pragma unroll
            for (int tap = 0; tap < 9; tap++)
                umma::mma<kNetIdesc>(tmem + 16 * warp, a0 + (tap / 3) * kPitch + tap % 3, b0 + 32 * tap, tap > 0);
            umma::commit(tbar + warp);
        }
        if (net_ok) {
            for (int t = warp >> 2; t < kMT2; t += kThreads / 128) {
                ok = __all_sync(0xffffffffu, ok && umma::mbar_wait(tbar + t, 1, kNetSpin));  // warp-uniform
                umma::fence_after();
                if (!ok) break;
                uint32_t r[16];
                umma::ld16(tmem + tlane + 16 * t, r);
                umma::wait_ld();
                float part = 0.0f;
#pragma unroll
                for (int c = 0; c < 16; c++) part = fmaf(par[32 + c], fmaxf(__uint_as_float(r[c]) + par[16 + c], 0.0f), part);
                const int j = 128 * t + (warp & 3) * 32 + lane, qy = j / kPitch, qx = j - qy * kPitch;
                if (qy < kQH && qx < kQW) qs[qy * kQW + qx] = 1.0f / (1.0f + __expf(-(part + par[48])));
            }
            net_ok = __syncthreads_and(ok);
        }
        if (!net_ok) {
            // gave up: let what is in flight drain (bounded) before the TMEM is
            // freed; the last committed phase implies the earlier one
            for (int t = 0; t < kMT1; t++) {
                if (issued2)
                    umma::mbar_wait(tbar + t, 1, kNetSpin);
                else if (issued1)
                    umma::mbar_wait(tbar + t, 0, kNetSpin);
            }
            if (!issued1) umma::mbar_wait(wbar, 0, kNetSpin);
        }
        if (!net_ok && tid == 0) atomicOr(g.err, kErrMmaWait);
        umma::fence_before();
        __syncthreads();
        if (warp == 0) {
            umma::fence_after();
            umma::tmem_dealloc(tmem, kTmemCols);
        }
        // gate: min of q over the (2 kQM + 1)^2 neighbourhood >= tau, as a
        // row pass (into the dead layer-1 region) and a column pass
        float* qrow = reinterpret_cast<float*>(smem + L.h1);
        for (int e = tid; e < kQH * kTW; e += kThreads) {
            const float* q0 = qs + (e / kTW) * kQW + e % kTW;
            float m = q0[0];
#pragma unroll
            for (int ox = 1; ox <= 2 * kQM; ox++) m = fminf(m, q0[ox]);
            qrow[e] = m;
        }
        __syncthreads();
        bool gated = false;
        if (inside && Dc > 0) {
            float qmin = qrow[row * kTW + lane];
#pragma unroll
            for (int oy = 1; oy <= 2 * kQM; oy++) qmin = fminf(qmin, qrow[(row + oy) * kTW + lane]);
            gated = net_ok && qmin >= gv.tau;  // no pixel is certified if the network did not finish
        }
        const bool any = __syncthreads_or(gated);
        int* rs = reinterpret_cast<int*>(smem + L.feat);  // features and layer 1 are dead: row sums
        int* list = reinterpret_cast<int*>(smem + L.q);    // q is dead once the gates are known: work list
        if (any) {
            // per row entry (tile rows -kFastR .. kTH - 1 + kFastR), over the
            // valid samples of |u| <= kFastR and |u| <= 2: count, sum u,
            // sum u^2, sum D, sum u D
            for (int e = tid; e < kRS; e += kThreads) {
                const int rr = e / kTW, cx = e % kTW;
                const int2* p = tile + (rr - kFastR + R) * TW + cx + R;
                int a0 = 0, a1 = 0, a2 = 0, d0 = 0, d1 = 0, e0 = 0, e1 = 0, e2 = 0, f0 = 0, f1 = 0;
#pragma unroll
                for (int u = -kFastR; u <= kFastR; u++) {
                    const int D = p[u].x;
                    const int v = D > 0 ? 1 : 0;
                    a0 += v;
                    a1 += u * v;
                    a2 += u * u * v;
                    d0 += D;
                    d1 += u * D;
                    if (u >= -2 && u <= 2) {
                        e0 += v;
                        e1 += u * v;
                        e2 += u * u * v;
                        f0 += D;
                        f1 += u * D;
                    }
                }
                rs[0 * kRS + e] = a0;
                rs[1 * kRS + e] = a1;
                rs[2 * kRS + e] = a2;
                rs[3 * kRS + e] = d0;
                rs[4 * kRS + e] = d1;
                rs[5 * kRS + e] = e0;
                rs[6 * kRS + e] = e1;
                rs[7 * kRS + e] = e2;
                rs[8 * kRS + e] = f0;
                rs[9 * kRS + e] = f1;
            }
        }
        __syncthreads();
        if (inside) {
            if (gated) {
                WinSums w2{}, wa{};
#pragma unroll
                for (int j = 0; j <= 2 * kFastR; j++) {
                    const int v = j - kFastR;
                    const int e = (row + j) * kTW + lane;
                    const int a0 = rs[e], a1 = rs[kRS + e], a2 = rs[2 * kRS + e], d0 = rs[3 * kRS + e],
                              d1 = rs[4 * kRS + e];
                    wa.n += a0;
                    wa.Su += a1;
                    wa.Sv += v * a0;
                    wa.Suu += a2;
                    wa.Suv += v * a1;
                    wa.Svv += v * v * a0;
                    wa.SD += d0;
                    wa.SuD += d1;
                    wa.SvD += v * d0;
                    if (v >= -2 && v <= 2) {
                        const int e0 = rs[5 * kRS + e], e1 = rs[6 * kRS + e], e2 = rs[7 * kRS + e],
                                  f0 = rs[8 * kRS + e], f1 = rs[9 * kRS + e];
                        w2.n += e0;
                        w2.Su += e1;
                        w2.Sv += v * e0;
                        w2.Suu += e2;
                        w2.Suv += v * e1;
                        w2.Svv += v * v * e0;
                        w2.SD += f0;
                        w2.SuD += f1;
                        w2.SvD += v * f0;
                    }
                }
                PixOut r;
                fast_pixel(g, Dc, w2, wa, x, y, r);
                emit(g, o, x, y, r);
            } else if (Dc > 0) {
                list[atomicAdd(cnt, 1)] = tid;
            } else {
                PixOut r;
                pix_zero(r);
                emit(g, o, x, y, r);
            }
        }
        __syncthreads();
        // the uncertified pixels, packed so that whole warps walk star rays
        const int nl = *cnt;
        for (int i = tid; i < nl; i += kThreads) {
            const int p = list[i];
            const int px = p % kTW, py = p / kTW;
            PixOut r;
            plain_pixel<VAR, R, RD>(g, T, tile + (py + R) * TW + px + R, TW, x0 + px, y0 + py, r);
            emit(g, o, x0 + px, y0 + py, r);
        }
    }
}

// Raises a kernel's dynamic shared-memory limit once per device, to the most
// any parameter set of its variant can ask for (so no launch, and no launch
// under stream capture, changes function attributes).  `done` is the
// per-variant record of the devices already set.
template <class Kernel>
cudaError_t smem_limit_once(Kernel k, size_t bytes, std::atomic<unsigned long long>& done) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (done.load() & bit) return cudaSuccess;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) done.fetch_or(bit);
    return e;
}

template <int IN, int VAR, int R, int RD>
cudaError_t launch_in(const Geo& g, const StarTable& t, const char* d, size_t dp, const FrameOut& o,
                      const GateView& gv, cudaStream_t s) {
    constexpr int Rmax = R > 0 ? R : (VAR == 0 ? 15 : (VAR == 4 ? kMaxSteps + 1 : kMaxSteps));
    const int Rr = R > 0 ? R : max(g.r_d, VAR == 0 ? g.r_a : (VAR == 4 ? g.steps + 1 : g.steps));
    constexpr int TH = frame_th(VAR);
    constexpr bool kTma = frame_tma(VAR, R);
    const size_t bytes = kTma ? tma_raw_off<IN, VAR, R>() + tma_raw_bytes<IN, VAR, R>() + 16
                              : (VAR == 3 ? learned_layout(frame_smem(R)).end : frame_smem(Rr, VAR == 4, TH));
    const size_t bytes_max = kTma ? bytes : (VAR == 3 ? learned_layout(frame_smem(R)).end : frame_smem(Rmax, VAR == 4, TH));
    CUtensorMap dmap{};
    if constexpr (kTma) {
        const cudaError_t me = encode_disp_map(&dmap, d, dp, g.W, g.H, IN, tma_bw<IN, R, kTW + 2 * R>(), TH + 2 * R);
        if (me != cudaSuccess) return me;
    }
    const dim3 grid((g.W + kTW - 1) / kTW, (g.H + TH - 1) / TH), block(kTW, TH);
    static std::atomic<unsigned long long> done{0};
    const cudaError_t e = smem_limit_once(k_frame<IN, VAR, R, RD>, bytes_max, done);
    if (e != cudaSuccess) return e;
    k_frame<IN, VAR, R, RD><<<grid, block, bytes, s>>>(g, t, d, dp, o, gv, dmap);
    return cudaGetLastError();
}

template <int VAR, int R, int RD>
cudaError_t launch_var(const Geo& g, const StarTable& t, const void* disp, size_t dp, const FrameOut& o,
                       const GateView& gv, cudaStream_t s) {
    const char* d = static_cast<const char*>(disp);
    switch (g.in_dtype) {
        case SN_IN_F32: return launch_in<SN_IN_F32, VAR, R, RD>(g, t, d, dp, o, gv, s);
        case SN_IN_F16: return launch_in<SN_IN_F16, VAR, R, RD>(g, t, d, dp, o, gv, s);
        default: return launch_in<SN_IN_U16X256, VAR, R, RD>(g, t, d, dp, o, gv, s);
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
    stage_tile<IN, R, kSTH, kTW * kSTH>(tile, raw, &dmap, use_tma, disp, dp, x0, y0, g, true);
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

cudaError_t launch_net_image(const GateView& gv, void* img, cudaStream_t s) {
    k_net_image<<<(16 * 144 + 255) / 256, 256, 0, s>>>(gv, static_cast<unsigned char*>(img));
    return cudaGetLastError();
}

cudaError_t launch_frame(const Geo& g, const StarTable& t, bool star8, const void* disp, size_t dp,
                         const FrameOut& o, const GateView* gv, cudaStream_t s, Marks& mk) {
    cudaError_t e;
    const GateView none{};
    const bool learned = gv && star8 && g.r_d == 2;
    if (learned)
        e = launch_var<3, 10, 2>(g, t, disp, dp, o, *gv, s);
    else if (g.support == SN_SUPPORT_STARFILL_CD && star8)
        e = g.r_d == 2 ? launch_var<2, 10, 2>(g, t, disp, dp, o, none, s)
                       : launch_var<2, 10, 0>(g, t, disp, dp, o, none, s);
    else if (g.support == SN_SUPPORT_STARFILL_CD)
        e = launch_var<1, 0, 0>(g, t, disp, dp, o, none, s);
    else if (g.support == SN_SUPPORT_STARFILL_ST && star8)
        e = g.r_d == 2 ? launch_var<5, 11, 2>(g, t, disp, dp, o, none, s)
                       : launch_var<5, 11, 0>(g, t, disp, dp, o, none, s);
    else if (g.support == SN_SUPPORT_STARFILL_ST)
        e = launch_var<4, 0, 0>(g, t, disp, dp, o, none, s);
    else if (g.r_a == 4 && g.r_d == 2)
        e = launch_var<0, 4, 2>(g, t, disp, dp, o, none, s);  // the 9x9 window with the 5x5 denoise
    else
        e = launch_var<0, 0, 0>(g, t, disp, dp, o, none, s);
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
