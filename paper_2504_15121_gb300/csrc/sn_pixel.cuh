// Per-pixel device code of the fused frame kernels: the star-fill walks
// (compile-time M = 8 rays and star tables), the fixed window, the exact
// denoise, the solve-and-emit of one pixel, the learned fast path's solve,
// and the tile staging by TMA.  Included by the translation units of the
// plain and the learned frame kernels; everything here has internal
// linkage.
#pragma once

#include <atomic>

#include <cuda.h>  // CUtensorMap
#include <cuda_bf16.h>

#include "sn_device.cuh"
#include "sn_umma.cuh"

namespace sn {

namespace {

constexpr int kTW = kFrameTW, kTH = kFrameTH, kThreads = kTW * kTH;
// Tile height of each variant.  The compile-time M = 8, s = 10 star takes
// 32 x 8 tiles, 4 CTAs of 256 threads per SM (more independent CTAs hide the
// barrier and staging stalls better than 2 CTAs of 512: 130 vs 139 us per
// 2048x1024 frame); the variants with larger halos (star tables up to
// s = 30, the table-driven ST, fixed windows of a runtime radius) keep
// 32 x 16.
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

// Exact decision from the two extreme reciprocals: w is within 1 ulp of 1/D
// and D < 2^17, so rint(1/w) recovers D exactly.
__device__ __forceinline__ bool cd_stop_from_w(float wlo, float whi, int Dc, int K) {
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
// moments of the included prefix 1..n are closed forms.  With TAIL false a
// ray that would need the exact test only raises `unsure` (the caller then
// walks the star again with TAIL true).
template <int SU, int SV, int L, int STRIDE, bool TAIL>
__device__ __forceinline__ void ray8(const int2* __restrict__ c, int Dc, float wc, const Thr& th, AffSums& s,
                                     bool& unsure) {
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
    if constexpr (TAIL) {
        if (n < L && !(whi - wlo > th.hi)) ray8_exact_tail<SU, SV, L, STRIDE>(c, Dc, th.K, &n, &A);
    } else {
        unsure |= n < L && !(whi - wlo > th.hi);
    }
    // T1 = sum t, T2 = sum t^2 over t = 1..n: T2 = T1 (2n + 1) / 3, an exact
    // multiple of 3, divided by multiplying with the inverse of 3 modulo 2^32
    const int T1 = (n * (n + 1)) >> 1;
    const int T2 = (int)((unsigned)(T1 * (2 * n + 1)) * 0xAAAAAAABu);
    // the data sums take A = sum t D itself; the star subtracts Dc times the
    // first moments once, after its last ray
    s.N += n;
    if (SU != 0) {
        s.Su += SU * T1;
        s.Suu += T2;
        s.Bu += SU * A;
    }
    if (SV != 0) {
        s.Sv += SV * T1;
        s.Svv += T2;
        s.Bv += SV * A;
    }
    if (SU != 0 && SV != 0) s.Suv += SU * SV * T2;
}

template <int S, int STRIDE, bool TAIL>
__device__ __forceinline__ bool star8_rays(const int2* c, int Dc, float wc, const Thr& th, AffSums& s) {
    constexpr int LD = diag_len(S);
    bool unsure = false;
    aff_zero(s);
    ray8<1, 0, S, STRIDE, TAIL>(c, Dc, wc, th, s, unsure);
    ray8<1, 1, LD, STRIDE, TAIL>(c, Dc, wc, th, s, unsure);
    ray8<0, 1, S, STRIDE, TAIL>(c, Dc, wc, th, s, unsure);
    ray8<-1, 1, LD, STRIDE, TAIL>(c, Dc, wc, th, s, unsure);
    ray8<-1, 0, S, STRIDE, TAIL>(c, Dc, wc, th, s, unsure);
    ray8<-1, -1, LD, STRIDE, TAIL>(c, Dc, wc, th, s, unsure);
    ray8<0, -1, S, STRIDE, TAIL>(c, Dc, wc, th, s, unsure);
    ray8<1, -1, LD, STRIDE, TAIL>(c, Dc, wc, th, s, unsure);
    // sum u (D - Dc) = sum u D - Dc sum u (|sum u D| < 6 x 55 x 2^17 < 2^31)
    s.Bu -= Dc * s.Su;
    s.Bv -= Dc * s.Sv;
    return unsure;
}

// The star again with the exact tails (a spread inside the rounding band:
// rare), out of line so that the common walk has no call in it.
template <int S, int STRIDE>
__device__ __noinline__ AffSums star8_exact(const int2* c, int Dc, float wc, Thr th) {
    AffSums s;
    star8_rays<S, STRIDE, true>(c, Dc, wc, th, s);
    return s;
}

template <int S, int STRIDE>
__device__ __forceinline__ void star8(const int2* c, int Dc, float wc, const Thr& th, AffSums& s) {
    if (star8_rays<S, STRIDE, false>(c, Dc, wc, th, s)) s = star8_exact<S, STRIDE>(c, Dc, wc, th);
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

// Fixed (2R + 1)^2 window on the packed tile, sample by sample.
__device__ __forceinline__ void fixed_packed(const int2* c, int stride, int R, int Dc, AffSums& s) {
    aff_zero(s);
    for (int ov = -R; ov <= R; ov++) {
        const int2* row = c + ov * stride;
        for (int ou = -R; ou <= R; ou++) {
            const int Di = row[ou].x;
            if (Di > 0 && (ou | ov) != 0) aff_add(s, ou, ov, Di - Dc);
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
        // from population counts of column, row and product classes; the data
        // sums collect D itself (sum D < 25 2^17) and drop Dc once at the end
        unsigned m = 0;
        const int off = lo - Dc;  // D - Dc + lo = D + off
#pragma unroll
        for (int ov = -2; ov <= 2; ov++) {
#pragma unroll
            for (int ou = -2; ou <= 2; ou++) {
                const int D = c[ov * stride + ou].x;
                if ((unsigned)(D + off) <= span) {
                    m |= 1u << ((ov + 2) * 5 + (ou + 2));
                    b0 += D;
                    b1 += ou * D;
                    b2 += ov * D;
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
        b0 -= n * Dc;
        b1 -= Su * Dc;
        b2 -= Sv * Dc;
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
    const float inv = rcp_approx(r.dtil);  // dtil > 0 for every pixel that gets a point
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
// star-fill), two-pass fit, normal, point.  c points at the pixel in the tile;
// T (the star table) is read only by the table-driven variants 1 and 4.
// F64: how the rare FP64 solve is reached (F64Call).
template <int VAR, int R, int RD, int F64 = kF64ByRef>
__device__ __forceinline__ void plain_pixel(const Geo& g, const StarTable* T, const int2* c, int TWR, int x, int y,
                                            PixOut& r, const uint8_t* ec = nullptr) {
    pix_zero(r);
    const int2 cc = c[0];
    const int Dc = cc.x;
    if (Dc <= 0) return;
    r.m = SN_MASK_VALID;
    long long num, det;
    const bool fit = denoise_exact<RD>(c, TWR, g.r_d, Dc, g.K_range, num, det);
    // a 5x5 det is below 2^24 (exact in FP32); the intercept's fraction
    // needs no correctly rounded division (its error is below the outputs'
    // tolerances by orders of magnitude)
    const float dcf =
        fit ? (RD == 2 ? i64_to_f32(num) * rcp_approx((float)(int)det) : i64_to_f32(num) / i64_to_f32(det)) : 0.0f;
    if (fit) r.m |= SN_MASK_DENOISED;
    r.dtil = ((float)Dc + dcf) * (1.0f / 256.0f);
    AffSums s;
    if constexpr (VAR == 4) {
        star_table_st(c, ec, TWR, Dc, *T, g.dirs, g.steps, s);
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
        star_table(c, TWR, Dc, __int_as_float(cc.y), make_thr(g, Dc), *T, g.dirs, g.steps, g.star_pm, s);
    } else {
        // fixed windows of a runtime radius (radii 2..7 with the 5x5 denoise
        // take the convolution-form kernel instead)
        fixed_packed(c, TWR, g.r_a, Dc, s);
    }
    bool fp64;
    if (solve_normal_dc<VAR == 2 || VAR == 5, F64>(
            s, Dc, dcf, [=] { return fit ? (double)num / (double)det : 0.0; }, r.dtil, x, y, g, r.n, fp64))
        r.m |= SN_MASK_NORMAL | (fp64 ? SN_MASK_FP64 : 0);
    pix_points(g, x, y, r);
}

// Sums over the valid samples of a square window around a pixel (offsets
// u, v): moments and the data sums of D, u D, v D.
struct WinSums {
    int n, Su, Sv, Suu, Suv, Svv, SD, SuD, SvD;
};

// The denoise fit over the samples a 5x5 window's sums w2 cover (the same
// integers as denoise_exact<2> over the same samples): intercept
// Dc + num / det; false where det <= 0 or the intercept is not positive.
// The 5x5 window bounds the moments: the cofactors and det fit in 32 bits,
// det below 2^24.
__device__ __forceinline__ bool denoise_from_sums(const WinSums& w2, int Dc, long long& num, long long& det) {
    const int b0 = w2.SD - w2.n * Dc, b1 = w2.SuD - w2.Su * Dc, b2 = w2.SvD - w2.Sv * Dc;
    const int M00 = w2.Suu * w2.Svv - w2.Suv * w2.Suv;
    const int M10 = w2.Su * w2.Svv - w2.Sv * w2.Suv;
    const int M20 = w2.Su * w2.Suv - w2.Sv * w2.Suu;
    const int d = w2.n * M00 - w2.Su * M10 + w2.Sv * M20;
    det = d;
    num = (long long)b0 * M00 - (long long)b1 * M10 + (long long)b2 * M20;
    return d > 0 && (long long)Dc * d + num > 0;
}

// The learned fast path of a certified pixel (its (2 kFastR + 1)^2 window
// shows one surface): the denoise fit takes every valid sample of the 5x5
// window (no range gate) and the affine fit every valid sample of the full
// window except the centre (no star-fill).
__device__ __forceinline__ void fast_pixel(const Geo& g, int Dc, const WinSums& w2, const WinSums& wa, int x, int y,
                                           PixOut& r) {
    pix_zero(r);
    r.m = SN_MASK_VALID | SN_MASK_LEARNED;
    long long num, det;
    const bool fit = denoise_from_sums(w2, Dc, num, det);
    const float dcf = fit ? i64_to_f32(num) * rcp_approx((float)(int)det) : 0.0f;
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

// What stage_tile writes beside each code D: nothing (0), 1/D (FP32
// within 1 ulp; +inf for an invalid code) or D + 2^24 [D > 0] (the code and
// its validity in one word, for window sums).
enum StageY { kStageZero = 0, kStageRcp = 1, kStagePacked = 2 };

// Stages the (32 + 2R) x (TH + 2R) tile around (x0, y0) as (D, y) pairs, y
// as `ymode` (a StageY) says: one TMA copy of the raw box into `raw`
// (128-byte aligned, tma_bw x (TH + 2R) elements, then an 8-byte mbarrier),
// then a conversion pass.  If `use_tma` is off or `raw` is not 128-byte
// aligned, the tile is loaded with plain loads instead.  Ends with a block
// barrier.
template <int IN, int R, int TH, int NT, bool UNROLL = true>
__device__ __forceinline__ void stage_tile(int2* tile, unsigned char* raw, const CUtensorMap* dmap, bool use_tma,
                                           const char* disp, size_t dp, int x0, int y0, const Geo& g, int ymode) {
    constexpr int TW = kTW + 2 * R, N = TW * (TH + 2 * R), BW = tma_bw<IN, R, TW>();
    constexpr int kRawBytes = BW * (TH + 2 * R) * tma_esize<IN>();
    static_assert(kRawBytes % 16 == 0 && (BW * tma_esize<IN>()) % 16 == 0, "TMA box rows of whole 16-byte units");
    uint64_t* sbar = reinterpret_cast<uint64_t*>(raw + kRawBytes);
    const int tid = threadIdx.y * kTW + threadIdx.x;  // blocks are kTW wide, NT threads
    const bool tma = use_tma && (umma::smem_addr(raw) & 127u) == 0;
    // One thread issues the copy and waits for it (sleeping between polls,
    // so that the copy's latency costs the SM no issue slots); the block
    // barrier then publishes the copy and the outcome to every thread.
    bool ok = true;
    if (tma) {
        if (tid == 0) {
            umma::mbar_init(sbar, 1);
            umma::mbar_expect_tx(sbar, kRawBytes);
            umma::tma_load_2d(raw, dmap, x0 - tma_xpad<IN, R>(), y0 - R, sbar);
            ok = umma::mbar_wait_ns(sbar, 0, umma::kWaitNs);
            if (!ok) {
                // Gave up: report it, and wait once more (bounded) for the
                // copy still in flight, so that this CTA's shared memory is
                // not handed to another CTA while the copy may still write
                // it.  No box entry is converted (the tile's codes become
                // invalid); the frame's outputs are undefined after this.
                atomicOr(g.err, kErrMmaWait);
                umma::mbar_wait_ns(sbar, 0, umma::kDrainNs);
            }
        }
        ok = __syncthreads_and(ok);
    }
    ok = tma && ok;
    // UNROLL: the passes unrolled (the conversion loop of a kernel with
    // registers to spare); else a plain strided loop
#pragma unroll(UNROLL ? (N + NT - 1) / NT : 1)
    for (int pass = 0; pass < (N + NT - 1) / NT; pass++) {
        const int i = tid + pass * NT;
        if (N % NT != 0 && i >= N) break;
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
        int y = 0;
        if (ymode == kStageRcp)
            y = __float_as_int(D > 0 ? rcp_approx((float)D) : __int_as_float(0x7f800000));
        else if (ymode == kStagePacked)
            y = D + (D > 0 ? 1 << 24 : 0);
        tile[i] = make_int2(D, y);
    }
    __syncthreads();
}
constexpr size_t align16z(size_t b) { return (b + 15) & ~(size_t)15; }
constexpr size_t align128z(size_t b) { return (b + 127) & ~(size_t)127; }

// Raises a kernel's dynamic shared-memory limit once per device, to the most
// any launch of it can ask for (so no launch, and no launch under stream
// capture, changes function attributes).  `done` is the kernel's record of
// the devices already set.
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

}  // namespace

}  // namespace sn
