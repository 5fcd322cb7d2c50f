// Device helpers shared by the kernels: ingest to the integer disparity
// grid, shared-memory tile loads, the exact integer predicates, the
// per-pixel least-squares pieces and the union-find primitives.
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

#include "sn_internal.h"

namespace sn {

constexpr int kFindLimit = 1 << 22;   // > any parent chain of a 16384^2 frame
constexpr int kUnionLimit = 1 << 20;  // retries of one lock-free union

// Reciprocal with at most 1 ulp error (PTX rcp.approx, flushing denormals);
// every input here is a positive normal number (codes 1..131071, positive
// disparities, 256 det with det >= 1).
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// ---------------------------------------------------------------- ingest
// D = rint(256 d) (ties to even) if d is finite, d > 0 and 1 <= D <= 131071,
// else 0 (invalid).  256 d is exact in binary floating point, so the
// comparisons below decide exactly the same as the definition.
__device__ __forceinline__ int code_from_float(float d) {
    const float x = d * 256.0f;
    return (x > 0.5f && x < 131071.5f) ? __float2int_rn(x) : 0;
}

template <int IN>
__device__ __forceinline__ int load_code(const char* __restrict__ base, size_t pitch, int x, int y,
                                         int W, int H) {
    if ((unsigned)x >= (unsigned)W || (unsigned)y >= (unsigned)H) return 0;
    const char* row = base + (size_t)y * pitch;
    if constexpr (IN == SN_IN_F32) {
        return code_from_float(__ldg(reinterpret_cast<const float*>(row) + x));
    } else if constexpr (IN == SN_IN_F16) {
        return code_from_float(__half2float(__ldg(reinterpret_cast<const __half*>(row) + x)));
    } else {
        return __ldg(reinterpret_cast<const unsigned short*>(row) + x);
    }
}

// Loads the integer codes of the rectangle [gx0, gx0 + TWR) x [gy0, gy0 + THR)
// into `tile` (row-major, row length TWR); outside the image: 0.
template <int IN>
__device__ __forceinline__ void load_tile(int* tile, int TWR, int THR, const char* disp, size_t pitch,
                                          int gx0, int gy0, int W, int H) {
    const int n = TWR * THR;
    const int nt = blockDim.x * blockDim.y;
    for (int i = threadIdx.y * blockDim.x + threadIdx.x; i < n; i += nt) {
        const int ly = i / TWR;
        const int lx = i - ly * TWR;
        tile[i] = load_code<IN>(disp, pitch, gx0 + lx, gy0 + ly, W, H);
    }
}

// ---------------------------------------------------------------- predicates
// 2^16 |a - b| <= K min(a, b), both valid
__device__ __forceinline__ bool pair_edge(int a, int b, int K) {
    if (a <= 0 || b <= 0) return false;
    const unsigned diff = (unsigned)abs(a - b);
    const unsigned mn = (unsigned)min(a, b);
    return ((unsigned long long)diff << 16) <= (unsigned long long)(unsigned)K * mn;
}

// The same test from per-pixel thresholds t = floor(K D / 2^16): for
// integers, 2^16 |a - b| <= K m  <=>  |a - b| <= floor(K m / 2^16), and
// floor(K m / 2^16) with m = min(a, b) is min(t_a, t_b) (it is monotone).
__device__ __forceinline__ int pair_thr(int D, int K) {
    return (int)(((unsigned long long)(unsigned)K * (unsigned)D) >> 16);
}
// With t = -1 for an invalid code (pair_thr_v) the test needs no validity
// check: min(t_a, t_b) = -1 < 0 <= |a - b| whenever either code is invalid.
__device__ __forceinline__ int pair_thr_v(int D, int K) { return D > 0 ? pair_thr(D, K) : -1; }
__device__ __forceinline__ bool pair_edge_v(int a, int ta, int b, int tb) { return abs(a - b) <= min(ta, tb); }

// covered-depth stop: (nmax - nmin) Dc 2^16 > K nmin nmax
__device__ __forceinline__ bool cd_stop(int nmin, int nmax, int Dc, int K) {
    const unsigned long long lhs = ((unsigned long long)(unsigned)(nmax - nmin) * (unsigned)Dc) << 16;
    const unsigned long long rhs =
        (unsigned long long)(unsigned)K * ((unsigned long long)(unsigned)nmin * (unsigned)nmax);
    return lhs > rhs;
}

// ---------------------------------------------------------------- denoise
// Least-squares plane c + g . o over the range-gated window around the
// centre `c` of a shared-memory tile with row stride TWR.  The sums are of
// integers (exact); the 3x3 solve for the intercept uses exact int64
// cofactors, and only the final quotient is rounded.  Returns den in pixels.
__device__ __forceinline__ float denoise_at(const int* c, int TWR, int R, int Dc, int K_range,
                                            bool& fit) {
    const int thr = (int)(((unsigned long long)(unsigned)K_range * (unsigned)Dc) >> 16);
    int n = 0, Su = 0, Sv = 0, Suu = 0, Suv = 0, Svv = 0, b0 = 0, b1 = 0, b2 = 0;
    for (int ov = -R; ov <= R; ov++) {
        const int* row = c + ov * TWR;
        for (int ou = -R; ou <= R; ou++) {
            const int Di = row[ou];
            const int dd = Di - Dc;
            if (Di > 0 && abs(dd) <= thr) {
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
    // cofactor expansion of det(A) and of det(A with column 0 := b) along
    // column 0; A = [[n, Su, Sv], [Su, Suu, Suv], [Sv, Suv, Svv]]
    const long long M00 = (long long)Suu * Svv - (long long)Suv * Suv;
    const long long M10 = (long long)Su * Svv - (long long)Sv * Suv;
    const long long M20 = (long long)Su * Suv - (long long)Sv * Suu;
    const long long det = n * M00 - Su * M10 + Sv * M20;
    const long long num = b0 * M00 - b1 * M10 + b2 * M20;  // intercept - Dc, times det
    fit = det > 0 && (long long)Dc * det + num > 0;
    if (!fit) return (float)Dc * (1.0f / 256.0f);
    const float dc = (float)num / (float)det;
    return ((float)Dc + dc) * (1.0f / 256.0f);
}

// ---------------------------------------------------------------- affine
// Pass-1 moments and pass-2 data sums over the support (all integers).
struct AffSums {
    int N, Su, Sv, Suu, Suv, Svv, Bu, Bv;
};

__device__ __forceinline__ void aff_zero(AffSums& s) {
    s.N = s.Su = s.Sv = s.Suu = s.Suv = s.Svv = s.Bu = s.Bv = 0;
}

__device__ __forceinline__ void aff_add(AffSums& s, int ou, int ov, int dd) {
    s.N++;
    s.Su += ou;
    s.Sv += ov;
    s.Suu += ou * ou;
    s.Suv += ou * ov;
    s.Svv += ov * ov;
    s.Bu += ou * dd;
    s.Bv += ov * dd;
}

__device__ __forceinline__ void fixed_support(const int* c, int TWR, int R, int Dc, AffSums& s) {
    aff_zero(s);
    for (int ov = -R; ov <= R; ov++) {
        const int* row = c + ov * TWR;
        for (int ou = -R; ou <= R; ou++) {
            const int Di = row[ou];
            if (Di > 0 && (ou | ov) != 0) aff_add(s, ou, ov, Di - Dc);
        }
    }
}

// Star-fill with the covered-depth stop.  All threads of a warp walk the
// same table entry in lock step (the table index is uniform).
__device__ __forceinline__ void star_support(const int* c, int TWR, int Dc, int K,
                                             const StarTable& T, int dirs, int steps, AffSums& s) {
    aff_zero(s);
    unsigned long long bits = 0ull;
    for (int j = 0; j < dirs; j++) {
        int dmin = Dc, dmax = Dc;
        const int e0 = j * steps;
        for (int k = 0; k < steps; k++) {
            const int e = e0 + k;
            const int cls = T.cls[e];
            if (cls == 0) continue;  // same pixel as the previous step: cannot stop the ray
            const int ou = T.ou[e], ov = T.ov[e];
            const int Di = c[ov * TWR + ou];
            if (Di <= 0) break;
            const int nmin = min(dmin, Di), nmax = max(dmax, Di);
            if (cd_stop(nmin, nmax, Dc, K)) break;
            dmin = nmin;
            dmax = nmax;
            if (cls == 1)
                aff_add(s, ou, ov, Di - Dc);
            else
                bits |= 1ull << T.bit[e];
        }
    }
    for (int b = 0; b < T.nshared; b++) {
        if ((bits >> b) & 1ull) {
            const int ou = T.sou[b], ov = T.sov[b];
            aff_add(s, ou, ov, c[ov * TWR + ou] - Dc);
        }
    }
}

// ST edge test (Sec. III-D, simple thresholding) of a pixel from its own
// and its 4-neighbours' codes: an invalid neighbour makes an edge; otherwise
// the pixel is an edge iff |((z_l + z_r) + (z_u + z_d)) - 4 z_c| > t with
// z = F / D, F = 256 fx B, as evaluated in FP64 in exactly that order.  The
// FP32 evaluation takes z = F rcp(D) with F rounded to FP32 and the 1-ulp
// reciprocal (2^-23 relative at every code, checked by the tests), so each z
// lies within about 2^-22 of F / D relatively; with one rounding per sum
// (4 z_c is exact) the FP32 L differs from the exact value by less than
// 7 2^-24 S, S the sum of the terms' magnitudes, and |L| - t rounds within
// 2^-24 (S + t): together below 2^-21 (S + t).  Outside the band
// 2^-19 (S + t) the FP32 value decides, inside it the FP64 expression does
// (IEEE round-to-nearest operations, no contraction).
__device__ __forceinline__ bool st_edge(const Geo& g, int Dc, int Dl, int Dr, int Du, int Dd) {
    if (Dc <= 0 || Dl <= 0 || Dr <= 0 || Du <= 0 || Dd <= 0) return true;
    const float F = g.st_Ff;
    const float zc = F * rcp_approx((float)Dc), zl = F * rcp_approx((float)Dl), zr = F * rcp_approx((float)Dr);
    const float zu = F * rcp_approx((float)Du), zd = F * rcp_approx((float)Dd);
    const float S = zl + zr + zu + zd + 4.0f * zc;
    const float L = ((zl + zr) + (zu + zd)) - 4.0f * zc;
    const float dev = fabsf(L) - g.st_tf;
    const float band = 0x1p-19f * (S + g.st_tf);
    if (dev > band) return true;
    if (dev < -band) return false;
    const double F64 = g.st_F;
    const double dzc = __ddiv_rn(F64, (double)Dc), dzl = __ddiv_rn(F64, (double)Dl);
    const double dzr = __ddiv_rn(F64, (double)Dr), dzu = __ddiv_rn(F64, (double)Du);
    const double dzd = __ddiv_rn(F64, (double)Dd);
    const double c = __dadd_rn(__dadd_rn(dzl, dzr), __dadd_rn(dzu, dzd));
    return fabs(__dsub_rn(c, __dmul_rn(4.0, dzc))) > g.st_t;
}

// Star-fill with the ST stop on an int tile: a ray stops before the first
// invalid or edge pixel.  e points at the centre's entry of an edge-byte
// array laid out like the tile.
__device__ __forceinline__ void star_support_st(const int* c, const uint8_t* e, int TWR, int Dc,
                                                const StarTable& T, int dirs, int steps, AffSums& s) {
    aff_zero(s);
    unsigned long long bits = 0ull;
    for (int j = 0; j < dirs; j++) {
        const int e0 = j * steps;
        for (int k = 0; k < steps; k++) {
            const int en = e0 + k;
            const int cls = T.cls[en];
            if (cls == 0) continue;  // same pixel as the previous step
            const int ou = T.ou[en], ov = T.ov[en];
            const int Di = c[ov * TWR + ou];
            if (Di <= 0 || e[ov * TWR + ou]) break;
            if (cls == 1)
                aff_add(s, ou, ov, Di - Dc);
            else
                bits |= 1ull << T.bit[en];
        }
    }
    for (int b = 0; b < T.nshared; b++) {
        if ((bits >> b) & 1ull) {
            const int ou = T.sou[b], ov = T.sov[b];
            aff_add(s, ou, ov, c[ov * TWR + ou] - Dc);
        }
    }
}

// int64 -> float through two 32-bit conversions of |x| (the direct 64-bit
// conversion uses the slow FP64 pipe): correctly rounded for |x| < 2^32, at
// most ~1.5 ulp off above that (|x| < 2^55).
__device__ __forceinline__ float i64_to_f32(long long x) {
    const unsigned long long a = x < 0 ? 0ull - (unsigned long long)x : (unsigned long long)x;
    const float f = fmaf((float)(unsigned)(a >> 32), 4294967296.0f, (float)(unsigned)a);
    return x < 0 ? -f : f;
}

// FP64 solve for supports that trip the conditioning flag (rare; FP64 is a
// slow pipe on this GPU, so nothing of it runs on the common path).
__device__ __forceinline__ float3 normal_f64(long long nu_i, long long nv_i, long long cu, long long cv, long long det,
                                             int Dc, double dcd, int x, int y, double fx, double fy, double cx,
                                             double cy) {
    const double dd = ((double)Dc + dcd) * (1.0 / 256.0);
    const double inv = 1.0 / (256.0 * (double)det);
    const double gu = ((double)nu_i - dcd * (double)cu) * inv;
    const double gv = ((double)nv_i - dcd * (double)cv) * inv;
    const double mx = gu;
    const double my = gv * fy / fx;
    const double mz = (dd - gu * ((double)x - cx) - gv * ((double)y - cy)) / fx;
    const double r = 1.0 / sqrt(mx * mx + my * my + mz * mz);
    return make_float3((float)(-mx * r), (float)(-my * r), (float)(-mz * r));
}

// How a kernel reaches normal_f64.  Which form lets the compiler schedule
// the common path best differs by kernel and was measured: out of line with
// the constants by reference and the normal through a pointer to a
// temporary (the plain frame and stage kernels), out of line by value (the
// window kernel, the learned chain's certified pixels), inline (the learned
// chain's star walk).
enum F64Call { kF64ByRef, kF64ByValue, kF64Inline };

static __device__ __noinline__ void normal_f64_ref(long long nu_i, long long nv_i, long long cu, long long cv,
                                                   long long det, int Dc, double dcd, int x, int y, const Geo& g,
                                                   float n[3]) {
    const float3 v = normal_f64(nu_i, nv_i, cu, cv, det, Dc, dcd, x, y, g.dfx, g.dfy, g.dcx, g.dcy);
    n[0] = v.x;
    n[1] = v.y;
    n[2] = v.z;
}

static __device__ __noinline__ float3 normal_f64_val(long long nu_i, long long nv_i, long long cu, long long cv,
                                                     long long det, int Dc, double dcd, int x, int y, double fx,
                                                     double fy, double cx, double cy) {
    return normal_f64(nu_i, nv_i, cu, cv, det, Dc, dcd, x, y, fx, fy, cx, cy);
}

// Solves the 2x2 system of pass 2 and turns (g_u, g_v) into the
// camera-facing unit normal.  The data sums are anchored at the integer
// centre Dc; the anchor shift to the denoised centre (dcf in FP32, and
// anchor_f64() in FP64 when the conditioning flag trips, both in code units)
// enters through the first moments only.  dtil is the denoised disparity in
// pixels.  Returns false if the support does not determine the gradient.
// STAR8: the support lies in the compile-time M = 8, s = 10 star, so
// |Su|, |Sv| <= 222, Suu, Svv <= 1330 and |Suv| <= 560: det <= 1,768,900,
// 1024 det, alpha gamma and the first-moment cofactors fit in 32 bits (the
// data cofactors nu, nv still need 64).
template <bool STAR8 = false, int F64 = kF64ByValue, class AnchorF64>
__device__ __forceinline__ bool solve_normal_dc(const AffSums& s, int Dc, float dcf, AnchorF64 anchor_f64,
                                                float dtil, int x, int y, const Geo& g, float n[3],
                                                bool& fp64) {
    fp64 = false;
    if (s.N < 3) return false;
    long long det, nu_i, nv_i, cu, cv;
    float fdet, fcu, fcv;
    if constexpr (STAR8) {
        const int a = s.Suu, b = s.Suv, gm = s.Svv;
        const int d32 = a * gm - b * b;
        if (d32 <= 0) return false;
        fp64 = 1024 * d32 < a * gm;
        // exact parts of gamma b_u - beta b_v and alpha b_v - beta b_u
        nu_i = (long long)gm * s.Bu - (long long)b * s.Bv;
        nv_i = (long long)a * s.Bv - (long long)b * s.Bu;
        const int cu32 = gm * s.Su - b * s.Sv, cv32 = a * s.Sv - b * s.Su;
        det = d32;
        cu = cu32;
        cv = cv32;
        fdet = (float)d32;  // exact: below 2^24
        fcu = (float)cu32;
        fcv = (float)cv32;
    } else {
        const long long a = s.Suu, b = s.Suv, gm = s.Svv;
        det = a * gm - b * b;
        if (det <= 0) return false;
        fp64 = 1024ll * det < a * gm;
        // exact parts of gamma b_u - beta b_v and alpha b_v - beta b_u
        nu_i = gm * s.Bu - b * s.Bv;
        nv_i = a * s.Bv - b * s.Bu;
        cu = gm * s.Su - b * s.Sv;
        cv = a * s.Sv - b * s.Su;
        fdet = i64_to_f32(det);
        fcu = i64_to_f32(cu);
        fcv = i64_to_f32(cv);
    }
    if (fp64) {
        if constexpr (F64 == kF64ByRef) {
            // through a temporary, so that only the rare path addresses memory
            // (handing n itself over kept the caller's normal in local memory)
            float t[3];
            normal_f64_ref(nu_i, nv_i, cu, cv, det, Dc, anchor_f64(), x, y, g, t);
            n[0] = t[0];
            n[1] = t[1];
            n[2] = t[2];
        } else {
            const float3 v =
                F64 == kF64ByValue
                    ? normal_f64_val(nu_i, nv_i, cu, cv, det, Dc, anchor_f64(), x, y, g.dfx, g.dfy, g.dcx, g.dcy)
                    : normal_f64(nu_i, nv_i, cu, cv, det, Dc, anchor_f64(), x, y, g.dfx, g.dfy, g.dcx, g.dcy);
            n[0] = v.x;
            n[1] = v.y;
            n[2] = v.z;
        }
        return true;
    }
    {
        const float inv = rcp_approx(256.0f * fdet);
        const float gu = fmaf(-dcf, fcu, i64_to_f32(nu_i)) * inv;
        const float gv = fmaf(-dcf, fcv, i64_to_f32(nv_i)) * inv;
        const float mx = gu;
        const float my = gv * g.fy_over_fx;
        const float mz = (dtil - gu * ((float)x - g.cx) - gv * ((float)y - g.cy)) * g.inv_fx;
        const float r = rsqrtf(fmaf(mx, mx, fmaf(my, my, mz * mz)));
        n[0] = -mx * r;
        n[1] = -my * r;
        n[2] = -mz * r;
    }
    return true;
}

// Same, with the anchor taken from a denoised disparity dtil (pixels).
template <bool STAR8 = false>
__device__ __forceinline__ bool solve_normal(const AffSums& s, int Dc, float dtil, int x, int y,
                                             const Geo& g, float n[3], bool& fp64) {
    const float dcf = dtil * 256.0f - (float)Dc;
    return solve_normal_dc<STAR8, kF64ByRef>(
        s, Dc, dcf, [=] { return (double)dtil * 256.0 - (double)Dc; }, dtil, x, y, g, n, fp64);
}

__device__ __forceinline__ short snorm16(float v) {
    return (short)__float2int_rn(32767.0f * fminf(fmaxf(v, -1.0f), 1.0f));
}

// ---------------------------------------------------------------- learned gate
// Gate features of one pixel from the log2 of its own and its right / lower
// neighbours' codes, read from `tab` (FP32 log2 of every code, NaN for code
// 0): the FP32 differences (0 where either code is invalid) and the
// validity.  The training kernels use this function; the inference kernel
// computes the same values from a staged tile.
__device__ __forceinline__ void gate_feature(const float* __restrict__ tab, int Dc, int Dr, int Dd, float f[3]) {
    const float Lc = __ldg(tab + Dc);
    f[0] = (Dc > 0 && Dr > 0) ? __ldg(tab + Dr) - Lc : 0.0f;
    f[1] = (Dc > 0 && Dd > 0) ? __ldg(tab + Dd) - Lc : 0.0f;
    f[2] = Dc > 0 ? 1.0f : 0.0f;
}

// ---------------------------------------------------------------- union-find
// Parent arrays hold row-major pixel indices; parent[i] <= i always, so a
// root is the smallest index of its tree.

// Root of x in a shared-memory parent array, with path halving: every node
// passed is re-pointed at its grandparent, an ancestor, so concurrent unions
// and finds stay correct (a parent only ever decreases towards the root).
// A tile holds at most 4096 entries, so no walk is longer than the loop's
// bound.
__device__ __forceinline__ int find_s_halve(volatile int* L, int x) {
    for (int it = 0; it < 4096; it++) {
        const int p = L[x];
        if (p == x) return x;
        const int gp = L[p];
        if (gp == p) return p;
        L[x] = gp;
        x = gp;
    }
    return x;
}

// lock-free union on a shared-memory parent array: link the larger root
// below the smaller one with atomicMin and retry on interference
__device__ __forceinline__ void union_s(int* L, int a, int b, int* err) {
    for (int it = 0; it < kUnionLimit; it++) {
        a = find_s_halve(L, a);
        b = find_s_halve(L, b);
        if (a == b) return;
        if (a < b) {
            const int t = a;
            a = b;
            b = t;
        }
        const int old = atomicMin(&L[a], b);
        if (old == a) return;
        a = old;
    }
    atomicOr(err, kErrUnionLimit);
}

// Address of label i = v W + u (row v, column u) in a buffer of pitch
// pitch_elems; the row comes from the multiply by ceil(2^64 / W) (Geo::w_rcp).
struct LabelIndex {
    int W;
    unsigned long long w_rcp;
    size_t pitch_elems;
    __device__ __forceinline__ size_t addr(int i) const {
        const unsigned v = W == 1 ? (unsigned)i : (unsigned)__umul64hi((unsigned long long)(unsigned)i, w_rcp);
        return (size_t)(unsigned)i + (size_t)v * (pitch_elems - (size_t)W);
    }
};

// limit: parent steps a walk may take (a context setting, default
// kFindLimit); a walk that runs out sets kErrFindLimit and returns where it is.
__device__ __forceinline__ int find_g(const int* L, const LabelIndex& li, int x, int* err, int limit) {
    for (int it = 0; it < limit; it++) {
        const int p = __ldcg(L + li.addr(x));
        if (p == x) return x;
        x = p;
    }
    atomicOr(err, kErrFindLimit);
    return x;
}

// Root of x with path halving: every node passed is re-pointed at its
// grandparent (an ancestor, so concurrent unions stay correct).
__device__ __forceinline__ int find_halve(int* L, const LabelIndex& li, int x, int* err, int limit) {
    for (int it = 0; it < limit; it++) {
        const int p = __ldcg(L + li.addr(x));
        if (p == x) return x;
        const int gp = __ldcg(L + li.addr(p));
        if (gp == p) return p;
        __stcg(L + li.addr(x), gp);
        x = gp;
    }
    atomicOr(err, kErrFindLimit);
    return x;
}

// Lock-free union: the larger root is linked to the smaller by atomicMin;
// a lost race retries from the value found.
__device__ __forceinline__ void union_g(int* L, const LabelIndex& li, int a, int b, int* err, int limit) {
    for (int it = 0; it < kUnionLimit; it++) {
        a = find_halve(L, li, a, err, limit);
        b = find_halve(L, li, b, err, limit);
        if (a == b) return;
        if (a < b) {
            const int t = a;
            a = b;
            b = t;
        }
        const int old = atomicMin(L + li.addr(a), b);
        if (old == a) return;
        a = old;
    }
    atomicOr(err, kErrUnionLimit);
}

}  // namespace sn
