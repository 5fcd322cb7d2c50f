// Comparison estimators of the paper's experiments (Sec. IV, "Implemented
// algorithms"): Cross, the normal from two tangents to the neighbours' 3-D
// points, and PCA over an n x n window, the eigenvector of the smallest
// eigenvalue of the points' 3x3 covariance in closed form.  They share the
// ingest and the point model of the chain; they are not part of
// sn_run_frame.
#include "sn_device.cuh"

namespace sn {

namespace {

constexpr int kCW = 32, kCH = 8;  // tile: one warp per row

// Offset of pixel q's 3-D point from the centre's, times the positive factor
// D_q D_c / (256 B).  With X = 256 B (u - cx, fx/fy (v - cy), fx) / D, the
// x component of X_q - X_c is 256 B ((u_q - u_c) D_c + (u_c - cx)(D_c - D_q))
// / (D_q D_c): the exact integer difference D_c - D_q carries the
// cancellation between two nearly equal points.  uc = u_c - cx,
// vc = v_c - cy, fxfy = fx / fy.
__device__ __forceinline__ void point_diff(int du, int dv, float uc, float vc, float fxfy, float fx, int Dc, int Dq,
                                           float t[3]) {
    const float dD = (float)(Dc - Dq);
    t[0] = (float)(du * Dc) + uc * dD;
    t[1] = fxfy * ((float)(dv * Dc) + vc * dD);
    t[2] = fx * dD;
}

__device__ __forceinline__ void cross3(const float a[3], const float b[3], float c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

// Unit normal n (camera-facing: n . (uc, fxfy vc, fx) < 0, the centre's
// point up to a positive factor); false when m is zero.
__device__ __forceinline__ bool face_camera(const float m[3], float uc, float vc, float fxfy, float fx, float n[3]) {
    const float l2 = m[0] * m[0] + m[1] * m[1] + m[2] * m[2];
    if (!(l2 > 0.0f)) return false;
    float s = rsqrtf(l2);
    if (m[0] * uc + m[1] * fxfy * vc + m[2] * fx > 0.0f) s = -s;
    n[0] = m[0] * s;
    n[1] = m[1] * s;
    n[2] = m[2] * s;
    return true;
}

__device__ __forceinline__ void write_normal(const Geo& g, char* nrm, size_t np, int x, int y, const float n[3]) {
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
}

// ---------------------------------------------------------------- Cross
template <int IN>
__global__ void __launch_bounds__(kCW* kCH)
    k_cross(const Geo g, const char* __restrict__ disp, size_t dp, char* __restrict__ nrm, size_t np,
            uint8_t* __restrict__ mask, size_t mp) {
    const int x = blockIdx.x * kCW + threadIdx.x, y = blockIdx.y * kCH + threadIdx.y;
    if (x >= g.W || y >= g.H) return;
    const int Dc = load_code<IN>(disp, dp, x, y, g.W, g.H);
    float n[3] = {0.0f, 0.0f, 0.0f};
    uint8_t m = 0;
    if (Dc > 0) {
        m = SN_MASK_VALID;
        const float uc = (float)x - g.cx, vc = (float)y - g.cy, fxfy = g.fx / g.fy;
        const int Dr = load_code<IN>(disp, dp, x + 1, y, g.W, g.H), Dl = load_code<IN>(disp, dp, x - 1, y, g.W, g.H);
        const int Dd = load_code<IN>(disp, dp, x, y + 1, g.W, g.H), Du = load_code<IN>(disp, dp, x, y - 1, g.W, g.H);
        // forward tangent X(q) - X(c), else backward X(c) - X(q): the sign
        // keeps the direction; the positive scale of point_diff drops out
        float tu[3], tv[3];
        const bool hu = Dr > 0 || Dl > 0, hv = Dd > 0 || Du > 0;
        if (Dr > 0) {
            point_diff(1, 0, uc, vc, fxfy, g.fx, Dc, Dr, tu);
        } else {
            point_diff(-1, 0, uc, vc, fxfy, g.fx, Dc, Dl, tu);
            tu[0] = -tu[0], tu[1] = -tu[1], tu[2] = -tu[2];
        }
        if (Dd > 0) {
            point_diff(0, 1, uc, vc, fxfy, g.fx, Dc, Dd, tv);
        } else {
            point_diff(0, -1, uc, vc, fxfy, g.fx, Dc, Du, tv);
            tv[0] = -tv[0], tv[1] = -tv[1], tv[2] = -tv[2];
        }
        if (hu && hv) {
            // unit-scale tangents: the cross product stays in FP32 range on any frame size
            const float su = 1.0f / (fabsf(tu[0]) + fabsf(tu[1]) + fabsf(tu[2]));
            const float sv = 1.0f / (fabsf(tv[0]) + fabsf(tv[1]) + fabsf(tv[2]));
            tu[0] *= su, tu[1] *= su, tu[2] *= su;
            tv[0] *= sv, tv[1] *= sv, tv[2] *= sv;
            float c[3];
            cross3(tu, tv, c);
            if (face_camera(c, uc, vc, fxfy, g.fx, n)) m |= SN_MASK_NORMAL;
        }
    }
    write_normal(g, nrm, np, x, y, n);
    mask[(size_t)y * mp + x] = m;
}

// ---------------------------------------------------------------- PCA
// Eigenvector of the smallest eigenvalue of the symmetric matrix
// C = [[a, b, c], [b, d, e], [c, e, f]] in closed form.  The trigonometric
// solution of the characteristic cubic gives each eigenvalue; with
// r = det((C - q I) / p) / 2 in [-1, 1], the smallest root is well
// conditioned for r < 0 (the two larger eigenvalues are the closer pair) and
// the largest for r >= 0 (the two smaller are, as for the elongated clouds
// that depth noise along the viewing rays makes).  For r < 0 the vector is
// the null vector of C - lambda_min I (the largest cross product of two of
// its rows); for r >= 0 the largest eigenvalue's vector w is found that way
// and the answer is the smaller eigenvector of the 2x2 restriction of C to
// the plane orthogonal to w (atan2).  Either way the error is about
// eps lambda_max / (lambda_mid - lambda_min), as for an FP64 solver's.
__device__ __forceinline__ void smallest_eigvec(float a, float b, float c, float d, float e, float f, float v[3]) {
    const float q = (a + d + f) * (1.0f / 3.0f);
    const float p1 = b * b + c * c + e * e;
    const float a0 = a - q, d0 = d - q, f0 = f - q;
    const float p = sqrtf((a0 * a0 + d0 * d0 + f0 * f0 + 2.0f * p1) * (1.0f / 6.0f));
    float lam = q, r = 0.0f;
    if (p > 0.0f) {
        const float ip = 1.0f / p;
        const float A = a0 * ip, Bb = b * ip, Cc = c * ip, Dd = d0 * ip, Ee = e * ip, Ff = f0 * ip;
        const float det = A * (Dd * Ff - Ee * Ee) - Bb * (Bb * Ff - Ee * Cc) + Cc * (Bb * Ee - Dd * Cc);
        r = fminf(fmaxf(0.5f * det, -1.0f), 1.0f);
        const float phi = acosf(r) * (1.0f / 3.0f);
        lam = q + 2.0f * p * cosf(r >= 0.0f ? phi : phi + 2.0943951023931953f);
    }
    const float r0[3] = {a - lam, b, c}, r1[3] = {b, d - lam, e}, r2[3] = {c, e, f - lam};
    float x0[3], x1[3], x2[3];
    cross3(r0, r1, x0);
    cross3(r0, r2, x1);
    cross3(r1, r2, x2);
    const float n0 = x0[0] * x0[0] + x0[1] * x0[1] + x0[2] * x0[2];
    const float n1 = x1[0] * x1[0] + x1[1] * x1[1] + x1[2] * x1[2];
    const float n2 = x2[0] * x2[0] + x2[1] * x2[1] + x2[2] * x2[2];
    float w[3] = {x0[0], x0[1], x0[2]};
    float nb = n0;
    if (n1 > nb) w[0] = x1[0], w[1] = x1[1], w[2] = x1[2], nb = n1;
    if (n2 > nb) w[0] = x2[0], w[1] = x2[1], w[2] = x2[2], nb = n2;
    if (nb > 0.0f) {
        const float s = rsqrtf(nb);
        w[0] *= s, w[1] *= s, w[2] *= s;
    } else {
        w[0] = 1.0f, w[1] = 0.0f, w[2] = 0.0f;  // isotropic: any axis
    }
    if (r < 0.0f) {
        v[0] = w[0], v[1] = w[1], v[2] = w[2];
        return;
    }
    // orthonormal basis (e1, e2) of the plane orthogonal to w
    const float ax = fabsf(w[0]), ay = fabsf(w[1]), az = fabsf(w[2]);
    const float axis[3] = {(ax <= ay && ax <= az) ? 1.0f : 0.0f, (ay < ax && ay <= az) ? 1.0f : 0.0f,
                           (az < ax && az < ay) ? 1.0f : 0.0f};
    float e1[3], e2[3];
    cross3(w, axis, e1);
    const float s1 = rsqrtf(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
    e1[0] *= s1, e1[1] *= s1, e1[2] *= s1;
    cross3(w, e1, e2);
    const float c1[3] = {a * e1[0] + b * e1[1] + c * e1[2], b * e1[0] + d * e1[1] + e * e1[2],
                         c * e1[0] + e * e1[1] + f * e1[2]};
    const float c2[3] = {a * e2[0] + b * e2[1] + c * e2[2], b * e2[0] + d * e2[1] + e * e2[2],
                         c * e2[0] + e * e2[1] + f * e2[2]};
    const float a2 = e1[0] * c1[0] + e1[1] * c1[1] + e1[2] * c1[2];
    const float b2 = e1[0] * c2[0] + e1[1] * c2[1] + e1[2] * c2[2];
    const float d2 = e2[0] * c2[0] + e2[1] * c2[1] + e2[2] * c2[2];
    float sn, cs;
    sincosf(0.5f * atan2f(2.0f * b2, a2 - d2), &sn, &cs);  // (cs, sn): the larger eigenvalue's vector
    v[0] = cs * e2[0] - sn * e1[0];
    v[1] = cs * e2[1] - sn * e1[1];
    v[2] = cs * e2[2] - sn * e1[2];
}

template <int IN>
__global__ void __launch_bounds__(kCW* kCH)
    k_pca(const Geo g, const char* __restrict__ disp, size_t dp, int r, char* __restrict__ nrm, size_t np,
          uint8_t* __restrict__ mask, size_t mp) {
    extern __shared__ int tile[];
    const int TWR = kCW + 2 * r, THR = kCH + 2 * r;
    const int x0 = blockIdx.x * kCW, y0 = blockIdx.y * kCH;
    load_tile<IN>(tile, TWR, THR, disp, dp, x0 - r, y0 - r, g.W, g.H);
    __syncthreads();
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    if (x >= g.W || y >= g.H) return;
    const int* cp = tile + (threadIdx.y + r) * TWR + threadIdx.x + r;
    const int Dc = cp[0];
    float n[3] = {0.0f, 0.0f, 0.0f};
    uint8_t m = 0;
    if (Dc > 0) {
        m = SN_MASK_VALID;
        const float uc = (float)x - g.cx, vc = (float)y - g.cy, fxfy = g.fx / g.fy;
        int cnt = 0, su = 0, sv = 0, suu = 0, suv = 0, svv = 0;
        float s1[3] = {0.0f, 0.0f, 0.0f}, s2[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        for (int ov = -r; ov <= r; ov++) {
            const int* row = cp + ov * TWR;
            for (int ou = -r; ou <= r; ou++) {
                const int Dq = row[ou];
                if (Dq <= 0) continue;
                cnt++;
                su += ou;
                sv += ov;
                suu += ou * ou;
                suv += ou * ov;
                svv += ov * ov;
                // (X_q - X_c) D_c / (256 B): the factor 1 / D_q of point_diff's
                // scale is applied, the factor common to the window dropped
                float t[3];
                point_diff(ou, ov, uc, vc, fxfy, g.fx, Dc, Dq, t);
                const float w = 1.0f / (float)Dq;
                const float y0v = t[0] * w, y1v = t[1] * w, y2v = t[2] * w;
                s1[0] += y0v;
                s1[1] += y1v;
                s1[2] += y2v;
                s2[0] += y0v * y0v;
                s2[1] += y0v * y1v;
                s2[2] += y0v * y2v;
                s2[3] += y1v * y1v;
                s2[4] += y1v * y2v;
                s2[5] += y2v * y2v;
            }
        }
        const long long A = (long long)cnt * suu - (long long)su * su;
        const long long Cv = (long long)cnt * svv - (long long)sv * sv;
        const long long Bc = (long long)cnt * suv - (long long)su * sv;
        if (cnt >= 3 && A * Cv - Bc * Bc > 0) {
            const float ic = 1.0f / (float)cnt;
            float C[6] = {s2[0] - s1[0] * s1[0] * ic, s2[1] - s1[0] * s1[1] * ic, s2[2] - s1[0] * s1[2] * ic,
                          s2[3] - s1[1] * s1[1] * ic, s2[4] - s1[1] * s1[2] * ic, s2[5] - s1[2] * s1[2] * ic};
            // scale to unit trace (same eigenvectors): the solver's products of
            // entries stay in FP32 range across depth steps at close range
            const float tr = C[0] + C[3] + C[5];
            const float it = tr > 0.0f ? 1.0f / tr : 1.0f;
#pragma unroll
            for (int k = 0; k < 6; k++) C[k] *= it;
            float v[3];
            smallest_eigvec(C[0], C[1], C[2], C[3], C[4], C[5], v);
            if (face_camera(v, uc, vc, fxfy, g.fx, n)) m |= SN_MASK_NORMAL;
        }
    }
    write_normal(g, nrm, np, x, y, n);
    mask[(size_t)y * mp + x] = m;
}

}  // namespace

cudaError_t launch_cross(const Geo& g, const void* disp, size_t dp, void* nrm, size_t np, uint8_t* mask,
                         size_t mp, cudaStream_t s, Marks& mk) {
    const dim3 grid((g.W + kCW - 1) / kCW, (g.H + kCH - 1) / kCH), block(kCW, kCH);
    const char* d = static_cast<const char*>(disp);
    char* n = static_cast<char*>(nrm);
    switch (g.in_dtype) {
        case SN_IN_F32: k_cross<SN_IN_F32><<<grid, block, 0, s>>>(g, d, dp, n, np, mask, mp); break;
        case SN_IN_F16: k_cross<SN_IN_F16><<<grid, block, 0, s>>>(g, d, dp, n, np, mask, mp); break;
        default: k_cross<SN_IN_U16X256><<<grid, block, 0, s>>>(g, d, dp, n, np, mask, mp); break;
    }
    mk.after(s);
    return cudaGetLastError();
}

cudaError_t launch_pca(const Geo& g, const void* disp, size_t dp, int r, void* nrm, size_t np, uint8_t* mask,
                       size_t mp, cudaStream_t s, Marks& mk) {
    const dim3 grid((g.W + kCW - 1) / kCW, (g.H + kCH - 1) / kCH), block(kCW, kCH);
    const size_t smem = sizeof(int) * (size_t)(kCW + 2 * r) * (kCH + 2 * r);
    const char* d = static_cast<const char*>(disp);
    char* n = static_cast<char*>(nrm);
    switch (g.in_dtype) {
        case SN_IN_F32: k_pca<SN_IN_F32><<<grid, block, smem, s>>>(g, d, dp, r, n, np, mask, mp); break;
        case SN_IN_F16: k_pca<SN_IN_F16><<<grid, block, smem, s>>>(g, d, dp, r, n, np, mask, mp); break;
        default: k_pca<SN_IN_U16X256><<<grid, block, smem, s>>>(g, d, dp, r, n, np, mask, mp); break;
    }
    mk.after(s);
    return cudaGetLastError();
}

}  // namespace sn
