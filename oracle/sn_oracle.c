/*
 * sn_oracle.c -- plain FP64 CPU oracle for the stereo surface-normal chain.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * statement of what the CUDA library computes; it is called by the test
 * suite, by the package's smoke check and by the benchmark's CPU-baseline
 * leg, and by nothing else.  It shares no code, header, table or constant
 * with the CUDA library.
 *
 * Method: "Robust and Real-time Surface Normal Estimation from Stereo
 * Disparities using Affine Transformations" (arXiv 2504.15121).
 *
 * Conventions.  u is the column, v the row, both 0-based, pixel centres at
 * integer (u, v).  Disparity is positive, d = u_left - u_right = fx B / z;
 * the paper's own disparity (Sec. III-B, correspondence equation) is the
 * negative of this.  Every discrete decision works on the integer grid
 * D = rint(256 d), so masks and labels are exact.
 *
 * Readings of the paper taken here (the paper is silent or garbled there):
 *   R1  denoising = least-squares plane d = c + g.o over a range-gated
 *       (2 r_d + 1)^2 window; the output is the intercept c (abstract:
 *       "inspired by convolutional operations"; Sec. III-B/III-C).
 *   R2  the affine fit is anchored at the denoised centre value.
 *   R3  invalid samples are dropped from fixed windows.
 *   R4  pixels outside the image are invalid.
 *   R5  normal: the cross product of Sec. III-A, with the sign of the
 *       printed third component corrected, turned to face the camera.
 *   R7  star-fill: direction j at angle 2 pi j / M, step k at offset
 *       (round(k cos), round(k sin)) rounding halves away from zero; the
 *       support is the set union of visited offsets; the stopping pixel and
 *       invalid pixels are excluded; the centre contributes nothing.
 *   R8  covered-depth test in exact integer form.
 *   R9  simple-thresholding stop (ST, Sec. III-D): an edge pixel is one whose
 *       5-point depth Laplacian ((z_l + z_r) + (z_u + z_d)) - 4 z_c, with
 *       z = (256 fx B) / D in metres, exceeds t in magnitude, or one with an
 *       invalid 4-neighbour; evaluated in FP64 in exactly that order with no
 *       fused multiply-add; a ray stops before the first invalid or edge
 *       pixel (excluded, as R7's stopping pixel).
 *   R10 components: 4-connected, edge iff both valid and
 *       2^16 |Dp - Dq| <= K_pair min(Dp, Dq); label = minimum row-major index.
 *   R11 normal valid iff centre valid, >= 3 support pixels, det > 0;
 *       FP64 flag iff 1024 det < alpha gamma.
 *
 * The denoised value on degenerate (rank < 3) windows, or where the fitted
 * intercept is not positive, falls back to the raw centre value: no passage
 * of the paper fixes it, so it is this oracle's reading; the CPU tests pin
 * it with hand-built singular windows (isolated pixel, one row, one column,
 * a diagonal) and a determined fit whose least-squares intercept is
 * negative, each checked against numpy's rank and lstsq.
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_DMAX 131071 /* largest integer disparity code: d < 512 px */

enum { ORC_F32 = 0, ORC_F16 = 1, ORC_U16X256 = 2 };
enum { ORC_FIXED = 0, ORC_STAR_CD = 1, ORC_STAR_ST = 2 };
enum {
    ORC_M_VALID = 1,     /* input disparity valid */
    ORC_M_NORMAL = 2,    /* normal valid */
    ORC_M_FP64 = 4,      /* conditioning flag tripped */
    ORC_M_LEARNED = 8,   /* learned fast path taken */
    ORC_M_DENOISED = 16  /* 3-parameter denoise fit was determined */
};

/* Radius of the full window that a pixel certified by the learned gate fits
 * (the gate certifies the union of the 5x5 patches centred at the lattice
 * points, both coordinates even, within radius - 1 of the pixel). */
#define ORC_LEARNED_RADIUS 6

int orc_learned_radius(void) { return ORC_LEARNED_RADIUS; }

/* Host threads of the OpenMP loops (for timing the oracle single-threaded
 * and on all cores); returns the count in effect. */
int orc_set_threads(int n)
{
    if (n > 0)
        omp_set_num_threads(n);
    return omp_get_max_threads();
}

typedef struct {
    double fx, fy, cx, cy, baseline;
} orc_camera;

typedef struct {
    int r_denoise;
    int r_affine;
    int support;
    int dirs;
    int steps;
    double k_cd;
    double k_pair;
    double k_range;
    double st_t; /* ST threshold on the depth Laplacian, metres */
} orc_params;

/* K = rint(k 2^16): fixed-point form of a relative threshold. */
static int64_t kfix(double k) { return (int64_t)nearbyint(k * 65536.0); }

/* IEEE 754 binary16 -> double, from the format's definition. */
static double half_to_double(uint16_t h)
{
    int s = h >> 15, e = (h >> 10) & 31, m = h & 1023;
    double x;
    if (e == 0)
        x = ldexp((double)m, -24);
    else if (e == 31)
        x = m ? NAN : INFINITY;
    else
        x = ldexp((double)(1024 + m), e - 25);
    return s ? -x : x;
}

/* ---------------------------------------------------------------------
 * Ingest: integer disparity code D = rint(256 d), 0 = invalid.
 * Valid iff d is finite, d > 0 and 1 <= D <= ORC_DMAX (missing
 * disparities, Sec. III-B and Fig. "examples").
 * ------------------------------------------------------------------- */
int orc_ingest(const void *disp, int dtype, size_t pitch_bytes, int W, int H, int32_t *D)
{
    int nvalid = 0;
    for (int v = 0; v < H; v++) {
        const char *row = (const char *)disp + (size_t)v * pitch_bytes;
        for (int u = 0; u < W; u++) {
            int32_t code = 0;
            if (dtype == ORC_U16X256) {
                code = ((const uint16_t *)row)[u];
            } else {
                double d = dtype == ORC_F32 ? (double)((const float *)row)[u]
                                            : half_to_double(((const uint16_t *)row)[u]);
                if (isfinite(d) && d > 0.0) {
                    double r = nearbyint(256.0 * d);
                    if (r >= 1.0 && r <= (double)ORC_DMAX)
                        code = (int32_t)r;
                }
            }
            D[(size_t)v * W + u] = code;
            nvalid += code > 0;
        }
    }
    return nvalid;
}

static int32_t at(const int32_t *D, int W, int H, int u, int v)
{
    if (u < 0 || v < 0 || u >= W || v >= H)
        return 0; /* R4: outside the image is invalid */
    return D[(size_t)v * W + u];
}

/* ---------------------------------------------------------------------
 * Denoise (R1).  Model d(p + o) = c + g_u o_u + g_v o_v over
 * W_d = { o in [-r, r]^2 : p + o valid, 2^16 |D(p+o) - D(p)| <= K D(p) }.
 * Normal equations A x = b with phi = (1, o_u, o_v): A = sum phi phi^T,
 * b = sum phi d.  c by Cramer's rule; all determinants are of integer
 * matrices (exact in FP64).
 * ------------------------------------------------------------------- */
static double det3(double a[3][3])
{
    return a[0][0] * (a[1][1] * a[2][2] - a[1][2] * a[2][1]) -
           a[0][1] * (a[1][0] * a[2][2] - a[1][2] * a[2][0]) +
           a[0][2] * (a[1][0] * a[2][1] - a[1][1] * a[2][0]);
}

static void denoise_impl(const int32_t *D, int W, int H, const orc_params *P, const uint8_t *gate,
                         double *den, uint8_t *fit_ok);

void orc_denoise(const int32_t *D, int W, int H, const orc_params *P, double *den, uint8_t *fit_ok)
{
    denoise_impl(D, W, H, P, NULL, den, fit_ok);
}

/* gate (may be NULL): pixels certified by the learned gate use every valid
 * sample of the window (no range gate). */
static void denoise_impl(const int32_t *D, int W, int H, const orc_params *P, const uint8_t *gate,
                         double *den, uint8_t *fit_ok)
{
    const int r = P->r_denoise;
    const int64_t K = kfix(P->k_range);
#pragma omp parallel for schedule(dynamic, 4)
    for (int v = 0; v < H; v++) {
        for (int u = 0; u < W; u++) {
            size_t idx = (size_t)v * W + u;
            int32_t Dc = D[idx];
            den[idx] = 0.0;
            if (fit_ok)
                fit_ok[idx] = 0;
            if (Dc <= 0)
                continue;
            double A[3][3] = {{0}}, b[3] = {0};
            for (int ov = -r; ov <= r; ov++)
                for (int ou = -r; ou <= r; ou++) {
                    int32_t Di = at(D, W, H, u + ou, v + ov);
                    if (Di <= 0)
                        continue;
                    int64_t diff = (int64_t)Di - Dc;
                    if (diff < 0)
                        diff = -diff;
                    if (!(gate && gate[idx]) && diff * 65536 > K * (int64_t)Dc)
                        continue;
                    double phi[3] = {1.0, (double)ou, (double)ov};
                    double di = Di / 256.0;
                    for (int i = 0; i < 3; i++) {
                        for (int j = 0; j < 3; j++)
                            A[i][j] += phi[i] * phi[j];
                        b[i] += phi[i] * di;
                    }
                }
            double dA = det3(A);
            double c = Dc / 256.0;
            int ok = 0;
            if (dA > 0.0) {
                double Ac[3][3];
                memcpy(Ac, A, sizeof(Ac));
                for (int i = 0; i < 3; i++)
                    Ac[i][0] = b[i];
                double num = det3(Ac);
                if (num > 0.0) {
                    c = num / dA;
                    ok = 1;
                }
            }
            den[idx] = c;
            if (fit_ok)
                fit_ok[idx] = (uint8_t)ok;
        }
    }
}

/* ---------------------------------------------------------------------
 * Star-fill offset table (R7): M directions x s steps, row-major (j, k-1).
 * ------------------------------------------------------------------- */
int orc_star_offsets(int M, int s, int *ou, int *ov)
{
    for (int j = 0; j < M; j++) {
        double th = 2.0 * M_PI * (double)j / (double)M;
        for (int k = 1; k <= s; k++) {
            ou[j * s + k - 1] = (int)round(k * cos(th));
            ov[j * s + k - 1] = (int)round(k * sin(th));
        }
    }
    return M * s;
}

/* Covered-depth stop (Sec. III-D, R8): with depth z = fx B / d the ray stops
 * when z_max - z_min > k z_c; on the integer grid this is
 * (Dmax - Dmin) Dc 2^16 > K Dmin Dmax. */
static int cd_stop(int64_t Dmin, int64_t Dmax, int64_t Dc, int64_t K)
{
    return (Dmax - Dmin) * Dc * 65536 > K * Dmin * Dmax;
}

/* ST edge map (R9): E[v W + u] = 1 for an edge pixel. */
void orc_st_edges(const int32_t *D, int W, int H, const orc_camera *cam, double t, uint8_t *E)
{
    const double F = (256.0 * cam->fx) * cam->baseline;
#pragma omp parallel for schedule(static)
    for (int v = 0; v < H; v++)
        for (int u = 0; u < W; u++) {
            const int32_t Dc = at(D, W, H, u, v), Dl = at(D, W, H, u - 1, v), Dr = at(D, W, H, u + 1, v);
            const int32_t Du = at(D, W, H, u, v - 1), Dd = at(D, W, H, u, v + 1);
            uint8_t e = 1;
            if (Dc > 0 && Dl > 0 && Dr > 0 && Du > 0 && Dd > 0) {
                const double zc = F / (double)Dc, zl = F / (double)Dl, zr = F / (double)Dr;
                const double zu = F / (double)Du, zd = F / (double)Dd;
                const double a = zl + zr;
                const double b = zu + zd;
                const double c = a + b;
                const double L = c - 4.0 * zc;
                e = fabs(L) > t;
            }
            E[(size_t)v * W + u] = e;
        }
}

/* Support of pixel (u, v): incl is a (2R+1)^2 grid of offsets, R the
 * support radius.  Returns the number of included (non-centre) offsets.
 * stedge: the ST edge map (ST support only). */
static int support_of(const int32_t *D, int W, int H, int u, int v, const orc_params *P,
                      const int *tou, const int *tov, uint8_t *incl, int R, const uint8_t *stedge)
{
    int side = 2 * R + 1, n = 0;
    memset(incl, 0, (size_t)side * side);
    int32_t Dc = at(D, W, H, u, v);
    if (Dc <= 0)
        return 0;
    if (P->support == ORC_FIXED) {
        for (int ov = -P->r_affine; ov <= P->r_affine; ov++)
            for (int ou = -P->r_affine; ou <= P->r_affine; ou++) {
                if (ou == 0 && ov == 0)
                    continue;
                if (at(D, W, H, u + ou, v + ov) > 0) {
                    incl[(ov + R) * side + ou + R] = 1;
                    n++;
                }
            }
        return n;
    }
    if (P->support == ORC_STAR_ST) {
        for (int j = 0; j < P->dirs; j++)
            for (int k = 1; k <= P->steps; k++) {
                int ou = tou[j * P->steps + k - 1], ov = tov[j * P->steps + k - 1];
                int uu = u + ou, vv = v + ov;
                if (at(D, W, H, uu, vv) <= 0 || stedge[(size_t)vv * W + uu])
                    break; /* an invalid or edge pixel stops the ray and is excluded */
                uint8_t *cell = &incl[(ov + R) * side + ou + R];
                if (!*cell) {
                    *cell = 1;
                    n++;
                }
            }
        return n;
    }
    const int64_t K = kfix(P->k_cd);
    for (int j = 0; j < P->dirs; j++) {
        int64_t Dmin = Dc, Dmax = Dc;
        for (int k = 1; k <= P->steps; k++) {
            int ou = tou[j * P->steps + k - 1], ov = tov[j * P->steps + k - 1];
            int32_t Di = at(D, W, H, u + ou, v + ov);
            if (Di <= 0)
                break; /* an invalid pixel stops the ray */
            int64_t nmin = Di < Dmin ? Di : Dmin;
            int64_t nmax = Di > Dmax ? Di : Dmax;
            if (cd_stop(nmin, nmax, Dc, K))
                break; /* the stopping pixel is excluded */
            Dmin = nmin;
            Dmax = nmax;
            uint8_t *cell = &incl[(ov + R) * side + ou + R];
            if (!*cell) {
                *cell = 1;
                n++;
            }
        }
    }
    return n;
}

static int support_radius(const orc_params *P)
{
    return P->support == ORC_FIXED ? P->r_affine : P->steps;
}

/* Exposed for tests: the support set of one pixel (stedge: the ST edge
 * map, for the ST support only). */
int orc_support_mask(const int32_t *D, int W, int H, int u, int v, const orc_params *P, const uint8_t *stedge,
                     uint8_t *incl)
{
    int R = support_radius(P);
    int *tou = malloc(sizeof(int) * (P->dirs * P->steps + 1));
    int *tov = malloc(sizeof(int) * (P->dirs * P->steps + 1));
    orc_star_offsets(P->dirs, P->steps, tou, tov);
    int n = support_of(D, W, H, u, v, P, tou, tov, incl, R, stedge);
    free(tou);
    free(tov);
    return n;
}

/* ---------------------------------------------------------------------
 * Affine parameters and normals.
 *
 * Sec. III-B: one row per support pixel, v_i . (a1 - 1, a2) = d_i - d_c;
 * Sec. III-C: a = S d with S = (V^T V)^-1 V^T, V^T V = [[alpha, beta],
 * [beta, gamma]], s_1i = (gamma v_ix - beta v_iy) / det and
 * s_2i = (-beta v_ix + alpha v_iy) / det (eqs. convprep, convprep2).
 * With positive disparity the same sums give the disparity gradient
 * g = (g_u, g_v); the paper's parameters are a1 = 1 - g_u, a2 = -g_v.
 *
 * Sec. III-A: n is orthogonal to a1 v1 - v2 and to a2 v3 - v4 with
 * v1 = X, v2 = X - b e_x, v3 = fy X, v4 = (0, -b fx, 0), so n is their cross
 * product (the printed closed form has the wrong sign on its b term; R5).
 * X is the centre pixel triangulated from the denoised disparity.
 *
 * diag (optional, 8 doubles per pixel): N, alpha, beta, gamma, det, g_u, g_v,
 * support flag bits.
 * ------------------------------------------------------------------- */
static void affine_impl(const int32_t *D, const double *den, int W, int H, const orc_camera *cam,
                        const orc_params *P, const uint8_t *gate, double *nrm, uint8_t *mask, double *diag);

void orc_affine_normals(const int32_t *D, const double *den, int W, int H, const orc_camera *cam,
                        const orc_params *P, double *nrm, uint8_t *mask, double *diag)
{
    affine_impl(D, den, W, H, cam, P, NULL, nrm, mask, diag);
}

/* gate (may be NULL): pixels certified by the learned gate take the fixed
 * (2 ORC_LEARNED_RADIUS + 1)^2 window as their support and get
 * ORC_M_LEARNED. */
static void affine_impl(const int32_t *D, const double *den, int W, int H, const orc_camera *cam,
                        const orc_params *P, const uint8_t *gate, double *nrm, uint8_t *mask, double *diag)
{
    int R = support_radius(P);
    if (gate && R < ORC_LEARNED_RADIUS)
        R = ORC_LEARNED_RADIUS;
    const int side = 2 * R + 1;
    orc_params Pg = *P;
    Pg.support = ORC_FIXED;
    Pg.r_affine = ORC_LEARNED_RADIUS;
    int *tou = malloc(sizeof(int) * (P->dirs * P->steps + 1));
    int *tov = malloc(sizeof(int) * (P->dirs * P->steps + 1));
    orc_star_offsets(P->dirs, P->steps, tou, tov);
    uint8_t *stedge = NULL;
    if (P->support == ORC_STAR_ST) {
        stedge = malloc((size_t)W * H);
        orc_st_edges(D, W, H, cam, P->st_t, stedge);
    }
#pragma omp parallel
    {
        uint8_t *incl = malloc((size_t)side * side);
#pragma omp for schedule(dynamic, 4)
        for (int v = 0; v < H; v++) {
            for (int u = 0; u < W; u++) {
                size_t idx = (size_t)v * W + u;
                double *n = &nrm[3 * idx];
                n[0] = n[1] = n[2] = 0.0;
                uint8_t m = 0;
                if (diag)
                    memset(&diag[8 * idx], 0, 8 * sizeof(double));
                int32_t Dc = D[idx];
                if (Dc <= 0) {
                    mask[idx] = 0;
                    continue;
                }
                m |= ORC_M_VALID;
                const int certified = gate && gate[idx];
                if (certified)
                    m |= ORC_M_LEARNED;
                int N = support_of(D, W, H, u, v, certified ? &Pg : P, tou, tov, incl, R, stedge);
                double alpha = 0, beta = 0, gamma = 0;
                for (int ov = -R; ov <= R; ov++)
                    for (int ou = -R; ou <= R; ou++)
                        if (incl[(ov + R) * side + ou + R]) {
                            alpha += (double)ou * ou;
                            beta += (double)ou * ov;
                            gamma += (double)ov * ov;
                        }
                double det = alpha * gamma - beta * beta;
                if (diag) {
                    double *q = &diag[8 * idx];
                    q[0] = N;
                    q[1] = alpha;
                    q[2] = beta;
                    q[3] = gamma;
                    q[4] = det;
                }
                if (N < 3 || det <= 0.0) {
                    mask[idx] = m;
                    continue;
                }
                if (1024.0 * det < alpha * gamma)
                    m |= ORC_M_FP64;
                double dc = den[idx];
                double gu = 0.0, gv = 0.0;
                for (int ov = -R; ov <= R; ov++)
                    for (int ou = -R; ou <= R; ou++)
                        if (incl[(ov + R) * side + ou + R]) {
                            double s1 = (gamma * ou - beta * ov) / det;
                            double s2 = (-beta * ou + alpha * ov) / det;
                            double di = at(D, W, H, u + ou, v + ov) / 256.0;
                            gu += s1 * (di - dc);
                            gv += s2 * (di - dc);
                        }
                double a1 = 1.0 - gu, a2 = -gv;
                double b = cam->baseline;
                double X[3] = {b * (u - cam->cx) / dc, b * cam->fx / cam->fy * (v - cam->cy) / dc,
                               cam->fx * b / dc};
                double p[3] = {a1 * X[0] - (X[0] - b), a1 * X[1] - X[1], a1 * X[2] - X[2]};
                double q[3] = {a2 * cam->fy * X[0], a2 * cam->fy * X[1] + b * cam->fx,
                               a2 * cam->fy * X[2]};
                double c[3] = {p[1] * q[2] - p[2] * q[1], p[2] * q[0] - p[0] * q[2],
                               p[0] * q[1] - p[1] * q[0]};
                double len = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
                if (!(len > 0.0)) {
                    mask[idx] = m & (uint8_t)~ORC_M_FP64;
                    continue;
                }
                double sgn = (c[0] * X[0] + c[1] * X[1] + c[2] * X[2]) > 0.0 ? -1.0 : 1.0;
                n[0] = sgn * c[0] / len;
                n[1] = sgn * c[1] / len;
                n[2] = sgn * c[2] / len;
                m |= ORC_M_NORMAL;
                mask[idx] = m;
                if (diag) {
                    diag[8 * idx + 5] = gu;
                    diag[8 * idx + 6] = gv;
                }
            }
        }
        free(incl);
    }
    free(tou);
    free(tov);
    free(stedge);
}

/* ---------------------------------------------------------------------
 * Connected surface components (R10): breadth-first flood fill in
 * row-major scan order, so that the first pixel reached in a component
 * is its smallest index.  Invalid pixels get -1.
 * ------------------------------------------------------------------- */
static int edge(const int32_t *D, size_t a, size_t b, int64_t K)
{
    int64_t Da = D[a], Db = D[b];
    if (Da <= 0 || Db <= 0)
        return 0;
    int64_t diff = Da > Db ? Da - Db : Db - Da;
    int64_t mn = Da < Db ? Da : Db;
    return diff * 65536 <= K * mn;
}

int orc_components(const int32_t *D, int W, int H, const orc_params *P, int32_t *labels)
{
    const int64_t K = kfix(P->k_pair);
    size_t n = (size_t)W * H;
    size_t *queue = malloc(sizeof(size_t) * (n ? n : 1));
    int ncomp = 0;
    for (size_t i = 0; i < n; i++)
        labels[i] = -1;
    for (size_t s = 0; s < n; s++) {
        if (D[s] <= 0 || labels[s] != -1)
            continue;
        ncomp++;
        size_t head = 0, tail = 0;
        labels[s] = (int32_t)s;
        queue[tail++] = s;
        while (head < tail) {
            size_t p = queue[head++];
            int u = (int)(p % W), v = (int)(p / W);
            size_t nb[4];
            int cnt = 0;
            if (u > 0)
                nb[cnt++] = p - 1;
            if (u + 1 < W)
                nb[cnt++] = p + 1;
            if (v > 0)
                nb[cnt++] = p - W;
            if (v + 1 < H)
                nb[cnt++] = p + W;
            for (int t = 0; t < cnt; t++) {
                size_t q = nb[t];
                if (labels[q] == -1 && edge(D, p, q, K)) {
                    labels[q] = (int32_t)s;
                    queue[tail++] = q;
                }
            }
        }
    }
    free(queue);
    return ncomp;
}

/* ---------------------------------------------------------------------
 * Oriented point cloud (abstract; Fig. 2): triangulate every valid pixel,
 * X = B (u - cx, fx/fy (v - cy), fx) / d~  (projection of Sec. II).
 * ------------------------------------------------------------------- */
void orc_points(const double *den, const uint8_t *mask, int W, int H, const orc_camera *cam, double *pts)
{
    const double b = cam->baseline;
#pragma omp parallel for schedule(static)
    for (int v = 0; v < H; v++)
        for (int u = 0; u < W; u++) {
            size_t idx = (size_t)v * W + u;
            double *X = &pts[3 * idx];
            if (!(mask[idx] & ORC_M_VALID)) {
                X[0] = X[1] = X[2] = 0.0;
                continue;
            }
            double d = den[idx];
            X[0] = b * (u - cam->cx) / d;
            X[1] = b * cam->fx / cam->fy * (v - cam->cy) / d;
            X[2] = cam->fx * b / d;
        }
}

/* ---------------------------------------------------------------------
 * Whole chain for one frame: ingest, denoise, support + affine + normal,
 * components, points.  Outputs are dense [H][W] (x3 for vectors).
 * mask gets bits VALID | NORMAL | FP64 | DENOISED.
 * ------------------------------------------------------------------- */
int orc_run_frame_gated(const void *disp, int dtype, size_t pitch_bytes, int W, int H, const orc_camera *cam,
                        const orc_params *P, const uint8_t *gate, double *den, double *nrm, double *pts,
                        int32_t *labels, uint8_t *mask);

int orc_run_frame(const void *disp, int dtype, size_t pitch_bytes, int W, int H, const orc_camera *cam,
                  const orc_params *P, double *den, double *nrm, double *pts, int32_t *labels,
                  uint8_t *mask)
{
    return orc_run_frame_gated(disp, dtype, pitch_bytes, W, H, cam, P, NULL, den, nrm, pts, labels, mask);
}

/* The chain with the learned gate's decisions as input (gate may be NULL):
 * certified pixels take the un-gated 5x5 denoise window and the fixed
 * (2 ORC_LEARNED_RADIUS + 1)^2 affine window. */
int orc_run_frame_gated(const void *disp, int dtype, size_t pitch_bytes, int W, int H, const orc_camera *cam,
                        const orc_params *P, const uint8_t *gate, double *den, double *nrm, double *pts,
                        int32_t *labels, uint8_t *mask)
{
    size_t n = (size_t)W * H;
    int32_t *D = malloc(sizeof(int32_t) * (n ? n : 1));
    uint8_t *fit = malloc(n ? n : 1);
    orc_ingest(disp, dtype, pitch_bytes, W, H, D);
    denoise_impl(D, W, H, P, gate, den, fit);
    affine_impl(D, den, W, H, cam, P, gate, nrm, mask, NULL);
    for (size_t i = 0; i < n; i++)
        if (fit[i])
            mask[i] |= ORC_M_DENOISED;
    int ncomp = orc_components(D, W, H, P, labels);
    orc_points(den, mask, W, H, cam, pts);
    free(D);
    free(fit);
    return ncomp;
}
