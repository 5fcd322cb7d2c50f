"""Pins of the FP64 oracle to facts that do not come from the oracle itself.

Each test names the passage of the paper (or the piece of mathematics) that
fixes the expected value: plane geometry, closed forms of the least-squares
kernels, textbook operators, library routines (numpy.linalg.lstsq,
scipy.ndimage.label) and brute force on tiny inputs written independently in
Python.
"""
import math
import os

import numpy as np
import pytest

import oracle
from oracle import Params, FIXED, STAR_CD, M_VALID, M_NORMAL, M_FP64
from scenes import Camera

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load_rows(name):
    rows = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append([float(x) for x in line.split()])
    return np.array(rows)


def int_plane(W, H, C0, Gu, Gv):
    """Integer disparity codes exactly affine in (u, v): D = C0 + Gu u + Gv v."""
    u = np.arange(W)[None, :]
    v = np.arange(H)[:, None]
    return (C0 + Gu * u + Gv * v).astype(np.int32)


def triangulate(d, cam):
    H, W = d.shape
    u = np.arange(W)[None, :].astype(float)
    v = np.arange(H)[:, None].astype(float)
    B = cam.baseline
    X = B * (u - cam.cx) / d
    Y = B * cam.fx / cam.fy * (v - cam.cy) / d
    Z = cam.fx * B / d
    return np.stack([X, Y, Z + 0 * X], -1)


def geometric_normals(d, cam):
    """Camera-facing unit normals of the surface through the triangulated
    pixels, from the cross product of neighbouring 3-D differences (no
    affine parameters involved)."""
    P = triangulate(d, cam)
    a = P[1:-1, 2:] - P[1:-1, 1:-1]
    b = P[2:, 1:-1] - P[1:-1, 1:-1]
    n = np.cross(a, b)
    n /= np.linalg.norm(n, axis=-1, keepdims=True)
    flip = (n * P[1:-1, 1:-1]).sum(-1) > 0
    n[flip] *= -1
    out = np.zeros_like(P)
    out[1:-1, 1:-1] = n
    return out


CAM = Camera(fx=300.0, fy=280.0, cx=21.5, cy=14.0, baseline=0.12)


# ---------------------------------------------------------------- ingest
def test_ingest_rules():
    d = np.array([[0.0, -1.0, np.nan, np.inf, 1 / 512, 3 / 512, 100.25, 511.99, 512.0, 1e30]],
                 np.float32)
    D = oracle.ingest(d)
    # rint(256 d) with ties to even; valid iff d > 0 finite and 1 <= D <= 131071
    assert D.tolist() == [[0, 0, 0, 0, 0, 2, 25664, 131069, 0, 0]]


def test_ingest_f16_matches_numpy_half():
    rng = np.random.default_rng(0)
    h = (rng.uniform(0, 300, 4096)).astype(np.float16).reshape(64, 64)
    h.flat[:5] = [0, -2, np.inf, np.nan, 6e-8]
    D = oracle.ingest(h)
    ref = np.rint(h.astype(np.float64) * 256.0)
    ok = np.isfinite(ref) & (h.astype(np.float64) > 0) & (ref >= 1) & (ref <= 131071)
    assert np.array_equal(D, np.where(ok, ref, 0).astype(np.int32))


def test_ingest_u16_is_the_code():
    rng = np.random.default_rng(1)
    u = rng.integers(0, 65536, (17, 33)).astype(np.uint16)
    assert np.array_equal(oracle.ingest(u), u.astype(np.int32))


# ---------------------------------------------------------------- denoise
def test_denoise_full_window_is_box_mean():
    # Sec. III-C: with a full symmetric window the LSQ intercept is a plain
    # convolution (the box mean).
    rng = np.random.default_rng(2)
    D = rng.integers(20000, 20100, (40, 50)).astype(np.int32)
    den, ok = oracle.denoise(D, Params(k_range=1.0))
    from numpy.lib.stride_tricks import sliding_window_view
    box = sliding_window_view(D / 256.0, (5, 5)).mean(axis=(-1, -2))
    assert np.allclose(den[2:-2, 2:-2], box, rtol=0, atol=1e-10)
    assert ok[2:-2, 2:-2].all()


def test_denoise_masked_matches_lstsq():
    rng = np.random.default_rng(3)
    H, W = 14, 17
    D = rng.integers(10000, 10700, (H, W)).astype(np.int32)
    D[rng.random((H, W)) < 0.3] = 0
    p = Params(k_range=0.05)
    den, ok = oracle.denoise(D, p)
    K = round(0.05 * 65536)
    for v in range(H):
        for u in range(W):
            Dc = int(D[v, u])
            if Dc == 0:
                assert den[v, u] == 0.0
                continue
            rows, ys = [], []
            for ov in range(-2, 3):
                for ou in range(-2, 3):
                    uu, vv = u + ou, v + ov
                    if not (0 <= uu < W and 0 <= vv < H):
                        continue
                    Di = int(D[vv, uu])
                    if Di == 0 or abs(Di - Dc) * 65536 > K * Dc:
                        continue
                    rows.append([1.0, ou, ov])
                    ys.append(Di / 256.0)
            A = np.array(rows)
            if np.linalg.matrix_rank(A) < 3:
                assert den[v, u] == Dc / 256.0 and ok[v, u] == 0
                continue
            c = np.linalg.lstsq(A, np.array(ys), rcond=None)[0][0]
            assert ok[v, u] == 1
            assert abs(den[v, u] - c) < 1e-9


def test_denoise_gate_is_inclusive():
    # 2^16 |dD| <= K Dc admits equality: with K = rint(0.05 * 2^16) = 3277 and
    # Dc = 65536 a neighbour at Dc + 3277 is inside the gate, Dc + 3278 is not
    D = np.full((5, 5), 65536, np.int32)
    D[2, 3] = 65536 + 3277
    den, _ = oracle.denoise(D, Params(k_range=0.05))
    assert den[2, 2] == (24 * 65536 + 65536 + 3277) / 25 / 256.0
    D[2, 3] = 65536 + 3278
    den, _ = oracle.denoise(D, Params(k_range=0.05))
    # the gated-out sample leaves an asymmetric 24-pixel window; the plane
    # through constant data is still the constant
    assert den[2, 2] == 65536 / 256.0


def _lstsq_intercept(D, u, v, r, K):
    """Intercept of the least-squares plane over the range-gated window,
    by numpy's lstsq on the explicit design matrix, and its rank."""
    H, W = D.shape
    Dc = int(D[v, u])
    rows, ys = [], []
    for ov in range(-r, r + 1):
        for ou in range(-r, r + 1):
            uu, vv = u + ou, v + ov
            if 0 <= uu < W and 0 <= vv < H and D[vv, uu] > 0 and abs(int(D[vv, uu]) - Dc) * 65536 <= K * Dc:
                rows.append([1.0, ou, ov])
                ys.append(D[vv, uu] / 256.0)
    A = np.array(rows, np.float64)
    return np.linalg.lstsq(A, np.array(ys), rcond=None)[0][0], np.linalg.matrix_rank(A)


def test_denoise_fallback_on_singular_windows():
    # Reading: where the 3x3 normal matrix of the gated window is singular
    # (the passing samples lie on one line) the denoised value is the raw
    # centre code / 256 and DENOISED stays clear.  Hand-built cases: an
    # isolated pixel, a one-row strip, a one-column strip, a diagonal, and a
    # centre whose neighbours are all gated out but one.
    D = np.zeros((12, 30), np.int32)
    D[2, 2] = 5000                                   # isolated
    D[6, 4:14] = 7000 + 13 * np.arange(10)           # one row
    D[1:11, 20] = 9000 + 7 * np.arange(10)           # one column
    for k in range(6):
        D[5 + k % 6, 23 + k] = 4000 + 5 * k          # a diagonal
    D[9:12, 1:4] = 30000                             # 3x3 block ...
    D[10, 2] = 20000                                 # ... whose centre gates all but one out
    D[9, 1] = 20100
    den, ok = oracle.denoise(D, Params(k_range=0.05))
    K = round(0.05 * 65536)
    cases = [(2, 2), (6, 8), (6, 13), (4, 20), (10, 20), (7, 25), (10, 2)]
    for v, u in cases:
        c, rank = _lstsq_intercept(D, u, v, 2, K)
        assert rank < 3, (u, v)
        assert den[v, u] == D[v, u] / 256.0 and ok[v, u] == 0, (u, v, den[v, u])


def test_denoise_fallback_on_nonpositive_intercept():
    # Reading: a determined fit whose intercept c is <= 0 also falls back to
    # the raw centre code / 256 with DENOISED clear.  With k_range = 1 the gate
    # admits codes in [1, 2 Dc]; a centre of 100 between a column of 1s and
    # a column of 200s tilts the plane so that numpy's lstsq gives c < 0.
    D = np.zeros((9, 9), np.int32)
    D[4, 4] = 100
    D[2:7, 5] = 1
    D[2:7, 6] = 200
    K = 65536
    c, rank = _lstsq_intercept(D, 4, 4, 2, K)
    assert rank == 3 and c < 0, c
    den, ok = oracle.denoise(D, Params(k_range=1.0))
    assert den[4, 4] == 100 / 256.0 and ok[4, 4] == 0
    # control: the same window with the 200s lowered to 60 has c > 0 and
    # takes the fit
    D[2:7, 6] = 60
    c, rank = _lstsq_intercept(D, 4, 4, 2, K)
    assert rank == 3 and c > 0, c
    den, ok = oracle.denoise(D, Params(k_range=1.0))
    assert ok[4, 4] == 1 and abs(den[4, 4] - c) < 1e-9


def test_denoise_exact_on_plane():
    D = int_plane(30, 20, 20000, 37, -23)
    den, ok = oracle.denoise(D)
    assert np.abs(den - D / 256.0).max() < 1e-9
    assert ok.all()


# ---------------------------------------------------------------- star-fill
def _round_half_away(x):
    return int(math.copysign(math.floor(abs(x) + 0.5), x))


def test_star_offsets_m8():
    ou, ov = oracle.star_offsets(8, 10)
    k = np.arange(1, 11)
    assert np.array_equal(ou[0], k) and np.array_equal(ov[0], 0 * k)      # +u
    assert np.array_equal(ou[2], 0 * k) and np.array_equal(ov[2], k)      # +v
    assert np.array_equal(ou[4], -k) and np.array_equal(ov[4], 0 * k)     # -u
    assert np.array_equal(ou[6], 0 * k) and np.array_equal(ov[6], -k)     # -v
    # diagonals lie exactly on the diagonal, at Euclidean length k rounded
    for j, (sx, sy) in {1: (1, 1), 3: (-1, 1), 5: (-1, -1), 7: (1, -1)}.items():
        expect = np.array([_round_half_away(kk / math.sqrt(2)) for kk in k])
        assert np.array_equal(ou[j], sx * expect) and np.array_equal(ov[j], sy * expect)


def test_star_offsets_m16_geometry():
    ou, ov = oracle.star_offsets(16, 30)
    for j in range(16):
        th = 2 * math.pi * j / 16
        for k in range(1, 31):
            assert abs(ou[j, k - 1] - k * math.cos(th)) <= 0.5
            assert abs(ov[j, k - 1] - k * math.sin(th)) <= 0.5


def _brute_support(D, u, v, M, s, k_cd):
    """Star-fill with the covered-depth stop written in depth space
    (Sec. III-D): z = 1 / D up to a constant; a ray stops at the first
    invalid pixel or when max z - min z along it exceeds k z_centre.
    Returns the set of offsets and whether any decision was within 1e-9 of
    the threshold (such pixels are skipped by the caller)."""
    H, W = D.shape
    Dc = float(D[v, u])
    incl, close = set(), False
    for j in range(M):
        th = 2 * math.pi * j / M
        zmin = zmax = 1.0 / Dc
        for k in range(1, s + 1):
            o = (_round_half_away(k * math.cos(th)), _round_half_away(k * math.sin(th)))
            uu, vv = u + o[0], v + o[1]
            if not (0 <= uu < W and 0 <= vv < H) or D[vv, uu] <= 0:
                break
            z = 1.0 / float(D[vv, uu])
            nmin, nmax = min(zmin, z), max(zmax, z)
            lhs, rhs = nmax - nmin, k_cd / Dc
            if abs(lhs - rhs) < 1e-9 * rhs:
                close = True
            if lhs > rhs:
                break
            zmin, zmax = nmin, nmax
            incl.add(o)
    return incl, close


@pytest.mark.parametrize("M,s", [(8, 10), (16, 6)])
def test_star_support_brute_force(M, s):
    rng = np.random.default_rng(4 + M)
    H, W = 19, 23
    base = rng.integers(3000, 3400, (H, W))
    # blocky jumps so that rays stop inside the image
    blocks = rng.integers(0, 3, (H // 4 + 1, W // 4 + 1)).repeat(4, 0).repeat(4, 1)[:H, :W]
    D = (base * (1.0 + 0.3 * blocks)).astype(np.int32)
    D[rng.random((H, W)) < 0.08] = 0
    # k = 0.1 encodes exactly as K / 2^16 only approximately; use a k that is
    # an exact multiple of 2^-16 so both statements use the same threshold
    k_cd = 6554 / 65536
    p = Params(support=STAR_CD, dirs=M, steps=s, k_cd=k_cd)
    checked = 0
    for v in range(H):
        for u in range(W):
            if D[v, u] <= 0:
                continue
            want, close = _brute_support(D, u, v, M, s, k_cd)
            if close:
                continue
            got = oracle.support_mask(D, u, v, p)
            got_set = {(ou - s, ov - s) for ov, ou in zip(*np.nonzero(got))}
            assert got_set == want, (u, v)
            checked += 1
    assert checked > 300


def test_star_stops_before_invalid_and_edge():
    D = np.full((21, 31), 5000, np.int32)
    D[:, 20:] = 10000          # a depth jump 5 columns right of the centre
    D[10, 10 - 3] = 0          # an invalid pixel 3 steps to the left
    inc = oracle.support_mask(D, 15, 10, Params(support=STAR_CD, dirs=8, steps=10))
    s = 10
    row = inc[s]               # the v = 0 row of the support grid
    # +u ray: steps 1..4 included, step 5 (u = 20) crosses the jump and stops
    assert row[s + 1:s + 5].all() and not row[s + 5:].any()
    inc2 = oracle.support_mask(D, 10, 10, Params(support=STAR_CD, dirs=8, steps=10))
    row2 = inc2[s]
    # -u ray: steps 1, 2 included, step 3 is invalid and stops the ray
    assert row2[s - 2:s].all() and not row2[:s - 2].any()
    assert not inc[s, s] and not inc2[s, s]   # the centre contributes nothing


def test_cd_integer_form_matches_depth_form():
    # single-row images: only the +u ray stays inside (centre at u = 0)
    rng = np.random.default_rng(5)
    k_cd = 6554 / 65536
    p = Params(support=STAR_CD, dirs=8, steps=10, k_cd=k_cd)
    n = 0
    for _ in range(400):
        Dc = int(rng.integers(100, 131071))
        row = [Dc] + [int(max(1, min(131071, Dc * (1 + rng.normal(0, 0.04))))) for _ in range(10)]
        D = np.array([row], np.int32)
        want, close = _brute_support(D, 0, 0, 8, 10, k_cd)
        if close:
            continue
        got = oracle.support_mask(D, 0, 0, p)
        assert int(got.sum()) == len(want)
        n += 1
    assert n > 350


# ---------------------------------------------------------------- affine fit
def test_full_window_moments_closed_form():
    rows = _load_rows("full_window_moments.txt")
    for n, alpha in rows:
        r = int(n) // 2
        assert alpha == n * r * (r + 1) * (2 * r + 1) / 3
        D = np.full((2 * r + 3, 2 * r + 3), 4000, np.int32)
        den, _ = oracle.denoise(D)
        _, _, dg = oracle.affine_normals(D, den, CAM, Params(support=FIXED, r_affine=r), diag=True)
        N, a, b, g = dg[r + 1, r + 1, :4]
        assert (N, a, b, g) == (n * n - 1, alpha, 0.0, alpha)


def test_3x3_kernel_is_prewitt_over_6():
    rows = _load_rows("prewitt_3x3.txt")
    s1, s2 = rows[:3] / 6.0, rows[3:] / 6.0
    p = Params(support=FIXED, r_affine=1)
    base = np.full((3, 3), 8000, np.int32)
    for ov in range(-1, 2):
        for ou in range(-1, 2):
            if ou == 0 and ov == 0:
                continue
            D = base.copy()
            D[1 + ov, 1 + ou] += 256          # +1 px impulse at offset (ou, ov)
            den = np.full((3, 3), 8000 / 256.0)
            _, _, dg = oracle.affine_normals(D, den, CAM, p, diag=True)
            gu, gv = dg[1, 1, 5], dg[1, 1, 6]
            assert abs(gu - s1[1 + ov, 1 + ou]) < 1e-12
            assert abs(gv - s2[1 + ov, 1 + ou]) < 1e-12


def test_masked_affine_matches_lstsq():
    rng = np.random.default_rng(6)
    H, W = 15, 15
    D = rng.integers(9000, 9500, (H, W)).astype(np.int32)
    D[rng.random((H, W)) < 0.45] = 0
    D[7, 7] = 9200
    den = np.where(D > 0, D / 256.0 + 0.123, 0.0)   # arbitrary anchor
    p = Params(support=FIXED, r_affine=4)
    nrm, mask, dg = oracle.affine_normals(D, den, CAM, p, diag=True)
    checked = 0
    for v in range(H):
        for u in range(W):
            if D[v, u] == 0:
                continue
            V, y = [], []
            for ov in range(-4, 5):
                for ou in range(-4, 5):
                    uu, vv = u + ou, v + ov
                    if (ou, ov) == (0, 0) or not (0 <= uu < W and 0 <= vv < H) or D[vv, uu] == 0:
                        continue
                    V.append([ou, ov])
                    y.append(D[vv, uu] / 256.0 - den[v, u])
            V = np.array(V, float)
            if len(V) < 3 or np.linalg.matrix_rank(V) < 2:
                assert not (mask[v, u] & M_NORMAL)
                continue
            g = np.linalg.lstsq(V, np.array(y), rcond=None)[0]
            assert mask[v, u] & M_NORMAL
            assert np.allclose(dg[v, u, 5:7], g, atol=1e-10)
            checked += 1
    assert checked > 100


def test_gradient_noise_variance():
    # Sec. III-C: for a full window g_u = sum s_1i d_i with s_1i = v_ix / alpha,
    # so Var(g_u) = sigma^2 / alpha for iid disparity noise.
    rng = np.random.default_rng(7)
    H = W = 460
    sigma = 0.25
    d = 60.0 + 0.02 * np.arange(W)[None, :] - 0.01 * np.arange(H)[:, None]
    d = d + rng.normal(0, sigma, (H, W))
    D = np.rint(d * 256).astype(np.int32)
    den, _ = oracle.denoise(D)
    p = Params(support=FIXED, r_affine=4)
    _, _, dg = oracle.affine_normals(D, den, CAM, p, diag=True)
    gu = dg[4:-4:9, 4:-4:9, 5].ravel()
    var_pred = (sigma ** 2 + (1 / 256) ** 2 / 12) / 540.0
    var = gu.var(ddof=1)
    se = var_pred * math.sqrt(2.0 / (gu.size - 1))
    assert abs(var - var_pred) < 4 * se
    assert abs(gu.mean() - 0.02) < 4 * math.sqrt(var_pred / gu.size)


# ---------------------------------------------------------------- normals
@pytest.mark.parametrize("support", [FIXED, STAR_CD])
@pytest.mark.parametrize("G", [(37, -23, 20000), (-120, 64, 30000), (0, 0, 12000), (300, 250, 40000)])
def test_normals_exact_on_planes(support, G):
    Gu, Gv, C0 = G
    H, W = 30, 44
    D = int_plane(W, H, C0, Gu, Gv)
    den, _ = oracle.denoise(D)
    nrm, mask = oracle.affine_normals(D, den, CAM, Params(support=support))
    gt = geometric_normals(D / 256.0, CAM)
    inner = (slice(1, -1), slice(1, -1))
    assert (mask[inner] & M_NORMAL).all()
    err = np.linalg.norm(nrm[inner] - gt[inner], axis=-1)
    assert err.max() < 1e-9
    # unit length and facing the camera (n . X < 0)
    assert np.allclose(np.linalg.norm(nrm[inner], axis=-1), 1.0, atol=1e-12)
    X = triangulate(D / 256.0, CAM)
    assert ((nrm * X).sum(-1)[inner] < 0).all()


def test_printed_normal_formula_fails_corrected_passes():
    # Sec. III-A prints n3 = -a1 kh x - a2 kv y + b kh + kh x; the two
    # orthogonality conditions it is derived from give -b kh instead.
    H, W = 30, 44
    D = int_plane(W, H, 30000, -120, 64)
    d = D / 256.0
    den, _ = oracle.denoise(D)
    _, _, dg = oracle.affine_normals(D, den, CAM, Params(support=FIXED), diag=True)
    gt = geometric_normals(d, CAM)
    X = triangulate(d, CAM)
    v, u = 15, 20
    a1, a2 = 1.0 - dg[v, u, 5], -dg[v, u, 6]
    x, y, z = X[v, u]
    kh, kv, b = CAM.fx, CAM.fy, CAM.baseline

    def unit_facing(n):
        n = np.array(n) / np.linalg.norm(n)
        return -n if n @ X[v, u] > 0 else n
    printed = unit_facing([kh * z * (a1 - 1), a2 * kv * z, -a1 * kh * x - a2 * kv * y + b * kh + kh * x])
    fixed = unit_facing([kh * z * (a1 - 1), a2 * kv * z, -a1 * kh * x - a2 * kv * y - b * kh + kh * x])
    ang = lambda a, c: math.degrees(math.acos(min(1.0, abs(a @ c))))
    assert ang(printed, gt[v, u]) > 1.0
    assert ang(fixed, gt[v, u]) < 1e-6


def test_fp64_flag_and_validity():
    # a support that is a line (det = 0) gives no normal
    D = np.zeros((21, 21), np.int32)
    D[10, :] = 6000
    den, _ = oracle.denoise(D)
    _, mask = oracle.affine_normals(D, den, CAM, Params(support=FIXED))
    assert (mask[10] & M_VALID).all() and not (mask[10] & M_NORMAL).any()
    # a support on the digital line (2k, k), k = -7..7, plus the pixel (1, 0)
    # is nearly collinear: alpha = 1121, beta = 560, gamma = 280, det = 280,
    # so 1024 det < alpha gamma and the conditioning flag trips
    D = np.zeros((41, 41), np.int32)
    for k in range(-7, 8):
        D[20 + k, 20 + 2 * k] = 6000 + 10 * k
    D[20, 21] = 6003
    den, _ = oracle.denoise(D)
    _, mask, dg = oracle.affine_normals(D, den, CAM, Params(support=FIXED, r_affine=15), diag=True)
    assert tuple(dg[20, 20, 1:5]) == (1121.0, 560.0, 280.0, 280.0)
    assert mask[20, 20] & M_NORMAL and mask[20, 20] & M_FP64
    # with k = -6..6 instead: alpha = 729, beta = 364, gamma = 182, det = 182,
    # alpha gamma / det = 729 < 1024, so the flag stays clear
    D[20 - 7, 20 - 14] = 0
    D[20 + 7, 20 + 14] = 0
    den, _ = oracle.denoise(D)
    _, mask, dg = oracle.affine_normals(D, den, CAM, Params(support=FIXED, r_affine=15), diag=True)
    assert tuple(dg[20, 20, 1:5]) == (729.0, 364.0, 182.0, 182.0)
    assert mask[20, 20] & M_NORMAL and not mask[20, 20] & M_FP64


def test_minimum_support_size():
    # two non-collinear support pixels determine (a1, a2) exactly, but the
    # normal is only reported from three or more
    D = np.zeros((9, 9), np.int32)
    D[4, 4] = 5000
    D[4, 5] = 5010
    D[5, 4] = 5020
    den, _ = oracle.denoise(D)
    _, mask, dg = oracle.affine_normals(D, den, CAM, Params(support=FIXED, r_affine=1), diag=True)
    assert dg[4, 4, 0] == 2 and dg[4, 4, 4] == 1.0
    assert mask[4, 4] == M_VALID
    D[3, 3] = 4990
    den, _ = oracle.denoise(D)
    _, mask = oracle.affine_normals(D, den, CAM, Params(support=FIXED, r_affine=1))
    assert mask[4, 4] == M_VALID | M_NORMAL


# ---------------------------------------------------------------- components
def _min_index_relabel(lab):
    out = np.full(lab.shape, -1, np.int64)
    flat = lab.ravel()
    for l in np.unique(flat[flat > 0]):
        idx = np.flatnonzero(flat == l)
        out.ravel()[idx] = idx.min()
    return out


def test_components_all_true_predicate_is_scipy_label():
    from scipy import ndimage
    rng = np.random.default_rng(8)
    for trial in range(5):
        H, W = rng.integers(5, 40, 2)
        D = rng.integers(100, 200, (H, W)).astype(np.int32)
        D[rng.random((H, W)) < 0.45] = 0
        lab, n = oracle.components(D, Params(k_pair=1000.0))
        ref, nref = ndimage.label(D > 0, structure=[[0, 1, 0], [1, 1, 1], [0, 1, 0]])
        assert n == nref
        assert np.array_equal(lab, _min_index_relabel(ref))


def _uf_components(D, K):
    H, W = D.shape
    parent = list(range(H * W))

    def find(x):
        while parent[x] != x:
            x = parent[x]
        return x

    def edge(a, b):
        Da, Db = int(D.flat[a]), int(D.flat[b])
        return Da > 0 and Db > 0 and abs(Da - Db) * 65536 <= K * min(Da, Db)
    for v in range(H):
        for u in range(W):
            p = v * W + u
            for q in ([p + 1] if u + 1 < W else []) + ([p + W] if v + 1 < H else []):
                if edge(p, q):
                    ra, rb = find(p), find(q)
                    parent[max(ra, rb)] = min(ra, rb)
    lab = np.array([find(i) if D.flat[i] > 0 else -1 for i in range(H * W)]).reshape(H, W)
    return lab


def test_components_union_find_brute_force():
    rng = np.random.default_rng(9)
    for trial in range(6):
        H, W = rng.integers(3, 30, 2)
        D = rng.choice([0, 1000, 1030, 1049, 1051, 1200, 3000], size=(H, W)).astype(np.int32)
        lab, n = oracle.components(D, Params(k_pair=0.05))
        ref = _uf_components(D, round(0.05 * 65536))
        assert np.array_equal(lab, ref)
        assert n == len(np.unique(ref[ref >= 0]))


# ---------------------------------------------------------------- points
def test_points_reproject():
    rng = np.random.default_rng(10)
    H, W = 12, 16
    den = rng.uniform(5, 80, (H, W))
    mask = (rng.random((H, W)) > 0.2).astype(np.uint8) * M_VALID
    P = oracle.points(den, mask, CAM)
    u = np.arange(W)[None, :]
    v = np.arange(H)[:, None]
    ok = mask > 0
    X, Y, Z = P[..., 0], P[..., 1], P[..., 2]
    with np.errstate(divide="ignore", invalid="ignore"):
        assert np.allclose((CAM.fx * X / Z + CAM.cx)[ok], np.broadcast_to(u, (H, W))[ok])
        assert np.allclose((CAM.fy * Y / Z + CAM.cy)[ok], np.broadcast_to(v, (H, W))[ok])
    with np.errstate(divide="ignore", invalid="ignore"):
        assert np.allclose((CAM.fx * CAM.baseline / Z)[ok], den[ok])
    assert (P[~ok] == 0).all()


# ---------------------------------------------------------------- chain
def test_run_frame_on_noiseless_plane():
    H, W = 40, 50
    D = int_plane(W, H, 25000, 41, 17)
    disp = (D / 256.0).astype(np.float32)
    fr = oracle.run_frame(disp, CAM)
    assert fr.n_components == 1 and (fr.labels == 0).all()
    gt = geometric_normals(D / 256.0, CAM)
    inner = (slice(1, -1), slice(1, -1))
    assert np.linalg.norm(fr.normals[inner] - gt[inner], axis=-1).max() < 1e-9
    assert (fr.mask & 0x17 == 0x13).all()  # valid | normal | denoised, no FP64 flag


def test_gated_chain_is_box_mean_and_full_window():
    # a certified pixel takes every valid sample of the 5x5 window (the box
    # mean, no range gate) and the fixed (2 r + 1)^2 window as its support
    rng = np.random.default_rng(12)
    H, W = 30, 40
    D = (20000 + 40 * np.arange(W)[None, :] - 25 * np.arange(H)[:, None]
         + rng.integers(-300, 300, (H, W))).astype(np.int32)
    D[rng.random((H, W)) < 0.03] = 0
    disp = (D / 256.0).astype(np.float32)
    gate = np.zeros((H, W), bool)
    r = oracle.learned_radius()
    assert 3 <= r <= 9
    gate[r + 2:-r - 2, r + 2:-r - 2] = True
    gate &= D > 0
    fr = oracle.run_frame(disp, CAM, gate=gate)
    fixed = oracle.run_frame(disp, CAM, Params(support=FIXED, r_affine=r, k_range=1.0))
    from numpy.lib.stride_tricks import sliding_window_view
    vals = sliding_window_view(np.pad(D, 2) / 256.0, (5, 5))
    cnt = sliding_window_view(np.pad(D > 0, 2), (5, 5)).sum((-1, -2))
    box = vals.sum((-1, -2)) / np.maximum(cnt, 1)
    g = gate & (fr.mask & 16 > 0)
    assert np.abs(fr.den[g] - fixed.den[g]).max() < 1e-9
    full = g & (cnt == 25)
    assert np.abs(fr.den[full] - box[full]).max() < 1e-9
    assert np.abs(fr.normals[g] - fixed.normals[g]).max() < 1e-12
    assert ((fr.mask[gate] & oracle.M_LEARNED) > 0).all() and not (fr.mask[~gate] & oracle.M_LEARNED).any()
    plain = oracle.run_frame(disp, CAM)
    assert np.array_equal(fr.normals[~gate], plain.normals[~gate])


# ---------------------------------------------------------------- ST stop (Sec. III-D)
def test_st_edges_constant_and_step():
    # constant depth: Laplacian 0 inside; the border and invalid pixels'
    # neighbours are edges (a 4-neighbour is missing)
    D = np.full((12, 16), 6000, np.int32)
    D[5, 7] = 0
    E = oracle.st_edges(D, CAM, 0.01)
    inner = np.zeros_like(E)
    inner[1:-1, 1:-1] = True
    want = ~inner
    for (v, u) in [(5, 7), (4, 7), (6, 7), (5, 6), (5, 8)]:
        want[v, u] = True
    assert np.array_equal(E, want)
    # a depth step between columns 7 and 8: the two columns beside it see
    # |Laplacian| = |z1 - z2|, an edge iff that exceeds t
    D = np.full((12, 16), 6000, np.int32)
    D[:, 8:] = 6200
    F = 256.0 * CAM.fx * CAM.baseline
    dz = F / 6000 - F / 6200
    for t, edge in [(0.5 * dz, True), (1.5 * dz, False)]:
        E = oracle.st_edges(D, CAM, t)
        assert (E[1:-1, 7] == edge).all() and (E[1:-1, 8] == edge).all()
        assert not E[1:-1, 1:7].any() and not E[1:-1, 9:-1].any()


def test_st_laplacian_scale_on_a_paraboloid():
    # z = z0 + a (u^2 + v^2) has 5-point Laplacian 4a everywhere; the codes
    # round z, so thresholds 10 % either side of 4a switch every interior pixel
    H, W, a, z0 = 20, 24, 0.02, 1.5
    F = 256.0 * CAM.fx * CAM.baseline
    u = np.arange(W)[None, :] - W / 2
    v = np.arange(H)[:, None] - H / 2
    D = np.rint(F / (z0 + a * (u * u + v * v))).astype(np.int32)
    assert (D > 0).all() and (D <= 131071).all()
    assert oracle.st_edges(D, CAM, 0.9 * 4 * a)[1:-1, 1:-1].all()
    assert not oracle.st_edges(D, CAM, 1.1 * 4 * a)[1:-1, 1:-1].any()


def test_st_support_brute_force():
    # rays stop before the first invalid or edge pixel, which is excluded
    rng = np.random.default_rng(9)
    H, W = 30, 34
    D = rng.integers(5000, 5100, (H, W)).astype(np.int32)
    D[:, 17:] += 900
    D[rng.random((H, W)) < 0.05] = 0
    t = 0.05
    E = oracle.st_edges(D, CAM, t)
    M, s = 8, 10
    p = Params(support=oracle.STAR_ST, dirs=M, steps=s, st_t=t)
    checked = 0
    for v in range(H):
        for u in range(W):
            if D[v, u] <= 0:
                continue
            want = set()
            for j in range(M):
                th = 2 * math.pi * j / M
                for k in range(1, s + 1):
                    o = (_round_half_away(k * math.cos(th)), _round_half_away(k * math.sin(th)))
                    uu, vv = u + o[0], v + o[1]
                    if not (0 <= uu < W and 0 <= vv < H) or D[vv, uu] <= 0 or E[vv, uu]:
                        break
                    want.add(o)
            got = oracle.support_mask(D, u, v, p, cam=CAM)
            assert {(ou - s, ov - s) for ov, ou in zip(*np.nonzero(got))} == want, (u, v)
            checked += 1
    assert checked > 900
    assert 0.05 < E.mean() < 0.6      # the test exercises both outcomes
