"""CUDA path (through the C ABI) against the FP64 oracle, element by element.

Tolerances are in tests/parity.py.  Inputs are seeded: scenes from the
generator (the benchmark workloads at full size included), ragged and tiny
images, adversarial component shapes and constructed ill-conditioned
supports.
"""
import numpy as np
import pytest
import torch

import oracle
from scenes import Camera, make_scene
from parity import compare_frame, compare_normals, oracle_params, run_gpu, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2504_15121_gb300 as P
    return P


CAM = Camera(fx=300.0, fy=280.0, cx=21.5, cy=14.0, baseline=0.12)


def chain(P, disp, cam, **params):
    H, W = disp.shape
    pipe = P.Pipeline(cam, W, H, **params)
    try:
        g = run_gpu(pipe, disp)
        ref = oracle.run_frame(disp, cam, oracle_params(pipe.params))
    finally:
        pipe.close()
    return g, ref


def codes_to_f32(D):
    return (D.astype(np.float64) / 256.0).astype(np.float32)


# ------------------------------------------------------------ scenes
@pytest.mark.parametrize("frame", [0, 1, 2])
@pytest.mark.parametrize("support", [1, 0])
def test_scene_320x240(P, frame, support):
    s = make_scene("planes_320x240", frame=frame)
    g, ref = chain(P, s.disp, s.camera, support=support)
    compare_frame(g, ref)


@pytest.mark.parametrize("name", ["planes_640x480", "mixed_1482x994", "driving_2048x1024"])
def test_scene_full_size(P, name):
    s = make_scene(name, frame=0)
    g, ref = chain(P, s.disp, s.camera)
    mean, mx = compare_frame(g, ref)
    print(f"{name}: normals mean {mean:.2e} max {mx:.2e} deg, {ref.n_components} components")


def test_starfill_s30_d16_full_size(P):
    # the paper's larger adaptive setting (Table perf-disc2, CD s30 d16) on a
    # whole 1482x994 frame: table-driven star with shared diagonal pixels
    s = make_scene("mixed_1482x994", frame=2)
    g, ref = chain(P, s.disp, s.camera, support=1, dirs=16, steps=30)
    mean, mx = compare_frame(g, ref)
    print(f"s30 d16: normals mean {mean:.2e} max {mx:.2e} deg")


@pytest.mark.parametrize("name", ["mixed_1482x994", "driving_2048x1024"])
def test_starfill_st_full_size(P, name):
    # ST s10 d8 t0.1 (Table perf-disc): rays stop at depth-Laplacian edges
    s = make_scene(name, frame=3)
    g, ref = chain(P, s.disp, s.camera, support=2, st_t=0.1)
    mean, mx = compare_frame(g, ref)
    print(f"ST {name}: normals mean {mean:.2e} max {mx:.2e} deg")


def test_st_threshold_at_the_laplacian(P):
    # t set to the FP32-rounded |Laplacian| of chosen pixels, so that the
    # kernel's FP32 band cannot decide there and the exact FP64 expression
    # does; the edge bytes decide the supports, hence the normals and masks
    rng = np.random.default_rng(21)
    H, W = 40, 48
    D = (9000 + 40 * np.arange(W)[None, :] + rng.integers(-60, 60, (H, W))).astype(np.int32)
    F = 256.0 * CAM.fx * CAM.baseline
    z = F / D.astype(np.float64)
    for (v, u) in [(20, 24), (7, 9), (31, 40)]:
        L = ((z[v, u - 1] + z[v, u + 1]) + (z[v - 1, u] + z[v + 1, u])) - 4.0 * z[v, u]
        t = float(np.float32(abs(L)))
        g, ref = chain(P, codes_to_f32(D), CAM, support=2, st_t=t)
        compare_frame(g, ref)
        E = oracle.st_edges(D, CAM, t)
        assert 0 < E[1:-1, 1:-1].mean() < 1


@pytest.mark.parametrize("support", [0, 1, 2])
def test_driving_u16_and_f16_inputs(P, support):
    # 16-bit inputs through the 16-byte aligned TMA boxes of the 9x9 window,
    # the covered-depth and the ST star
    s = make_scene("driving_2048x1024", frame=1)
    for arr, dt in ((s.disp_u16, P.sn.SN_IN_U16X256), (s.disp_f16, P.sn.SN_IN_F16)):
        g, ref = chain(P, arr, s.camera, in_dtype=dt, support=support, st_t=0.1)
        compare_frame(g, ref)


def test_snorm16_output(P):
    s = make_scene("planes_640x480", frame=3)
    H, W = s.disp.shape
    pipe32 = P.Pipeline(s.camera, W, H)
    pipe16 = P.Pipeline(s.camera, W, H, normal_fmt=P.sn.SN_NORMALS_SNORM16X4)
    try:
        g32 = run_gpu(pipe32, s.disp)
        g16 = run_gpu(pipe16, s.disp)
    finally:
        pipe32.close()
        pipe16.close()
    q = g16["normals"].astype(np.int64)
    assert (q[..., 3] == 0).all()
    # the code is rint(32767 n) of the FP32 normal, decided in FP32 as on the GPU
    n32 = torch.from_numpy(g32["normals"].astype(np.float32))
    want = torch.round(32767.0 * n32.clamp(-1, 1)).to(torch.int64).numpy()
    assert np.array_equal(q[..., :3], want)
    ref = oracle.run_frame(s.disp, s.camera)
    ok = (ref.mask & oracle.M_NORMAL) > 0
    assert np.abs(q[..., :3][ok] - 32767.0 * ref.normals[ok]).max() <= 1.0
    assert np.array_equal(g16["mask"], ref.mask)


# ------------------------------------------------------------ tiny and ragged
@pytest.mark.parametrize("H,W", [(1, 1), (1, 7), (7, 1), (5, 7), (17, 33), (40, 65), (9, 129),
                                 (70, 1), (300, 20), (20, 600)])
@pytest.mark.parametrize("support", [1, 0, 2])
def test_ragged_random(P, H, W, support):
    # (70, 1), (300, 20): component tiles in one column, borders only
    # between rows (a width of 1 takes the label addressing's own branch);
    # (20, 600): borders only between columns, shorter than one block of the
    # border merge, whose further blocks along the border exit at once
    rng = np.random.default_rng(H * 1000 + W)
    base = rng.integers(4000, 4400, (H, W))
    blocks = rng.integers(0, 3, (H // 3 + 1, W // 3 + 1)).repeat(3, 0).repeat(3, 1)[:H, :W]
    D = (base * (1 + 0.25 * blocks)).astype(np.int32)
    D[rng.random((H, W)) < 0.2] = 0
    cam = Camera(300.0, 300.0, W / 2, H / 2, 0.1)
    g, ref = chain(P, codes_to_f32(D), cam, support=support)
    compare_frame(g, ref)


@pytest.mark.parametrize("r", [2, 3, 5, 6, 7])
def test_fixed_window_radii_full_size(P, r):
    # every radius of the convolution-form window kernel (r_a 2..7 with the
    # 5x5 denoise): FP32 input on the box-and-curve scene, 16-bit input on
    # the driving scene
    s = make_scene("mixed_1482x994", frame=2)
    g, ref = chain(P, s.disp, s.camera, support=0, r_affine=r)
    compare_frame(g, ref)
    s = make_scene("driving_2048x1024", frame=5)
    g16, ref16 = chain(P, s.disp_u16, s.camera, support=0, r_affine=r, in_dtype=P.sn.SN_IN_U16X256)
    compare_frame(g16, ref16)
    if r in (2, 7):  # FP16 input (the box's other 16-bit element type)
        gh, refh = chain(P, s.disp_f16, s.camera, support=0, r_affine=r, in_dtype=P.sn.SN_IN_F16)
        compare_frame(gh, refh)


@pytest.mark.parametrize("H,W", [(1, 1), (5, 7), (17, 33), (40, 65)])
@pytest.mark.parametrize("r", [2, 7])
def test_ragged_fixed_window_radii(P, H, W, r):
    rng = np.random.default_rng(H * 977 + W + r)
    base = rng.integers(4000, 4400, (H, W))
    blocks = rng.integers(0, 3, (H // 3 + 1, W // 3 + 1)).repeat(3, 0).repeat(3, 1)[:H, :W]
    D = (base * (1 + 0.25 * blocks)).astype(np.int32)
    D[rng.random((H, W)) < 0.2] = 0
    cam = Camera(300.0, 300.0, W / 2, H / 2, 0.1)
    g, ref = chain(P, codes_to_f32(D), cam, support=0, r_affine=r)
    compare_frame(g, ref)


def _extreme_codes(kind, H=72, W=100):
    """Integer codes at the ends of the 17-bit range: 'high' is a tilted
    plane of codes within 200 of the largest (131071) with 5 % invalid
    pixels (window sums at their largest); 'mixed' puts codes 1..4 beside
    codes near the largest in random blocks (the widest spreads)."""
    rng = np.random.default_rng(7 if kind == "high" else 11)
    u = np.arange(W)[None, :]
    v = np.arange(H)[:, None]
    if kind == "high":
        D = 131071 - ((u + 2 * v) % 200)
    else:
        blocks = rng.integers(0, 2, (H // 4 + 1, W // 4 + 1)).repeat(4, 0).repeat(4, 1)[:H, :W]
        D = np.where(blocks > 0, 131071 - rng.integers(0, 64, (H, W)), rng.integers(1, 5, (H, W)))
    D = D.astype(np.int32)
    D[rng.random((H, W)) < 0.05] = 0
    return D


@pytest.mark.parametrize("kind", ["high", "mixed"])
@pytest.mark.parametrize("params", [dict(support=1), dict(support=2), dict(support=0, r_affine=2),
                                    dict(support=0, r_affine=4), dict(support=0, r_affine=5),
                                    dict(support=0, r_affine=6), dict(support=0, r_affine=7)])
def test_extreme_codes(P, kind, params):
    # the packed window sums and the star walk's integer sums at the largest
    # codes, and the covered-depth and range gates across the widest spreads
    D = _extreme_codes(kind)
    H, W = D.shape
    cam = Camera(500.0, 500.0, W / 2, H / 2, 0.12)
    g, ref = chain(P, codes_to_f32(D), cam, **params)
    compare_frame(g, ref)


def test_reciprocal_of_every_code_within_one_ulp(P):
    # the covered-depth band and the ST edge band both assume that the
    # kernels' FP32 1/D lies within 2^-23 of 1/D relatively, for every code
    r = P.sn.sn_rcp_table()
    assert np.isposinf(r[0])
    D = np.arange(1, r.size, dtype=np.float64)
    rel = np.abs(r[1:].astype(np.float64) * D - 1.0)  # r D is exact in FP64
    ulps = np.abs(r[1:].astype(np.float64) - 1.0 / D) / np.spacing(r[1:]).astype(np.float64)
    print(f"rcp over codes 1..131071: max relative error {rel.max():.3e} ({np.log2(rel.max()):.2f} in log2), "
          f"max {ulps.max():.3f} ulp")
    assert rel.max() <= 2.0 ** -23


def test_covered_depth_at_the_threshold(P):
    # k_cd = 0.1 (K = 6554): with Dc = Dmin = 29491 the stop test
    # (Dmax - Dmin) Dc 2^16 > K Dmin Dmax holds from Dmax = 32769 on and is an
    # equality at Dmax = 32768, so rays meeting such samples sit exactly on the
    # threshold, inside every FP32 rounding band: the exact test must decide
    K = int(round(0.1 * 65536))
    assert (32768 - 29491) * 29491 * 65536 == K * 29491 * 32768
    assert (32769 - 29491) * 29491 * 65536 > K * 29491 * 32769
    rng = np.random.default_rng(17)
    H, W = 64, 96
    D = np.full((H, W), 29491, np.int32)
    sites = rng.random((H, W))
    D[sites < 0.03] = 32768
    D[(sites >= 0.03) & (sites < 0.06)] = 32769
    D[(sites >= 0.06) & (sites < 0.08)] = 0
    cam = Camera(400.0, 400.0, W / 2, H / 2, 0.1)
    for params in (dict(support=1), dict(support=1, dirs=16, steps=12)):
        g, ref = chain(P, codes_to_f32(D), cam, **params)
        compare_frame(g, ref)


def _fallback_frame(rng, H=96, W=160):
    """Integer codes with the denoise fallback's windows placed on purpose:
    isolated pixels, one-row and one-column strips, diagonals (singular
    normal matrices), and centres of 100 between a column of 1s and a column
    of 200s (with k_range = 1 a determined fit with intercept < 0), over a
    sparse random background."""
    D = np.where(rng.random((H, W)) < 0.15, rng.integers(3000, 60000, (H, W)), 0).astype(np.int32)
    for _ in range(12):
        v, u = int(rng.integers(3, H - 3)), int(rng.integers(3, W - 12))
        D[v - 2:v + 3, u - 2:u + 3] = 0
        D[v, u] = int(rng.integers(100, 90000))                    # isolated
    for _ in range(6):
        v, u = int(rng.integers(3, H - 3)), int(rng.integers(3, W - 14))
        D[v - 2:v + 3, u - 2:u + 12] = 0
        D[v, u:u + 10] = 5000 + 17 * np.arange(10)               # one row
        v, u = int(rng.integers(3, H - 14)), int(rng.integers(3, W - 3))
        D[v - 2:v + 12, u - 2:u + 3] = 0
        D[v:v + 10, u] = 8000 + 11 * np.arange(10)               # one column
        v, u = int(rng.integers(3, H - 10)), int(rng.integers(3, W - 10))
        D[v - 2:v + 9, u - 2:u + 9] = 0
        for k in range(7):
            D[v + k, u + k] = 4000 + 3 * k                        # diagonal
    for _ in range(10):
        v, u = int(rng.integers(3, H - 3)), int(rng.integers(3, W - 4))
        D[v - 2:v + 3, u - 2:u + 3] = 0
        D[v, u] = 100
        D[v - 2:v + 3, u + 1] = 1
        D[v - 2:v + 3, u + 2] = 200                               # intercept < 0 at (u, v)
    return D


@pytest.mark.parametrize("k_range", [0.05, 1.0])
def test_denoise_fallback_windows(P, k_range):
    # the denoise fallback (singular window, or intercept <= 0 with k_range =
    # 1) on purpose, through the fused chain and the stage entry point: den =
    # D / 256 and DENOISED clear exactly where the oracle falls back
    rng = np.random.default_rng(int(k_range * 100) + 5)
    D = _fallback_frame(rng)
    disp = codes_to_f32(D)
    H, W = D.shape
    g, ref = chain(P, disp, CAM, k_range=k_range)
    compare_frame(g, ref)
    fb = (ref.mask & oracle.M_VALID > 0) & (ref.mask & oracle.M_DENOISED == 0)
    assert fb.sum() >= 40, fb.sum()
    assert (g["den"][fb] == D[fb] / 256.0).all()
    if k_range == 1.0:
        # some fallbacks are determined fits (rank 3) with intercept <= 0
        den_o, fit = oracle.denoise(D, oracle.Params(k_range=1.0))
        centres = (D == 100) & (fit == 0)
        assert centres.sum() >= 5
    pipe = P.Pipeline(CAM, W, H, k_range=k_range)
    try:
        sn = P.sn
        d = pipe.upload(disp)
        den = sn.empty_image(H, W, torch.float32)
        m1 = sn.empty_image(H, W, torch.uint8)
        sn.sn_denoise(pipe.ctx, d, den, m1)
        torch.cuda.synchronize()
        sn.sn_check_device(pipe.ctx)
        assert np.array_equal(m1.cpu().numpy(), ref.mask & (oracle.M_VALID | oracle.M_DENOISED))
        err = np.abs(den.cpu().numpy().astype(np.float64) - ref.den)
        assert (err <= 1e-6 * ref.den).all()
    finally:
        pipe.close()


def test_all_invalid(P):
    disp = np.zeros((37, 45), np.float32)
    disp[3, 4] = np.nan
    disp[5, 6] = -3.0
    disp[7, 8] = np.inf
    disp[9, 9] = 1.0 / 1024
    g, ref = chain(P, disp, CAM)
    compare_frame(g, ref)
    assert ref.n_components == 0 and (g["labels"] == -1).all() and (g["mask"] == 0).all()


def test_constant_and_planes(P):
    D = np.full((48, 70), 9000, np.int32)
    g, ref = chain(P, codes_to_f32(D), CAM)
    compare_frame(g, ref)
    u = np.arange(70)[None, :]
    v = np.arange(48)[:, None]
    D = (30000 - 120 * u + 64 * v).astype(np.int32)
    g, ref = chain(P, codes_to_f32(D), CAM)
    compare_frame(g, ref)


# ------------------------------------------------------------ parameters
@pytest.mark.parametrize("params", [
    dict(support=1, dirs=16, steps=30),
    dict(support=1, dirs=16, steps=6),
    dict(support=1, dirs=4, steps=3, k_cd=0.02),
    dict(support=1, dirs=12, steps=7, k_cd=0.3),
    dict(support=2),
    dict(support=2, dirs=16, steps=30, st_t=0.05),
    dict(support=2, dirs=5, steps=4, st_t=1.0),
    dict(support=0, r_affine=1),
    dict(support=0, r_affine=2),
    dict(support=0, r_affine=3),
    dict(support=0, r_affine=5),
    dict(support=0, r_affine=6),
    dict(support=0, r_affine=7),
    dict(support=0, r_affine=15),
    dict(support=0, r_affine=7, r_denoise=3),
    dict(r_denoise=1, k_range=0.01),
    dict(r_denoise=4, k_range=0.2),
    dict(r_denoise=3, k_range=1.0, k_cd=1.0),
    dict(k_cd=0.0),
    dict(k_pair=0.0),
    dict(k_pair=1.0),
])
def test_parameter_sweep(P, params):
    s = make_scene("planes_320x240", frame=5)
    g, ref = chain(P, s.disp, s.camera, **params)
    compare_frame(g, ref)


def test_fp64_fallback_support(P):
    # support = the digital line (2k, k), k = -7..7, plus (1, 0): 1024 det < alpha gamma
    D = np.zeros((41, 41), np.int32)
    for k in range(-7, 8):
        D[20 + k, 20 + 2 * k] = 6000 + 10 * k
    D[20, 21] = 6003
    g, ref = chain(P, codes_to_f32(D), CAM, support=0, r_affine=15)
    assert ref.mask[20, 20] & oracle.M_FP64
    compare_frame(g, ref)


# ------------------------------------------------------------ components
def spiral(n):
    """A one-pixel corridor winding inwards, laps separated by one-pixel
    walls: a single component whose min-index label must travel through
    every tile of the frame."""
    D = np.zeros((n, n), np.int32)
    dirs = [(1, 0), (0, 1), (-1, 0), (0, -1)]
    x = y = k = 0
    D[0, 0] = 5000
    stuck = 0
    while stuck < 2:
        dx, dy = dirs[k]
        nx, ny, fx, fy = x + dx, y + dy, x + 2 * dx, y + 2 * dy
        inside = 0 <= nx < n and 0 <= ny < n
        blocked = 0 <= fx < n and 0 <= fy < n and D[fy, fx] != 0
        if inside and D[ny, nx] == 0 and not blocked:
            x, y = nx, ny
            D[y, x] = 5000
            stuck = 0
        else:
            k = (k + 1) % 4
            stuck += 1
    return D


@pytest.mark.parametrize("shape", ["spiral", "comb", "checker", "stripes", "random_steps"])
def test_components_adversarial(P, shape):
    rng = np.random.default_rng(11)
    if shape == "spiral":
        D = spiral(131)
    elif shape == "comb":
        D = np.zeros((100, 150), np.int32)
        D[:, ::2] = 7000
        D[0, :] = 7000
        D[99, 1::4] = 7000
    elif shape == "checker":
        D = ((np.indices((70, 90)).sum(0) % 2) * 6000).astype(np.int32)
        D[::7] = 6000
    elif shape == "stripes":
        D = np.full((96, 96), 8000, np.int32)
        D[:, 31::32] = 16000       # steps exactly on tile borders
        D[31::32, :] = 4000
    else:
        D = rng.choice([0, 1000, 1030, 1049, 1051, 1200, 3000], size=(150, 200)).astype(np.int32)
    H, W = D.shape
    cam = Camera(300.0, 300.0, W / 2, H / 2, 0.1)
    pipe = P.Pipeline(cam, W, H)
    try:
        disp = pipe.upload(codes_to_f32(D))
        labels = P.sn.empty_image(H, W, torch.int32)
        nc = torch.zeros(1, dtype=torch.int32, device="cuda")
        P.sn.sn_components(pipe.ctx, disp, labels, nc)
        torch.cuda.synchronize()
        P.sn.sn_check_device(pipe.ctx)
        lab, n = oracle.components(D, oracle_params(pipe.params))
        assert np.array_equal(labels.cpu().numpy(), lab)
        assert int(nc.item()) == n
    finally:
        pipe.close()


# ------------------------------------------------------------ stage entry points
@pytest.mark.parametrize("support", [1, 2])
def test_stage_entry_points(P, support):
    s = make_scene("mixed_1482x994", frame=2)
    H, W = s.disp.shape
    pipe = P.Pipeline(s.camera, W, H, support=support)
    sn = P.sn
    try:
        disp = pipe.upload(s.disp)
        den = sn.empty_image(H, W, torch.float32)
        m1 = sn.empty_image(H, W, torch.uint8)
        sn.sn_denoise(pipe.ctx, disp, den, m1)
        nrm = sn.empty_planes(3, H, W)
        m2 = sn.empty_image(H, W, torch.uint8)
        sn.sn_affine_normals(pipe.ctx, disp, den, nrm, m2)
        pts = sn.empty_planes(3, H, W)
        sn.sn_pointcloud(pipe.ctx, den, m1, pts)
        lab = sn.empty_image(H, W, torch.int32)
        sn.sn_components(pipe.ctx, disp, lab, None)
        torch.cuda.synchronize()
        sn.sn_check_device(pipe.ctx)
        op = oracle_params(pipe.params)
        D = oracle.ingest(s.disp)
        den_o, fit = oracle.denoise(D, op)
        g_den = den.cpu().numpy().astype(np.float64)
        assert (np.abs(g_den - den_o) <= 1e-6 * den_o).all()
        want1 = (D > 0).astype(np.uint8) * oracle.M_VALID | fit * oracle.M_DENOISED
        assert np.array_equal(m1.cpu().numpy(), want1)
        nrm_o, mask_o = oracle.affine_normals(D, den_o, s.camera, op)
        assert np.array_equal(m2.cpu().numpy(), mask_o)
        compare_normals(nrm.permute(1, 2, 0).cpu().numpy().astype(np.float64), nrm_o, mask_o)
        pts_o = oracle.points(den_o, want1, s.camera)
        perr = np.linalg.norm(pts.permute(1, 2, 0).cpu().numpy() - pts_o, axis=-1)
        assert (perr <= 1e-6 * np.linalg.norm(pts_o, axis=-1) + 1e-30).all()
        lab_o, _ = oracle.components(D, op)
        assert np.array_equal(lab.cpu().numpy(), lab_o)
    finally:
        pipe.close()


def test_repeatable_and_den_optional(P):
    s = make_scene("planes_640x480", frame=7)
    H, W = s.disp.shape
    pipe = P.Pipeline(s.camera, W, H)
    try:
        disp = pipe.upload(s.disp)
        a, b = pipe.buffers(), pipe.buffers()
        pipe.run_frame(disp, a)
        pipe.run_frame(disp, b, write_den=False)
        torch.cuda.synchronize()
        ha, hb = to_host(a), to_host(b)
        for k in ("normals", "points", "labels", "mask"):
            assert np.array_equal(ha[k], hb[k]), k
    finally:
        pipe.close()


def test_streams_and_graph_capture(P):
    # sn_run_frame forks its component passes onto a side stream of the
    # context and joins them back: frames interleaved on three caller streams
    # of one context, a profiled (single-stream) run and a CUDA graph capture
    # with replay all give the oracle's results
    scenes = [make_scene("planes_640x480", frame=f) for f in range(6)]
    H, W = scenes[0].disp.shape
    pipe = P.Pipeline(scenes[0].camera, W, H)
    try:
        disp = [pipe.upload(s.disp) for s in scenes]
        refs = [oracle.run_frame(s.disp, s.camera, oracle_params(pipe.params)) for s in scenes]
        outs = [pipe.buffers() for _ in scenes]
        streams = [torch.cuda.Stream() for _ in range(3)]
        for _ in range(3):
            for i in range(len(scenes)):
                pipe.run_frame(disp[i], outs[i], stream=streams[i % 3])
        torch.cuda.synchronize()
        P.sn.sn_check_device(pipe.ctx)
        for o, r in zip(outs, refs):
            compare_frame(to_host(o), r)

        P.sn.sn_set_profiling(pipe.ctx, True)
        prof = pipe.buffers()
        pipe.run_frame(disp[1], prof)
        torch.cuda.synchronize()
        P.sn.sn_set_profiling(pipe.ctx, False)
        compare_frame(to_host(prof), refs[1])

        cap = [pipe.buffers() for _ in scenes]
        g = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            g.capture_begin()
            for i in range(len(scenes)):
                pipe.run_frame(disp[i], cap[i], stream=side)
            g.capture_end()
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        for o in cap:
            for t in (o.normals, o.points, o.labels, o.mask, o.num_components):
                t.zero_()
        g.replay()
        torch.cuda.synchronize()
        P.sn.sn_check_device(pipe.ctx)
        for o, r in zip(cap, refs):
            compare_frame(to_host(o), r)
        del g
    finally:
        pipe.close()


def test_run_frame_host(P):
    # the C ABI on host buffers: copies in and out around sn_run_frame on the
    # caller's stream; six frames on two streams cycle through the context's
    # four staging sets; pinned and pageable host memory; results equal the
    # device call's bit for bit
    scenes = [make_scene("planes_640x480", frame=f) for f in range(6)]
    H, W = scenes[0].disp.shape
    pipe = P.Pipeline(scenes[0].camera, W, H)
    try:
        ref = []
        for sc in scenes:
            o = pipe.buffers()
            pipe.run_frame(pipe.upload(sc.disp), o, write_den=False)
            torch.cuda.synchronize()
            ref.append(to_host(o))
        streams = [torch.cuda.Stream() for _ in range(2)]
        for pin in (True, False):
            ins = [torch.from_numpy(sc.disp).pin_memory() if pin else torch.from_numpy(sc.disp) for sc in scenes]
            outs = [pipe.host_buffers(pin=pin) for _ in scenes]
            for i in range(len(scenes)):
                pipe.run_frame_host(ins[i], outs[i], stream=streams[i % 2])
            torch.cuda.synchronize()
            P.sn.sn_check_device(pipe.ctx)
            for o, r in zip(outs, ref):
                assert np.array_equal(o.normals.permute(1, 2, 0).numpy().astype(np.float64), r["normals"])
                assert np.array_equal(o.points.permute(1, 2, 0).numpy().astype(np.float64), r["points"])
                assert np.array_equal(o.labels.numpy(), r["labels"])
                assert np.array_equal(o.mask.numpy(), r["mask"])
                assert int(o.num_components.item()) == r["n_components"]
        # argument errors are found on the host before anything is enqueued
        o = pipe.host_buffers()
        short = torch.zeros((H, W // 2), dtype=torch.float32)  # rows shorter than the frame
        with pytest.raises(P.sn.SnError) as ei:
            P.sn.sn_run_frame_host(pipe.ctx, short, o.normals, o.points, o.labels, o.mask)
        assert ei.value.status == P.sn.SN_EINVAL
    finally:
        pipe.close()


def test_argument_errors_on_device(P):
    s = make_scene("planes_320x240", frame=0)
    H, W = s.disp.shape
    pipe = P.Pipeline(s.camera, W, H)
    sn = P.sn
    try:
        disp = pipe.upload(s.disp)
        out = pipe.buffers()
        bad = torch.empty((H, W), dtype=torch.float32, device="cuda")   # pitch 1280: fine
        odd = torch.empty((H, W + 1), dtype=torch.float32, device="cuda")[:, :W]  # pitch 1284
        with pytest.raises(sn.SnError) as ei:
            sn.sn_denoise(pipe.ctx, disp, odd, out.mask)
        assert ei.value.status == sn.SN_EINVAL
        small = sn.empty_image(H, W - 8, torch.float32)
        with pytest.raises(sn.SnError):
            sn.sn_denoise(pipe.ctx, disp, small, out.mask)
        sn.sn_denoise(pipe.ctx, disp, bad, out.mask)
        torch.cuda.synchronize()
    finally:
        pipe.close()


def test_walk_limit_reports_timeout_and_context_recovers(P):
    # fault detection without a fault: a union-find walk bound of one step
    # cannot resolve the spiral's chains across tiles; the component passes
    # stop, the error word is set and sn_check_device reports SN_ETIMEOUT;
    # with the default bound the same context labels the frame correctly
    sn = P.sn
    D = spiral(150)
    disp = codes_to_f32(D)
    cam = Camera(300.0, 300.0, 75.0, 75.0, 0.1)
    pipe = P.Pipeline(cam, 150, 150)
    try:
        d = pipe.upload(disp)
        out = pipe.buffers()
        sn.sn_set_walk_limit(pipe.ctx, 1)
        pipe.run_frame(d, out)
        torch.cuda.synchronize()
        with pytest.raises(sn.SnError) as ei:
            sn.sn_check_device(pipe.ctx)
        assert ei.value.status == sn.SN_ETIMEOUT
        sn.sn_set_walk_limit(pipe.ctx, 0)
        pipe.run_frame(d, out)
        torch.cuda.synchronize()
        sn.sn_check_device(pipe.ctx)
        g = to_host(out)
    finally:
        pipe.close()
    compare_frame(g, oracle.run_frame(disp, cam))
