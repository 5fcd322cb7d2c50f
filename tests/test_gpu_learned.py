"""Learned form on the GPU (trained weights from paper_2504_15121_gb300/weights).

* q element by element: the gate's probability map from sn_gate_q lies, at
  every lattice point (pixels with both coordinates even; NaN elsewhere),
  inside the bounds oracle.gate.q_bounds derives for any kernel
  that computes the features exactly and accumulates in FP32 in any order
  (both roundings allowed where a layer-1 activation sits at a BF16 rounding
  boundary; the sigmoid within 2e-6); the table of log2 codes the features
  read equals numpy's FP32-rounded log2;
* gate decisions: the GPU's certified pixels (mask bit LEARNED) are those the
  bounds certify for sure, and none of those they exclude for sure; the
  pixels the bounds leave undecided are counted and reported;
* given those decisions the whole chain matches the oracle with the parity
  tolerances of tests/parity.py (masks and labels bit-exact);
* the gain: on each test scene the learned form certifies most pixels and
  its mean angular error against the generator's ground truth is no worse
  than the plain form's (the full window of radius 6 has more samples than
  the star and averages the noise down further).
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import gate as ogate
from scenes import make_scene
from parity import angle_deg, compare_frame, run_gpu

pytestmark = pytest.mark.gpu

TAU = float(np.float32(0.9))   # the library compares q with the FP32 tau


@pytest.fixture(scope="module")
def P():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2504_15121_gb300 as P
    return P


def gt_error(n, mask, scene):
    ok = ((mask & oracle.M_NORMAL) > 0) & ~scene.background
    return float(angle_deg(n[ok], scene.gt_normal[ok].astype(np.float64)).mean()), int(ok.sum())


def gpu_q(P, pipe, arr):
    sn = P.sn
    disp = pipe.upload(arr)
    q = sn.empty_image(pipe.H, pipe.W, torch.float32, fill=float("nan"))
    sn.sn_gate_q(pipe.ctx, disp, q)
    torch.cuda.synchronize()
    sn.sn_check_device(pipe.ctx)
    return q.cpu().numpy().astype(np.float64)


def check_gate(theta, D, q_gpu, gpu_gate, name):
    """q inside the oracle's bounds everywhere; decisions as the bounds
    force them; returns the number of undecided valid pixels."""
    sure, never, lo, hi = ogate.gate_bounds(D, theta, TAU, oracle.learned_radius())
    H, W = D.shape
    lat = np.zeros((H, W), bool)
    lat[::2, ::2] = True                      # q is evaluated at the lattice points only
    assert np.isnan(q_gpu[~lat]).all()
    out = lat & ((q_gpu < lo) | (q_gpu > hi) | ~np.isfinite(q_gpu))
    assert not out.any(), (name, int(out.sum()), np.argwhere(out)[:5],
                           np.abs(q_gpu - np.clip(q_gpu, lo, hi))[out].max())
    q_gpu, lo, hi = q_gpu[lat], lo[lat], hi[lat]
    assert not (sure & ~gpu_gate).any(), (name, int((sure & ~gpu_gate).sum()))
    assert not (never & gpu_gate).any(), (name, int((never & gpu_gate).sum()))
    undecided = int(((D > 0) & ~sure & ~never).sum())
    width = hi - lo
    print(f"{name}: q within bounds at {q_gpu.size} lattice points (width median {np.median(width):.1e}, "
          f"max {width.max():.1e}, max |q - q_fp64| {np.abs(q_gpu - 0.5 * (lo + hi)).max():.1e}); "
          f"undecided gate pixels {undecided}")
    return undecided


def test_log2_table_is_the_rounded_log2(P):
    t = P.sn.sn_gate_log2_table()
    assert np.isnan(t[0])
    ref = np.log2(np.arange(1, 131072, dtype=np.float64)).astype(np.float32)
    assert np.array_equal(t[1:], ref), np.argwhere(t[1:] != ref)[:5]


@pytest.mark.parametrize("name,frame", [("planes_640x480", 4), ("mixed_1482x994", 4), ("driving_2048x1024", 4)])
def test_learned_gate_and_chain(P, name, frame):
    from paper_2504_15121_gb300 import gate as G
    theta = G.load_weights().astype(np.float64)
    s = make_scene(name, frame=frame)
    pipe = P.Pipeline(s.camera, s.W, s.H, learned=1)
    try:
        g = run_gpu(pipe, s.disp)
        q = gpu_q(P, pipe, s.disp)
    finally:
        pipe.close()
    gpu_gate = (g["mask"] & oracle.M_LEARNED) > 0
    D = oracle.ingest(s.disp)
    undecided = check_gate(theta, D, q, gpu_gate, name)
    assert undecided <= 1e-3 * (D > 0).sum()
    ref = oracle.run_frame(s.disp, s.camera, gate=gpu_gate)
    compare_frame(g, ref)
    plain_ref = oracle.run_frame(s.disp, s.camera)
    e_learned, n_learned = gt_error(g["normals"], g["mask"], s)
    e_plain, n_plain = gt_error(plain_ref.normals, plain_ref.mask, s)
    frac = gpu_gate.sum() / max((D > 0).sum(), 1)
    print(f"{name}: certified {frac:.3f}, GT error learned {e_learned:.3f} deg "
          f"({n_learned}) vs plain {e_plain:.3f} deg ({n_plain})")
    assert frac > 0.3
    assert n_learned >= n_plain
    assert e_learned <= e_plain + 0.05


@pytest.mark.parametrize("dtype", ["f16", "u16"])
def test_learned_16bit_inputs(P, dtype):
    # the gate and chain kernels' 16-bit TMA boxes: q within the oracle's
    # bounds and the gated chain against the oracle, from FP16 and uint16 input
    from paper_2504_15121_gb300 import gate as G
    theta = G.load_weights().astype(np.float64)
    s = make_scene("driving_2048x1024", frame=3)
    arr, dt = (s.disp_f16, P.sn.SN_IN_F16) if dtype == "f16" else (s.disp_u16, P.sn.SN_IN_U16X256)
    pipe = P.Pipeline(s.camera, s.W, s.H, learned=1, in_dtype=dt)
    try:
        g = run_gpu(pipe, arr)
        q = gpu_q(P, pipe, arr)
    finally:
        pipe.close()
    gpu_gate = (g["mask"] & oracle.M_LEARNED) > 0
    D = oracle.ingest(arr)
    undecided = check_gate(theta, D, q, gpu_gate, f"driving {dtype}")
    assert undecided <= 1e-3 * (D > 0).sum()
    compare_frame(g, oracle.run_frame(arr, s.camera, gate=gpu_gate))


def test_learned_needs_weights_and_default_star(P):
    sn = P.sn
    s = make_scene("planes_320x240", frame=0)
    with pytest.raises(sn.SnError) as ei:
        sn.sn_create(s.camera, s.W, s.H, sn.default_params(learned=1, dirs=16))
    assert ei.value.status == sn.SN_ENOTSUP
    ctx = sn.sn_create(s.camera, s.W, s.H, sn.default_params(learned=1))
    try:
        pipe_out = P.FrameBuffers.allocate(s.W, s.H)
        disp = sn.empty_image(s.H, s.W, __import__("torch").float32, fill=1.0)
        with pytest.raises(sn.SnError) as ei:
            sn.sn_run_frame(ctx, disp, pipe_out.normals, pipe_out.points, pipe_out.labels, pipe_out.mask)
        assert ei.value.status == sn.SN_EINVAL
        with pytest.raises(sn.SnError):
            sn.sn_load_gate_weights(ctx, b"SNGW" + bytes(20))
    finally:
        sn.sn_destroy(ctx)


@pytest.mark.parametrize("H,W", [(1, 1), (7, 5), (17, 33), (40, 129), (70, 45)])
def test_learned_ragged(P, H, W):
    # frames smaller than, and not multiples of, the 32x16 tile: gate
    # decisions and the gated chain still match the oracle
    from paper_2504_15121_gb300 import gate as G
    from scenes import Camera
    theta = G.load_weights().astype(np.float64)
    rng = np.random.default_rng(H * 131 + W)
    base = rng.integers(6000, 6400, (H, W))
    blocks = rng.integers(0, 2, (H // 8 + 1, W // 8 + 1)).repeat(8, 0).repeat(8, 1)[:H, :W]
    D = (base * (1 + 0.3 * blocks)).astype(np.int32)
    D[rng.random((H, W)) < 0.05] = 0
    disp = (D / 256.0).astype(np.float32)
    cam = Camera(300.0, 300.0, W / 2, H / 2, 0.1)
    pipe = P.Pipeline(cam, W, H, learned=1)
    try:
        g = run_gpu(pipe, disp)
        q = gpu_q(P, pipe, disp)
    finally:
        pipe.close()
    gpu_gate = (g["mask"] & oracle.M_LEARNED) > 0
    check_gate(theta, D, q, gpu_gate, f"{H}x{W}")
    compare_frame(g, oracle.run_frame(disp, cam, gate=gpu_gate))


def test_learned_u16_matches_f32(P):
    # the learned kernel's TMA box for 16-bit input (16-byte aligned start
    # x0 - 16): uint16 codes and FP32 disparities on the same 1/256-px grid
    # give the same integer codes, hence identical outputs
    s = make_scene("driving_2048x1024", frame=6)
    same_codes = (s.disp_u16.astype(np.float64) / 256.0).astype(np.float32)
    out = []
    for arr, params in ((same_codes, {}), (s.disp_u16, dict(in_dtype=P.sn.SN_IN_U16X256))):
        pipe = P.Pipeline(s.camera, s.W, s.H, learned=1, **params)
        try:
            out.append(run_gpu(pipe, arr))
        finally:
            pipe.close()
    assert ((out[0]["mask"] & oracle.M_LEARNED) > 0).mean() > 0.5
    for k in ("normals", "points", "labels", "mask"):
        assert np.array_equal(out[0][k], out[1][k]), k
