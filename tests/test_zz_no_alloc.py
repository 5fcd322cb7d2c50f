"""sn_normals_noalloc: the allocation-free denoise + normals entry point.

It serves callers that cannot call cudaMalloc (a plugin whose host owns all
device memory, a real-time loop that must not allocate).  Through the C ABI it
must give the results of sn_denoise followed by sn_affine_normals: checked
against the FP64 oracle (masks bit-exact, normals within the tolerances of
tests/parity.py) and against the context path, on two calls in a row (the
second call reuses the static scratch the first one left behind), on a frame
that fills the scratch exactly (2048 x 1024), with 16-bit input and snorm16
normals, and with the fixed window.  Its error word, read by
sn_noalloc_check_device, stays clear.  This file sorts last so that a run
stopping at the first failure has run every other test.
"""
import numpy as np
import pytest
import torch

import oracle
from scenes import make_scene
from parity import NORMAL_MAX_DEG, NORMAL_MEAN_DEG, angle_deg, compare_normals, oracle_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2504_15121_gb300 as P
    return P


def reference_normals(P, pipe, disp):
    sn = P.sn
    H, W = disp.shape
    den = sn.empty_image(H, W, torch.float32)
    m1 = sn.empty_image(H, W, torch.uint8)
    sn.sn_denoise(pipe.ctx, disp, den, m1)
    nrm = sn.empty_planes(3, H, W) if pipe.params.normal_fmt == 0 else sn.empty_snorm(H, W)
    mask = sn.empty_image(H, W, torch.uint8)
    sn.sn_affine_normals(pipe.ctx, disp, den, nrm, mask)
    return nrm, mask


def normals_f64(P, nrm, normal_fmt, H, W):
    if normal_fmt == 0:
        return nrm.permute(1, 2, 0).cpu().numpy().astype(np.float64)
    q = nrm.cpu().numpy().astype(np.float64)          # [H, W, 4] snorm16
    return q[..., :3] / 32767.0


def noalloc_call(P, s, arr, **params):
    """One sn_normals_noalloc call on scene s (input array arr) next to the
    context path; both compared with the oracle.  Returns the mean and max
    normal deviation from the oracle (degrees)."""
    sn = P.sn
    H, W = arr.shape
    pipe = P.Pipeline(s.camera, W, H, **params)
    try:
        disp = pipe.upload(arr)
        fmt = pipe.params.normal_fmt
        want_n, want_m = reference_normals(P, pipe, disp)
        got_n = sn.empty_planes(3, H, W) if fmt == 0 else sn.empty_snorm(H, W)
        got_n.fill_(float("nan") if fmt == 0 else -12345)
        got_m = sn.empty_image(H, W, torch.uint8, fill=255)
        sn.sn_normals_noalloc(s.camera, pipe.params, disp, got_n, got_m)
        torch.cuda.synchronize()
        sn.sn_noalloc_check_device()
        gm, wm = got_m.cpu().numpy(), want_m.cpu().numpy()
        assert np.array_equal(gm, wm)
        gn = normals_f64(P, got_n, fmt, H, W)
        wn = normals_f64(P, want_n, fmt, H, W)
        ok = (wm & sn.SN_MASK_NORMAL) > 0
        assert (gn[~ok] == 0).all()
        ang = angle_deg(gn[ok], wn[ok])
        assert ang.mean() <= NORMAL_MEAN_DEG and ang.max() <= NORMAL_MAX_DEG
        # the FP64 oracle on the same codes
        op = oracle_params(pipe.params)
        D = oracle.ingest(arr)
        den_o, _ = oracle.denoise(D, op)
        nrm_o, mask_o = oracle.affine_normals(D, den_o, s.camera, op)
        assert np.array_equal(gm, mask_o)
        return compare_normals(gn, nrm_o, mask_o)
    finally:
        pipe.close()


def test_noalloc_matches_oracle_and_context_path_twice(P):
    # two calls in a row on different inputs of the same size
    for frame in (4, 5):
        s = make_scene("mixed_1482x994", frame=frame)
        noalloc_call(P, s, s.disp)


def test_noalloc_at_the_scratch_limit(P):
    # 2048 x 1024 fills the static scratch exactly (rows of 2048 floats)
    s = make_scene("driving_2048x1024", frame=2)
    noalloc_call(P, s, s.disp)


def test_noalloc_u16_input_snorm16_normals(P):
    s = make_scene("driving_2048x1024", frame=3)
    noalloc_call(P, s, s.disp_u16, in_dtype=P.sn.SN_IN_U16X256, normal_fmt=P.sn.SN_NORMALS_SNORM16X4)


@pytest.mark.parametrize("support,extra", [(0, {}), (2, {"st_t": 0.1}), (1, {"dirs": 16, "steps": 30})])
def test_noalloc_other_supports(P, support, extra):
    # the fixed 9x9 window, the ST star and a star table take the generic
    # stage kernels instead of the 5x5 / M = 8, s = 10 fast paths
    s = make_scene("planes_640x480", frame=6)
    noalloc_call(P, s, s.disp, support=support, **extra)


def test_noalloc_rejects_frames_beyond_the_scratch(P):
    sn = P.sn
    s = make_scene("planes_320x240", frame=0)
    H, W = 1025, 2048          # one row more than the 2048 x 1024 scratch holds
    disp = sn.empty_image(H, W, torch.float32, fill=0.0)
    nrm = sn.empty_planes(3, H, W)
    mask = sn.empty_image(H, W, torch.uint8)
    with pytest.raises(sn.SnError) as ei:
        sn.sn_normals_noalloc(s.camera, None, disp, nrm, mask)
    assert ei.value.status == sn.SN_EINVAL
    sn.sn_noalloc_check_device()
