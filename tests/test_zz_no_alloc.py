"""sn_normals_noalloc: the allocation-free denoise + normals entry point.

It serves callers that cannot call cudaMalloc (a plugin whose host owns all
device memory, a real-time loop that must not allocate).  Through the C ABI it
must give the results of sn_denoise followed by sn_affine_normals, within the
parity tolerances of tests/parity.py, on two calls in a row (the second call
reuses the static scratch the first one left behind).  This file sorts last
so that a run stopping at the first failure has run every other test.
"""
import numpy as np
import pytest
import torch

from scenes import make_scene
from parity import NORMAL_MAX_DEG, NORMAL_MEAN_DEG, angle_deg

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
    nrm = sn.empty_planes(3, H, W)
    mask = sn.empty_image(H, W, torch.uint8)
    sn.sn_affine_normals(pipe.ctx, disp, den, nrm, mask)
    return nrm, mask


def test_noalloc_matches_context_path_twice(P):
    sn = P.sn
    scenes = [make_scene("mixed_1482x994", frame=4), make_scene("mixed_1482x994", frame=5)]
    s0 = scenes[0]
    H, W = s0.disp.shape
    pipe = P.Pipeline(s0.camera, W, H)
    try:
        for s in scenes:     # two calls in a row on different inputs
            disp = pipe.upload(s.disp)
            want_n, want_m = reference_normals(P, pipe, disp)
            got_n = sn.empty_planes(3, H, W)
            got_n.fill_(float("nan"))
            got_m = sn.empty_image(H, W, torch.uint8, fill=255)
            sn.sn_normals_noalloc(s.camera, None, disp, got_n, got_m)
            torch.cuda.synchronize()
            gm, wm = got_m.cpu().numpy(), want_m.cpu().numpy()
            assert np.array_equal(gm, wm)
            ok = (wm & sn.SN_MASK_NORMAL) > 0
            gn = got_n.permute(1, 2, 0).cpu().numpy().astype(np.float64)
            wn = want_n.permute(1, 2, 0).cpu().numpy().astype(np.float64)
            assert (gn[~ok] == 0).all()
            ang = angle_deg(gn[ok], wn[ok])
            assert ang.mean() <= NORMAL_MEAN_DEG and ang.max() <= NORMAL_MAX_DEG
    finally:
        pipe.close()


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
