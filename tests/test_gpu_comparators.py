"""Comparison estimators (Cross, PCA n x n; Sec. IV) through the C ABI
against the FP64 oracle (oracle/comparators.py), element by element.

* masks: bit-exact (every decision is an integer test);
* Cross normals: the parity bar of tests/parity.py (0.01 deg mean, 0.1 deg
  max);
* PCA normals: the same bar where the normal is unique -- the oracle's
  eigenvalue gap (l1 - l0) >= 1e-3 l2 (an FP32 covariance moves the
  eigenvector by ~1e-7 l2 / (l1 - l0) rad), and only the axis where the
  fitted plane nearly contains the viewing ray (|n . X| < 1e-3 |X|: its
  camera-facing sign is then not unique); everywhere unit length and facing
  the camera.  Far in the driving scene depth noise along the rays makes the
  two lateral eigenvalues nearly equal on a third of the pixels;
* accuracy trend of Sec. IV / Table noise-compare: on the sphere the error
  falls as the window grows and Affine n x n beats PCA n x n (the paper's
  one exception, 3x3 under sigma = 1, excepted).
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import comparators as cmp
from scenes import make_scene
from parity import NORMAL_MAX_DEG, NORMAL_MEAN_DEG, angle_deg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sn():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2504_15121_gb300 import sn
    return sn


def run(sn, s, which, r=0, disp=None, in_dtype=0):
    disp = s.disp if disp is None else disp
    ctx = sn.sn_create(s.camera, s.W, s.H, sn.default_params(in_dtype=in_dtype))
    try:
        d = sn.empty_image(s.H, s.W, torch.from_numpy(disp).dtype)
        d.copy_(torch.from_numpy(disp))
        nrm = sn.empty_planes(3, s.H, s.W)
        msk = sn.empty_image(s.H, s.W, torch.uint8)
        if which == "cross":
            sn.sn_cross_normals(ctx, d, nrm, msk)
        else:
            sn.sn_pca_normals(ctx, d, r, nrm, msk)
        torch.cuda.synchronize()
        sn.sn_check_device(ctx)
        return nrm.permute(1, 2, 0).cpu().numpy().astype(np.float64), msk.cpu().numpy()
    finally:
        sn.sn_destroy(ctx)


def check_facing(n, ok, s):
    X = np.nan_to_num(cmp.points(oracle.ingest(s.disp), s.camera))
    assert np.abs(np.linalg.norm(n[ok], axis=-1) - 1).max() < 1e-5
    # camera-facing; at grazing pixels the kernel's FP32 sign test and this
    # FP64 dot product may disagree by rounding
    assert ((n * X).sum(-1)[ok] < 1e-5 * np.linalg.norm(X, axis=-1)[ok]).all()


@pytest.mark.parametrize("name", ["planes_320x240", "mixed_1482x994", "driving_2048x1024"])
def test_cross_parity(sn, name):
    s = make_scene(name, frame=1)
    n, m = run(sn, s, "cross")
    D = oracle.ingest(s.disp)
    no, oko = cmp.cross_normals(D, s.camera)
    assert np.array_equal(m, (D > 0) * oracle.M_VALID + oko * oracle.M_NORMAL)
    a = angle_deg(n[oko], no[oko])
    print(f"cross {name}: mean {a.mean():.2e} max {a.max():.2e} deg")
    assert a.mean() <= NORMAL_MEAN_DEG and a.max() <= NORMAL_MAX_DEG
    check_facing(n, oko, s)


@pytest.mark.parametrize("name,r", [("planes_320x240", 1), ("planes_320x240", 4), ("planes_320x240", 7),
                                    ("mixed_1482x994", 4), ("driving_2048x1024", 4)])
def test_pca_parity(sn, name, r):
    s = make_scene(name, frame=2)
    n, m = run(sn, s, "pca", r)
    D = oracle.ingest(s.disp)
    no, oko, w = cmp.pca_normals(D, s.camera, r)
    assert np.array_equal(m, (D > 0) * oracle.M_VALID + oko * oracle.M_NORMAL)
    sure = oko & (w[..., 1] - w[..., 0] >= 1e-3 * w[..., 2])
    X = np.nan_to_num(cmp.points(D, s.camera))
    grazing = np.abs((no * X).sum(-1)) < 1e-3 * np.linalg.norm(X, axis=-1)
    a = angle_deg(n[sure], no[sure])
    a = np.where(grazing[sure], np.minimum(a, 180.0 - a), a)
    print(f"pca r{r} {name}: {sure.sum()} of {oko.sum()} unique ({(sure & grazing).sum()} grazing), "
          f"mean {a.mean():.2e} max {a.max():.2e} deg")
    assert sure.sum() > (0.5 if name.startswith("driving") else 0.9) * oko.sum()
    assert a.mean() <= NORMAL_MEAN_DEG and a.max() <= NORMAL_MAX_DEG
    check_facing(n, oko, s)


def test_uint16_input_matches_f32(sn):
    s = make_scene("driving_2048x1024", frame=3)
    same_codes = (s.disp_u16.astype(np.float64) / 256.0).astype(np.float32)
    for which, r in (("cross", 0), ("pca", 2)):
        n32, m32 = run(sn, s, which, r, disp=same_codes)
        n16, m16 = run(sn, s, which, r, disp=s.disp_u16, in_dtype=sn.SN_IN_U16X256)
        assert np.array_equal(m32, m16) and np.array_equal(n32, n16)   # same integer grid, same arithmetic


def test_bad_radius(sn):
    s = make_scene("planes_320x240", frame=0)
    for r in (0, 8):
        with pytest.raises(sn.SnError) as ei:
            run(sn, s, "pca", r)
        assert ei.value.status == sn.SN_EINVAL


def test_sphere_trend(sn):
    # Table noise-compare: Affine n x n and PCA n x n on the sphere at two
    # noise levels; errors fall with n, and Affine beats PCA at equal n
    # except at 3x3 under sigma = 1, where the paper itself has PCA ahead
    # (50.36 vs 51.74 deg)
    rows = {}
    for sigma in (0.2, 1.0):
        s = make_scene("sphere_1024", frame=0, sigma=sigma)
        fg = ~s.background
        gt = s.gt_normal.astype(np.float64)
        for n_ in (3, 5, 9, 15):
            r = n_ // 2
            from paper_2504_15121_gb300 import Pipeline
            pipe = Pipeline(s.camera, s.W, s.H, support=sn.SN_SUPPORT_FIXED, r_affine=r)
            try:
                d = pipe.upload(s.disp)
                out = pipe.buffers()
                pipe.run_frame(d, out)
                torch.cuda.synchronize()
                na = out.normals.permute(1, 2, 0).cpu().numpy().astype(np.float64)
                ma = out.mask.cpu().numpy()
            finally:
                pipe.close()
            np_, mp = run(sn, s, "pca", r)
            oka = ((ma & oracle.M_NORMAL) > 0) & fg
            okp = ((mp & oracle.M_NORMAL) > 0) & fg
            rows[(sigma, n_)] = (angle_deg(na[oka], gt[oka]).mean(), angle_deg(np_[okp], gt[okp]).mean())
            print(f"sphere sigma {sigma} n {n_}: affine {rows[(sigma, n_)][0]:.2f} pca {rows[(sigma, n_)][1]:.2f} deg")
    for sigma in (0.2, 1.0):
        aff = [rows[(sigma, n_)][0] for n_ in (3, 5, 9, 15)]
        pca = [rows[(sigma, n_)][1] for n_ in (3, 5, 9, 15)]
        assert all(x > y for x, y in zip(aff, aff[1:])) and all(x > y for x, y in zip(pca, pca[1:]))
        assert all(a < p for a, p, n_ in zip(aff, pca, (3, 5, 9, 15)) if sigma < 0.5 or n_ > 3)
