"""Pins of the comparator oracle (oracle/comparators.py): the Cross and PCA
estimators named in Sec. IV.

* on an exact plane both return the plane's normal, known in closed form
  from its disparity gradient (d = gu u + gv v + c is the plane
  fB = gu fx x + gv fy y + (gu cx + gv cy + c) z);
* PCA equals, pixel by pixel, the last right singular vector of the centred
  window points (numpy SVD, a route that forms no covariance);
* Cross equals a triangle normal computed by hand, with the backward
  neighbour standing in for an invalid forward one;
* degenerate windows (fewer than 3 points, points on one image line) have
  no normal; normals face the camera.
"""
import numpy as np

from oracle import comparators as cmp
from scenes import Camera

CAM = Camera(fx=310.0, fy=290.0, cx=20.5, cy=13.0, baseline=0.12)


def plane_codes(H, W, gu=37, gv=-23, c=26000):
    u = np.arange(W)[None, :]
    v = np.arange(H)[:, None]
    return (c + gu * u + gv * v).astype(np.int64), (gu / 256.0, gv / 256.0, c / 256.0)


def plane_normal(g, cam):
    gu, gv, c = g
    n = np.array([gu * cam.fx, gv * cam.fy, gu * cam.cx + gv * cam.cy + c])
    return -n / np.linalg.norm(n)     # n . X = -fB / |n| < 0: faces the camera


def test_plane_gives_the_closed_form_normal():
    D, g = plane_codes(30, 41)
    want = plane_normal(g, CAM)
    nc, okc = cmp.cross_normals(D, CAM)
    assert okc.all()
    assert np.abs(nc - want).max() < 1e-9
    for r in (1, 2, 4):
        npca, okp, w = cmp.pca_normals(D, CAM, r)
        assert okp.all()
        assert np.abs(npca - want).max() < 1e-7
        assert (np.abs(w[..., 0]) < 1e-9 * w[..., 2]).all()     # the points are coplanar


def test_pca_matches_svd_of_centred_points():
    rng = np.random.default_rng(0)
    H, W, r = 9, 11, 2
    D, _ = plane_codes(H, W)
    D = D + rng.integers(-400, 400, D.shape)
    D[rng.random(D.shape) < 0.15] = 0
    n, ok, _ = cmp.pca_normals(D, CAM, r)
    X = cmp.points(D, CAM)
    checked = 0
    for v in range(H):
        for u in range(W):
            pts = [X[v + ov, u + ou] for ov in range(-r, r + 1) for ou in range(-r, r + 1)
                   if 0 <= v + ov < H and 0 <= u + ou < W and D[v + ov, u + ou] > 0]
            if not ok[v, u]:
                continue
            Pm = np.array(pts)
            _, _, Vt = np.linalg.svd(Pm - Pm.mean(0))
            want = Vt[-1] * (-1 if Vt[-1] @ X[v, u] > 0 else 1)
            assert np.abs(n[v, u] - want).max() < 1e-9, (v, u)
            checked += 1
    assert checked > 50


def test_cross_by_hand():
    D, _ = plane_codes(4, 5)
    D = D + np.array([[0, 300, -200, 0, 0], [0, -100, 50, 0, 0], [0, 0, 0, 0, 0], [0, 0, 0, 0, 0]])
    D[1, 2] = 0                        # pixel (1, 1): right neighbour invalid -> backward difference
    X = cmp.points(D, CAM)
    n, ok = cmp.cross_normals(D, CAM)
    # pixel (0, 1): forward in u and v
    tu = X[0, 2] - X[0, 1]
    tv = X[1, 1] - X[0, 1]
    m = np.cross(tu, tv)
    m = m / np.linalg.norm(m)
    m = -m if m @ X[0, 1] > 0 else m
    assert ok[0, 1] and np.abs(n[0, 1] - m).max() < 1e-12
    # pixel (1, 1): backward in u (X(u) - X(u-1)), forward in v
    tu = X[1, 1] - X[1, 0]
    tv = X[2, 1] - X[1, 1]
    m = np.cross(tu, tv)
    m = m / np.linalg.norm(m)
    m = -m if m @ X[1, 1] > 0 else m
    assert ok[1, 1] and np.abs(n[1, 1] - m).max() < 1e-12
    assert not ok[1, 2]                # invalid centre
    assert ((n * np.nan_to_num(X)).sum(-1)[ok] < 0).all()


def test_degenerate_windows_have_no_normal():
    D, _ = plane_codes(7, 9)
    only_row = np.zeros_like(D)
    only_row[3] = D[3]                 # every window holds points of one image row
    _, ok, _ = cmp.pca_normals(only_row, CAM, 2)
    assert not ok.any()
    two = np.zeros_like(D)
    two[3, 4] = D[3, 4]
    two[4, 5] = D[4, 5]                # two points
    _, ok, _ = cmp.pca_normals(two, CAM, 2)
    assert not ok.any()
    three = two.copy()
    three[2, 4] = D[2, 4]              # three points not on one line
    _, ok, _ = cmp.pca_normals(three, CAM, 2)
    assert ok[3, 4] and ok[4, 5] and ok.sum() == 3
    _, okc = cmp.cross_normals(only_row, CAM)
    assert not okc.any()               # no vertical tangent anywhere
