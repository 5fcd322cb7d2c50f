"""FP64 oracle of the paper's comparison estimators (test infrastructure only).

Only the test suite, the package's smoke check and the benchmark's CPU leg
may import this module; the product never does.

Sec. IV ("Implemented algorithms") names two in-house comparators besides
the affine method:

* **Cross**: the normal from two tangent vectors, found by triangulating the
  pixel and its horizontal and vertical neighbours;
* **PCA n x n**: the normal as the eigenvector of the smallest eigenvalue of
  the 3x3 covariance of the window's 3-D points (the paper uses closed-form
  eigen formulas; here numpy's symmetric eigensolver is the step).

Readings (the paper gives no further detail):

* points come from the disparity grid `d = D / 256` of the other steps:
  `X = B (u - cx, fx/fy (v - cy), fx) / d`; invalid pixels (D = 0, or outside
  the image) carry no point;
* Cross: `t_u = X(u+1, v) - X(u, v)` when the right neighbour is valid, else
  `X(u, v) - X(u-1, v)` when the left one is, else none; `t_v` likewise
  downwards / upwards; `n = t_u x t_v` normalised; no normal when the centre
  or either tangent is missing;
* PCA: the valid pixels of the (2r+1)^2 window, centre included; the normal
  exists iff the centre is valid, there are >= 3 such pixels and they are
  not all on one image line (exact integer test on their offsets: the 2x2
  scatter determinant `(n Suu - Su^2)(n Svv - Sv^2) - (n Suv - Su Sv)^2 > 0`);
  covariance `C = sum (X_i - m)(X_i - m)^T` (unnormalised, m the mean);
* both orient the normal towards the camera (`n . X < 0`).
"""
from __future__ import annotations

import numpy as np


def points(D, cam):
    """3-D points [H, W, 3] of an integer-code image (NaN where invalid)."""
    D = np.asarray(D)
    H, W = D.shape
    valid = D > 0
    d = np.where(valid, D, 1).astype(np.float64) / 256.0
    u = np.arange(W, dtype=np.float64)[None, :]
    v = np.arange(H, dtype=np.float64)[:, None]
    X = np.stack([cam.baseline * (u - cam.cx) / d,
                  cam.baseline * cam.fx / cam.fy * (v - cam.cy) / d,
                  np.broadcast_to(cam.fx * cam.baseline / d, (H, W))], axis=-1)
    X[~valid] = np.nan
    return X


def _orient(n, X):
    flip = (n * X).sum(-1) > 0
    n[flip] *= -1
    return n


def cross_normals(D, cam):
    """(normals [H, W, 3], valid [H, W]) of the Cross estimator."""
    D = np.asarray(D)
    H, W = D.shape
    X = points(D, cam)
    valid = D > 0

    def tangent(axis):
        fwd = np.full_like(X, np.nan)
        bwd = np.full_like(X, np.nan)
        if axis == 1:
            fwd[:, :-1] = X[:, 1:] - X[:, :-1]
            bwd[:, 1:] = X[:, 1:] - X[:, :-1]
        else:
            fwd[:-1] = X[1:] - X[:-1]
            bwd[1:] = X[1:] - X[:-1]
        ok_f = ~np.isnan(fwd).any(-1)
        t = np.where(ok_f[..., None], fwd, bwd)
        return t, ok_f | ~np.isnan(bwd).any(-1)

    tu, oku = tangent(1)
    tv, okv = tangent(0)
    n = np.cross(np.nan_to_num(tu), np.nan_to_num(tv))
    ln = np.linalg.norm(n, axis=-1)
    ok = valid & oku & okv & (ln > 0)
    n = np.where(ok[..., None], n / np.where(ln > 0, ln, 1.0)[..., None], 0.0)
    n = _orient(n, np.nan_to_num(X))
    return n, ok


def pca_normals(D, cam, r):
    """(normals [H, W, 3], valid [H, W], eigenvalues [H, W, 3] ascending) of
    PCA over the (2r+1)^2 window."""
    D = np.asarray(D)
    H, W = D.shape
    X = points(D, cam)
    valid = D > 0
    P = r
    Xp = np.full((H + 2 * P, W + 2 * P, 3), np.nan)
    Xp[P:P + H, P:P + W] = X
    n = np.zeros((H, W))
    su = np.zeros((H, W))
    sv = np.zeros((H, W))
    suu = np.zeros((H, W))
    suv = np.zeros((H, W))
    svv = np.zeros((H, W))
    s1 = np.zeros((H, W, 3))
    s2 = np.zeros((H, W, 3, 3))
    Xc = np.nan_to_num(X)
    for ov in range(-r, r + 1):
        for ou in range(-r, r + 1):
            Y = Xp[P + ov:P + ov + H, P + ou:P + ou + W]
            ok = ~np.isnan(Y).any(-1)
            dY = np.where(ok[..., None], Y - Xc, 0.0)      # shifted by the centre point
            n += ok
            su += ok * ou
            sv += ok * ov
            suu += ok * ou * ou
            suv += ok * ou * ov
            svv += ok * ov * ov
            s1 += dY
            s2 += dY[..., :, None] * dY[..., None, :]
    det2 = (n * suu - su * su) * (n * svv - sv * sv) - (n * suv - su * sv) ** 2
    ok = valid & (n >= 3) & (det2 > 0)
    nn = np.maximum(n, 1)[..., None, None]
    C = s2 - s1[..., :, None] * s1[..., None, :] / nn
    C = np.where(ok[..., None, None], C, np.eye(3))
    w, V = np.linalg.eigh(C)
    nrm = np.where(ok[..., None], V[..., :, 0], 0.0)
    nrm = _orient(nrm, Xc)
    return nrm, ok, np.where(ok[..., None], w, 0.0)
