"""Shared helpers of the GPU parity tests: run a frame through the C ABI and
through the oracle on the same seeded input, and compare element by element.

Tolerances (written out here, used by every parity test):
  * masks, labels, component counts: bit-exact;
  * normals: angle to the oracle's normal, mean <= 0.01 deg and
    max <= 0.1 deg over pixels with a valid normal (FP32 path);
  * denoised disparity: |gpu - oracle| <= 1e-6 * oracle (a few FP32 ulps;
    every window sum is an exact integer, only the final quotient rounds);
  * points: |gpu - oracle| <= 1e-6 * |X_oracle| per point.
"""
from __future__ import annotations

import numpy as np
import torch

import oracle

NORMAL_MEAN_DEG = 0.01
NORMAL_MAX_DEG = 0.1
DEN_RTOL = 1e-6
PTS_RTOL = 1e-6


def oracle_params(p) -> oracle.Params:
    """The oracle's parameter record for a library sn_params."""
    return oracle.Params(r_denoise=p.r_denoise, r_affine=p.r_affine, support=p.support,
                         dirs=p.dirs, steps=p.steps, k_cd=float(p.k_cd), k_pair=float(p.k_pair),
                         k_range=float(p.k_range), st_t=float(p.st_t))


def run_gpu(pipe, disp_np):
    disp = pipe.upload(disp_np)
    out = pipe.buffers()
    pipe.run_frame(disp, out)
    torch.cuda.synchronize()
    from paper_2504_15121_gb300 import sn
    sn.sn_check_device(pipe.ctx)
    return to_host(out, pipe.params.normal_fmt)


def to_host(out, normal_fmt=0):
    if normal_fmt == 0:
        nrm = out.normals.permute(1, 2, 0).cpu().numpy().astype(np.float64)
    else:
        nrm = out.normals.cpu().numpy()
    return dict(
        den=out.den.cpu().numpy().astype(np.float64),
        normals=nrm,
        points=out.points.permute(1, 2, 0).cpu().numpy().astype(np.float64),
        labels=out.labels.cpu().numpy(),
        mask=out.mask.cpu().numpy(),
        n_components=int(out.num_components.item()),
    )


def angle_deg(a, b):
    """Angle between vectors, atan2(|a x b|, a . b): accurate for tiny angles
    and insensitive to the FP32 rounding of the vectors' lengths (arccos of a
    dot product is not: near 1 it turns a 1e-7 length error into 0.02 deg)."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.degrees(np.arctan2(np.linalg.norm(np.cross(a, b), axis=-1), (a * b).sum(-1)))


def compare_normals(gpu_n, ref_n, ref_mask):
    ok = (ref_mask & oracle.M_NORMAL) > 0
    assert (gpu_n[~ok] == 0).all(), "normal written where the oracle has none"
    if not ok.any():
        return 0.0, 0.0
    ang = angle_deg(gpu_n[ok], ref_n[ok])
    assert np.isfinite(ang).all()
    assert ang.mean() <= NORMAL_MEAN_DEG, ang.mean()
    assert ang.max() <= NORMAL_MAX_DEG, ang.max()
    return float(ang.mean()), float(ang.max())


def compare_frame(g, ref, check_den=True):
    assert np.array_equal(g["mask"], ref.mask), mismatch("mask", g["mask"], ref.mask)
    assert np.array_equal(g["labels"], ref.labels), mismatch("labels", g["labels"], ref.labels)
    assert g["n_components"] == ref.n_components
    if check_den:
        err = np.abs(g["den"] - ref.den)
        assert (err <= DEN_RTOL * np.abs(ref.den)).all(), err.max()
    mean, mx = compare_normals(g["normals"], ref.normals, ref.mask)
    scale = np.linalg.norm(ref.points, axis=-1)
    perr = np.linalg.norm(g["points"] - ref.points, axis=-1)
    assert (perr <= PTS_RTOL * scale + 1e-30).all(), (perr / np.maximum(scale, 1e-30)).max()
    return mean, mx


def mismatch(name, a, b):
    bad = np.argwhere(a != b)
    if bad.size == 0:
        return f"{name}: shapes {a.shape} vs {b.shape}"
    v, u = bad[0]
    return f"{name}: {len(bad)} mismatches, first at (u={u}, v={v}): gpu {a[v, u]} oracle {b[v, u]}"
