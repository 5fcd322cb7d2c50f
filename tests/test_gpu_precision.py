"""Precision form: uint16 (256 d) or FP16 disparity in, snorm16 normals out.

Every output is compared with the FP64 oracle run on the same encoded input,
and the normals also with the generator's ground truth, next to the plain
FP32 form on the same scene.  Bounds:
  * mask, labels, component count: bit-exact;
  * denoised disparity and points: 1e-6 relative (FP32 arithmetic);
  * snorm16 normals: within one code of 32767 n_oracle per component;
  * mean angle to ground truth: the uint16 form equals the FP32 form's (the
    kernels quantise FP32 input to the same 1/256-px grid) up to snorm
    rounding, 0.005 deg; the FP16 form within 0.05 deg of it (FP16 spacing is
    1/64 px at 16-32 px, well below the 0.3 px noise).
"""
import numpy as np
import pytest
import torch

import oracle
from scenes import make_scene
from parity import angle_deg, oracle_params, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2504_15121_gb300 as P
    return P


def gt_angle(n, scene, mask):
    ok = ((mask & oracle.M_NORMAL) > 0) & ~scene.background
    return float(angle_deg(n[ok], scene.gt_normal[ok].astype(np.float64)).mean())


def decode_snorm(q):
    n = q[..., :3].astype(np.float64) / 32767.0
    return n


def run_form(P, scene, disp, in_dtype, normal_fmt):
    pipe = P.Pipeline(scene.camera, scene.W, scene.H, in_dtype=in_dtype, normal_fmt=normal_fmt)
    try:
        g = run_gpu(pipe, disp)
        ref = oracle.run_frame(disp, scene.camera, oracle_params(pipe.params))
    finally:
        pipe.close()
    return g, ref


def test_precision_form_error_report(P):
    sn = P.sn
    s = make_scene("driving_2048x1024", frame=3)
    report = {}
    g32, r32 = run_form(P, s, s.disp, sn.SN_IN_F32, sn.SN_NORMALS_F32X3)
    report["f32"] = gt_angle(g32["normals"], s, g32["mask"])
    for name, arr, dt in (("u16", s.disp_u16, sn.SN_IN_U16X256), ("f16", s.disp_f16, sn.SN_IN_F16)):
        g, ref = run_form(P, s, arr, dt, sn.SN_NORMALS_SNORM16X4)
        assert np.array_equal(g["mask"], ref.mask)
        assert np.array_equal(g["labels"], ref.labels) and g["n_components"] == ref.n_components
        den_err = np.abs(g["den"] - ref.den) / np.maximum(ref.den, 1e-30)
        assert den_err.max() <= 1e-6
        perr = np.linalg.norm(g["points"] - ref.points, axis=-1) / np.maximum(np.linalg.norm(ref.points, axis=-1), 1e-30)
        assert perr.max() <= 1e-6
        q = g["normals"].astype(np.int64)
        ok = (ref.mask & oracle.M_NORMAL) > 0
        code_err = np.abs(q[..., :3][ok] - 32767.0 * ref.normals[ok])
        assert code_err.max() <= 1.0
        n = decode_snorm(q)
        ang_oracle = angle_deg(n[ok], ref.normals[ok])
        report[name] = gt_angle(n, s, g["mask"])
        report[name + "_vs_oracle_mean_deg"] = float(ang_oracle.mean())
        report[name + "_vs_oracle_max_deg"] = float(ang_oracle.max())
        report[name + "_den_max_rel"] = float(den_err.max())
        report[name + "_points_max_rel"] = float(perr.max())
    print(report)
    assert abs(report["u16"] - report["f32"]) <= 0.005
    assert abs(report["f16"] - report["f32"]) <= 0.05
    assert report["u16_vs_oracle_max_deg"] <= 0.01
