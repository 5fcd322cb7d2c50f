"""Host-side checks of libsn.so that need no GPU: exported symbols against
include/sn.h, the star-fill table against the oracle's, defaults and
argument validation (errors returned before any CUDA call)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle
from scenes import Camera

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def sn():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2504_15121_gb300 import sn as m
    return m


def declared_functions():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(sn_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_every_declared_symbol_is_exported(sn):
    names = declared_functions()
    assert "sn_run_frame" in names and len(names) >= 14
    lib = C.CDLL(sn.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    from paper_2504_15121_gb300 import serve, gate
    assert set(names) <= set(sn.EXPORTS) | set(serve.EXPORTS) | set(gate.EXPORTS)
    assert "sn_server_simulate" in names and "sn_normals_noalloc" in names


def test_learned_radius_matches_oracle():
    # the header's constant (compiled into the kernel) and the oracle's own
    text = open(os.path.join(ROOT, "include", "sn.h")).read()
    r = int(re.search(r"#define SN_LEARNED_RADIUS (\d+)", text).group(1))
    assert r == oracle.learned_radius()


@pytest.mark.parametrize("M,s", [(8, 10), (16, 30), (4, 1), (12, 7), (16, 6)])
def test_star_table_matches_oracle(sn, M, s):
    ou, ov = sn.star_offsets(M, s)
    ou_o, ov_o = oracle.star_offsets(M, s)
    assert np.array_equal(ou, ou_o) and np.array_equal(ov, ov_o)


def test_defaults(sn):
    p = sn.default_params()
    assert (p.r_denoise, p.r_affine, p.support, p.dirs, p.steps) == (2, 4, sn.SN_SUPPORT_STARFILL_CD, 8, 10)
    assert abs(p.k_cd - 0.1) < 1e-7 and abs(p.k_pair - 0.05) < 1e-7 and abs(p.tau - 0.9) < 1e-7
    assert (p.in_dtype, p.normal_fmt, p.learned) == (sn.SN_IN_F32, sn.SN_NORMALS_F32X3, 0)
    assert abs(p.st_t - 0.1) < 1e-7


@pytest.mark.parametrize("bad", [
    dict(W=0), dict(H=-1), dict(W=20000), dict(r_denoise=0), dict(r_denoise=5), dict(r_affine=16),
    dict(dirs=3), dict(dirs=17), dict(steps=31), dict(k_cd=-0.1), dict(k_pair=1.5), dict(support=7),
    dict(in_dtype=9), dict(normal_fmt=3), dict(fx=0.0), dict(baseline=-1.0), dict(support=3),
    dict(support=2, st_t=-1.0), dict(support=2, st_t=float("nan"))])
def test_create_rejects_bad_arguments(sn, bad):
    bad = dict(bad)
    W, H = bad.pop("W", 64), bad.pop("H", 48)
    cam = Camera(bad.pop("fx", 300.0), 300.0, 32.0, 24.0, bad.pop("baseline", 0.1))
    p = sn.default_params(**bad)
    with pytest.raises(sn.SnError) as ei:
        sn.sn_create(cam, W, H, p)
    assert ei.value.status == sn.SN_EINVAL


def test_status_strings(sn):
    for st in range(7):
        assert sn.lib.sn_status_string(st)
    assert sn.lib.sn_star_offsets(17, 3, None, None) == -1


def test_server_rejects_bad_config_before_any_cuda_call(sn):
    from paper_2504_15121_gb300 import serve
    cfg = serve.sn_server_config(0, None, 1 << 30, 2, 2, 0, 4)
    h = C.c_void_p()
    assert serve.lib.sn_server_create(C.byref(cfg), C.byref(h)) == sn.SN_EINVAL
    cams = (serve.sn_server_camera * 1)(serve.camera(64, 48, Camera(300.0, 300.0, 32.0, 24.0, 0.1)))
    for bad in (dict(n_streams=0), dict(n_streams=17), dict(max_slots_per_camera=0), dict(queue_depth=0)):
        kw = dict(n_streams=2, max_slots_per_camera=2, queue_depth=4)
        kw.update(bad)
        cfg = serve.sn_server_config(1, cams, 1 << 30, kw["max_slots_per_camera"], kw["n_streams"], 0,
                                     kw["queue_depth"])
        assert serve.lib.sn_server_create(C.byref(cfg), C.byref(h)) == sn.SN_EINVAL


def test_gate_weights_format(sn):
    from paper_2504_15121_gb300 import gate
    from oracle import gate as ogate
    assert gate.N_PARAMS == ogate.N_PARAMS == 3505
    th = gate.init_params(1)
    assert np.array_equal(gate.parse_blob(gate.weights_blob(th)), th)
    with pytest.raises(ValueError):
        gate.parse_blob(b"XXXX" + gate.weights_blob(th)[4:])


def test_training_labels_and_codes(sn):
    from paper_2504_15121_gb300 import gate
    from oracle import gate as ogate
    import oracle as orc
    rng = np.random.default_rng(4)
    d_true = np.repeat(rng.uniform(20, 40, (3, 4)), 8, 0).repeat(8, 1) + 0.05 * rng.normal(size=(24, 32))
    disp = (d_true + rng.normal(0, 0.3, d_true.shape)).astype(np.float32)
    disp[rng.random(d_true.shape) < 0.1] = 0
    D = gate.codes(disp)
    assert np.array_equal(D, orc.ingest(disp))
    lab = gate.one_surface_labels(d_true, D)
    assert np.array_equal(lab, ogate.patch_labels(d_true, D > 0))
    assert 0.05 < lab.mean() < 0.95
