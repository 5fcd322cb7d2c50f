"""Thin ctypes binding of libsn.so (include/sn.h), same names as the C ABI.

Only argument marshalling happens here: torch tensors are turned into device
pointers and byte pitches and handed to the library, which enqueues its own
CUDA kernels on the given stream.  Nothing is computed in Python and there is
no fallback: if the library is missing, importing this module raises.

Tensor conventions (see include/sn.h):
  * a 2-D image is a view [H, W] of a pitched buffer: stride(1) == 1 and the
    row pitch in bytes is stride(0) * element_size, a multiple of 16;
  * a multi-plane output (normals as 3 float planes, points) is a view
    [3, H, W] whose planes are back to back: stride(0) == H * stride(1);
  * SNORM16x4 normals are an int16 view [H, W, 4] with stride(1) == 4.
Use `empty_image` / `empty_planes` to allocate such buffers.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libsn.so")

SN_OK, SN_EINVAL, SN_ENOMEM, SN_ECUDA, SN_ETIMEOUT, SN_EBUSY, SN_ENOTSUP = range(7)
SN_SUPPORT_FIXED, SN_SUPPORT_STARFILL_CD, SN_SUPPORT_STARFILL_ST = 0, 1, 2
SN_IN_F32, SN_IN_F16, SN_IN_U16X256 = 0, 1, 2
SN_NORMALS_F32X3, SN_NORMALS_SNORM16X4 = 0, 1
SN_MASK_VALID, SN_MASK_NORMAL, SN_MASK_FP64, SN_MASK_LEARNED, SN_MASK_DENOISED = 1, 2, 4, 8, 16


class sn_camera(C.Structure):
    _fields_ = [("fx", C.c_double), ("fy", C.c_double), ("cx", C.c_double), ("cy", C.c_double),
                ("baseline", C.c_double)]


class sn_params(C.Structure):
    _fields_ = [("r_denoise", C.c_int), ("r_affine", C.c_int), ("support", C.c_int),
                ("dirs", C.c_int), ("steps", C.c_int), ("k_cd", C.c_float), ("k_pair", C.c_float),
                ("k_range", C.c_float), ("tau", C.c_float), ("in_dtype", C.c_int),
                ("normal_fmt", C.c_int), ("learned", C.c_int), ("st_t", C.c_float)]


class sn_frame_in(C.Structure):
    _fields_ = [("disp", C.c_void_p), ("disp_pitch", C.c_size_t)]


class sn_frame_out(C.Structure):
    _fields_ = [("den", C.c_void_p), ("den_pitch", C.c_size_t),
                ("normals", C.c_void_p), ("normals_pitch", C.c_size_t),
                ("points", C.c_void_p), ("points_pitch", C.c_size_t),
                ("labels", C.c_void_p), ("labels_pitch", C.c_size_t),
                ("mask", C.c_void_p), ("mask_pitch", C.c_size_t),
                ("num_components", C.c_void_p)]


class SnError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built; run __graft_entry__.build() or "
                          "python -m paper_2504_15121_gb300.build")
    L = C.CDLL(LIB_PATH)
    vp, sz, i = C.c_void_p, C.c_size_t, C.c_int
    sig = {
        "sn_version": ([], i),
        "sn_default_params": ([C.POINTER(sn_params)], None),
        "sn_create": ([C.POINTER(sn_camera), i, i, C.POINTER(sn_params), C.POINTER(vp)], i),
        "sn_destroy": ([vp], i),
        "sn_denoise": ([vp, vp, sz, vp, sz, vp, sz, vp], i),
        "sn_affine_normals": ([vp, vp, sz, vp, sz, vp, sz, vp, sz, vp], i),
        "sn_components": ([vp, vp, sz, vp, sz, vp, vp], i),
        "sn_cross_normals": ([vp, vp, sz, vp, sz, vp, sz, vp], i),
        "sn_pca_normals": ([vp, vp, sz, i, vp, sz, vp, sz, vp], i),
        "sn_pointcloud": ([vp, vp, sz, vp, sz, vp, sz, vp], i),
        "sn_run_frame": ([vp, C.POINTER(sn_frame_in), C.POINTER(sn_frame_out), vp], i),
        "sn_run_frame_host": ([vp, C.POINTER(sn_frame_in), C.POINTER(sn_frame_out), vp], i),
        "sn_load_gate_weights": ([vp, vp, sz], i),
        "sn_star_offsets": ([i, i, vp, vp], i),
        "sn_check_device": ([vp, vp], i),
        "sn_set_walk_limit": ([vp, i], i),
        "sn_status_string": ([i], C.c_char_p),
        "sn_last_error": ([vp], C.c_char_p),
        "sn_set_profiling": ([vp, i], i),
        "sn_stage_count": ([vp], i),
        "sn_stage_name": ([vp, i], C.c_char_p),
        "sn_stage_times": ([vp, C.POINTER(C.c_double), i, C.POINTER(C.c_int), C.POINTER(C.c_double), i], i),
        "sn_launch_count": ([vp], C.c_uint64),
        "sn_normals_noalloc": ([C.POINTER(sn_camera), C.POINTER(sn_params), i, i, vp, sz, vp, sz, vp,
                                sz, vp], i),
        "sn_noalloc_check_device": ([vp], i),
        "sn_gate_q": ([vp, vp, sz, vp, sz, vp], i),
        "sn_gate_log2_table": ([vp, i], i),
        "sn_rcp_table": ([vp, i], i),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    return L


lib = _load()

# names the C ABI declares (used by the tests that check the exports)
EXPORTS = ("sn_version", "sn_default_params", "sn_create", "sn_destroy", "sn_denoise",
           "sn_affine_normals", "sn_components", "sn_pointcloud", "sn_run_frame",
           "sn_load_gate_weights", "sn_star_offsets", "sn_check_device", "sn_status_string",
           "sn_last_error", "sn_set_profiling", "sn_stage_count", "sn_stage_name",
           "sn_stage_times", "sn_launch_count", "sn_normals_noalloc", "sn_noalloc_check_device", "sn_cross_normals",
           "sn_pca_normals", "sn_set_walk_limit", "sn_run_frame_host", "sn_gate_q", "sn_gate_log2_table",
           "sn_rcp_table")


# ---------------------------------------------------------------- helpers
def _check(ctx, st):
    if st != SN_OK:
        msg = lib.sn_last_error(ctx).decode() if ctx else lib.sn_status_string(st).decode()
        raise SnError(st, msg)


def _stream(stream):
    if stream is None:
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def _img(t: torch.Tensor | None):
    """(pointer, pitch bytes) of a 2-D pitched view, or of the first plane of
    a [P, H, W] view with back-to-back planes, or of an [H, W, 4] int16 view."""
    if t is None:
        return None, 0
    if t.dim() == 2:
        assert t.stride(1) == 1
        return C.c_void_p(t.data_ptr()), t.stride(0) * t.element_size()
    if t.dim() == 3 and t.dtype == torch.int16 and t.shape[2] == 4:
        assert t.stride(2) == 1 and t.stride(1) == 4
        return C.c_void_p(t.data_ptr()), t.stride(0) * t.element_size()
    assert t.dim() == 3 and t.stride(2) == 1 and t.stride(0) == t.shape[1] * t.stride(1), \
        "planes must be back to back"
    return C.c_void_p(t.data_ptr()), t.stride(1) * t.element_size()


def pitch_elems(W: int, elem: int, align: int = 16) -> int:
    return ((W * elem + align - 1) // align * align) // elem


def empty_image(H, W, dtype, device="cuda", fill=None):
    """[H, W] view of a buffer whose rows are padded to 16 bytes."""
    elem = torch.empty((), dtype=dtype).element_size()
    base = torch.empty((H, pitch_elems(W, elem)), dtype=dtype, device=device)
    if fill is not None:
        base.fill_(fill)
    return base[:, :W]


def empty_planes(P, H, W, dtype=torch.float32, device="cuda"):
    """[P, H, W] view of P back-to-back pitched planes."""
    elem = torch.empty((), dtype=dtype).element_size()
    base = torch.empty((P, H, pitch_elems(W, elem)), dtype=dtype, device=device)
    return base[:, :, :W]


def empty_snorm(H, W, device="cuda"):
    base = torch.empty((H, pitch_elems(W * 4, 2) // 4, 4), dtype=torch.int16, device=device)
    return base[:, :W, :]


def default_params(**kw) -> sn_params:
    p = sn_params()
    lib.sn_default_params(C.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def star_offsets(dirs: int, steps: int):
    import numpy as np
    ou = np.zeros(dirs * steps, np.int8)
    ov = np.zeros(dirs * steps, np.int8)
    n = lib.sn_star_offsets(dirs, steps, ou.ctypes.data_as(C.c_void_p), ov.ctypes.data_as(C.c_void_p))
    if n < 0:
        raise SnError(SN_EINVAL, "bad star-fill size")
    return ou.reshape(dirs, steps).astype(int), ov.reshape(dirs, steps).astype(int)


# ---------------------------------------------------------------- C ABI
def sn_create(cam, W: int, H: int, params: sn_params | None = None):
    c = sn_camera(cam.fx, cam.fy, cam.cx, cam.cy, cam.baseline)
    out = C.c_void_p()
    st = lib.sn_create(C.byref(c), W, H, C.byref(params) if params is not None else None, C.byref(out))
    _check(None, st)
    return out


def sn_destroy(ctx):
    lib.sn_destroy(ctx)


def sn_denoise(ctx, disp, den, mask, stream=None):
    d, dp = _img(disp)
    o, op = _img(den)
    m, mp = _img(mask)
    _check(ctx, lib.sn_denoise(ctx, d, dp, o, op, m, mp, _stream(stream)))


def sn_affine_normals(ctx, disp, den, normals, mask, stream=None):
    d, dp = _img(disp)
    e, ep = _img(den)
    n, np_ = _img(normals)
    m, mp = _img(mask)
    _check(ctx, lib.sn_affine_normals(ctx, d, dp, e, ep, n, np_, m, mp, _stream(stream)))


def sn_cross_normals(ctx, disp, normals, mask, stream=None):
    d, dp = _img(disp)
    n, np_ = _img(normals)
    m, mp = _img(mask)
    _check(ctx, lib.sn_cross_normals(ctx, d, dp, n, np_, m, mp, _stream(stream)))


def sn_pca_normals(ctx, disp, r, normals, mask, stream=None):
    d, dp = _img(disp)
    n, np_ = _img(normals)
    m, mp = _img(mask)
    _check(ctx, lib.sn_pca_normals(ctx, d, dp, int(r), n, np_, m, mp, _stream(stream)))


def sn_components(ctx, disp, labels, num_components=None, stream=None):
    d, dp = _img(disp)
    l, lp = _img(labels)
    nc = C.c_void_p(num_components.data_ptr()) if num_components is not None else None
    _check(ctx, lib.sn_components(ctx, d, dp, l, lp, nc, _stream(stream)))


def sn_pointcloud(ctx, den, mask, points, stream=None):
    e, ep = _img(den)
    m, mp = _img(mask)
    p, pp = _img(points)
    _check(ctx, lib.sn_pointcloud(ctx, e, ep, m, mp, p, pp, _stream(stream)))


def sn_run_frame(ctx, disp, normals, points, labels, mask, den=None, num_components=None, stream=None):
    fi = sn_frame_in()
    d, fi.disp_pitch = _img(disp)
    fi.disp = d
    fo = sn_frame_out()
    e, fo.den_pitch = _img(den)
    fo.den = e
    n, fo.normals_pitch = _img(normals)
    fo.normals = n
    p, fo.points_pitch = _img(points)
    fo.points = p
    l, fo.labels_pitch = _img(labels)
    fo.labels = l
    m, fo.mask_pitch = _img(mask)
    fo.mask = m
    fo.num_components = C.c_void_p(num_components.data_ptr()) if num_components is not None else None
    _check(ctx, lib.sn_run_frame(ctx, C.byref(fi), C.byref(fo), _stream(stream)))


def sn_run_frame_host(ctx, disp, normals, points, labels, mask, num_components=None, stream=None):
    """sn_run_frame on host (CPU) tensors, pinned for asynchronous copies;
    same layouts as sn_run_frame's device outputs."""
    for t in (disp, normals, points, labels, mask) + ((num_components,) if num_components is not None else ()):
        assert not t.is_cuda, "sn_run_frame_host takes host tensors"
    fi = sn_frame_in()
    d, fi.disp_pitch = _img(disp)
    fi.disp = d
    fo = sn_frame_out()
    n, fo.normals_pitch = _img(normals)
    fo.normals = n
    p, fo.points_pitch = _img(points)
    fo.points = p
    l, fo.labels_pitch = _img(labels)
    fo.labels = l
    m, fo.mask_pitch = _img(mask)
    fo.mask = m
    fo.num_components = C.c_void_p(num_components.data_ptr()) if num_components is not None else None
    _check(ctx, lib.sn_run_frame_host(ctx, C.byref(fi), C.byref(fo), _stream(stream)))


def sn_set_walk_limit(ctx, steps: int):
    _check(ctx, lib.sn_set_walk_limit(ctx, int(steps)))


def sn_check_device(ctx, stream=None):
    _check(ctx, lib.sn_check_device(ctx, _stream(stream)))


def sn_load_gate_weights(ctx, blob: bytes):
    buf = C.create_string_buffer(blob, len(blob))
    _check(ctx, lib.sn_load_gate_weights(ctx, C.cast(buf, C.c_void_p), len(blob)))


def sn_set_profiling(ctx, on: bool):
    _check(ctx, lib.sn_set_profiling(ctx, int(bool(on))))


def sn_stage_times(ctx, cap: int = 4096):
    """({stage name: summed ms}, frame count, [per-frame ms]) since the
    previous call."""
    n = lib.sn_stage_count(ctx)
    ms = (C.c_double * n)()
    fm = (C.c_double * cap)()
    frames = C.c_int()
    _check(ctx, lib.sn_stage_times(ctx, ms, n, C.byref(frames), fm, cap))
    nf = min(frames.value, cap)
    return ({lib.sn_stage_name(ctx, i).decode(): ms[i] for i in range(n)}, frames.value,
            [fm[i] for i in range(nf)])


def sn_launch_count(ctx) -> int:
    return int(lib.sn_launch_count(ctx))


def sn_normals_noalloc(cam, params, disp, normals, mask, stream=None):
    """Denoise + normals with the library's static device scratch (no
    allocation, no context).  `params` None = defaults."""
    c = sn_camera(cam.fx, cam.fy, cam.cx, cam.cy, cam.baseline)
    H, W = disp.shape[0], disp.shape[1]
    d, dp = _img(disp)
    n, np_ = _img(normals)
    m, mp = _img(mask)
    st = lib.sn_normals_noalloc(C.byref(c), C.byref(params) if params is not None else None, W, H,
                                d, dp, n, np_, m, mp, _stream(stream))
    _check(None, st)


def sn_gate_q(ctx, disp, q, stream=None):
    """The learned gate's probability map q [H, W] (float32) of a learned
    context with weights loaded."""
    d, dp = _img(disp)
    qq, qp = _img(q)
    _check(ctx, lib.sn_gate_q(ctx, d, dp, qq, qp, _stream(stream)))


def sn_gate_log2_table():
    """The device table of FP32 log2 of every code (numpy float32 [131072])."""
    import numpy as np
    out = np.empty(131072, np.float32)
    _check(None, lib.sn_gate_log2_table(out.ctypes.data_as(C.c_void_p), out.size))
    return out


def sn_rcp_table():
    """The kernels' FP32 reciprocal of every code (numpy float32 [131072], +inf at 0)."""
    import numpy as np
    out = np.empty(131072, np.float32)
    _check(None, lib.sn_rcp_table(out.ctypes.data_as(C.c_void_p), out.size))
    return out


def sn_noalloc_check_device(stream=None):
    """Reads and clears the allocation-free path's device error word after
    `stream` completes; raises SnError(SN_ETIMEOUT) if a bounded wait gave up."""
    _check(None, lib.sn_noalloc_check_device(_stream(stream)))
