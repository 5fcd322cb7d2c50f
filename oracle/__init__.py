"""FP64 CPU oracle for the stereo surface-normal chain (test infrastructure).

Only the test suite, the package's smoke check and the benchmark's CPU
baseline may import this package.  The product (the CUDA library and its
binding) never imports, links or runs anything here, and this package
imports nothing from the product.

The arithmetic lives in ``sn_oracle.c`` (plain loops, FP64); this module only
builds it with gcc and marshals numpy arrays through ctypes.  Every function
returns dense arrays: [H, W] for scalars and [H, W, 3] for vectors.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sn_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "libsn_oracle.so")

F32, F16, U16X256 = 0, 1, 2
FIXED, STAR_CD, STAR_ST = 0, 1, 2
M_VALID, M_NORMAL, M_FP64, M_LEARNED, M_DENOISED = 1, 2, 4, 8, 16


class _Camera(C.Structure):
    _fields_ = [("fx", C.c_double), ("fy", C.c_double), ("cx", C.c_double),
                ("cy", C.c_double), ("baseline", C.c_double)]


class _Params(C.Structure):
    _fields_ = [("r_denoise", C.c_int), ("r_affine", C.c_int), ("support", C.c_int),
                ("dirs", C.c_int), ("steps", C.c_int), ("k_cd", C.c_double),
                ("k_pair", C.c_double), ("k_range", C.c_double), ("st_t", C.c_double)]


@dataclass
class Params:
    """Method parameters (defaults: 5x5 denoise, 9x9 fixed window, star-fill
    CD with 8 directions x 10 steps and k = 0.1, k_pair = k_range = 0.05)."""
    r_denoise: int = 2
    r_affine: int = 4
    support: int = STAR_CD
    dirs: int = 8
    steps: int = 10
    k_cd: float = 0.1
    k_pair: float = 0.05
    k_range: float = 0.05
    st_t: float = 0.1      # ST threshold on the depth Laplacian (metres)

    def c(self) -> _Params:
        return _Params(self.r_denoise, self.r_affine, self.support, self.dirs, self.steps,
                       self.k_cd, self.k_pair, self.k_range, self.st_t)


def build(force: bool = False) -> str:
    """Compile sn_oracle.c into a shared library (gcc, -O2, OpenMP)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        p = C.c_void_p
        L.orc_ingest.argtypes = [p, C.c_int, C.c_size_t, C.c_int, C.c_int, p]
        L.orc_ingest.restype = C.c_int
        L.orc_learned_radius.argtypes = []
        L.orc_learned_radius.restype = C.c_int
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_set_threads.restype = C.c_int
        L.orc_denoise.argtypes = [p, C.c_int, C.c_int, C.POINTER(_Params), p, p]
        L.orc_star_offsets.argtypes = [C.c_int, C.c_int, p, p]
        L.orc_star_offsets.restype = C.c_int
        L.orc_support_mask.argtypes = [p, C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(_Params), p, p]
        L.orc_st_edges.argtypes = [p, C.c_int, C.c_int, C.POINTER(_Camera), C.c_double, p]
        L.orc_st_edges.restype = None
        L.orc_support_mask.restype = C.c_int
        L.orc_affine_normals.argtypes = [p, p, C.c_int, C.c_int, C.POINTER(_Camera),
                                         C.POINTER(_Params), p, p, p]
        L.orc_components.argtypes = [p, C.c_int, C.c_int, C.POINTER(_Params), p]
        L.orc_components.restype = C.c_int
        L.orc_points.argtypes = [p, p, C.c_int, C.c_int, C.POINTER(_Camera), p]
        L.orc_run_frame.argtypes = [p, C.c_int, C.c_size_t, C.c_int, C.c_int, C.POINTER(_Camera),
                                    C.POINTER(_Params), p, p, p, p, p]
        L.orc_run_frame.restype = C.c_int
        L.orc_run_frame_gated.argtypes = [p, C.c_int, C.c_size_t, C.c_int, C.c_int, C.POINTER(_Camera),
                                          C.POINTER(_Params), p, p, p, p, p, p]
        L.orc_run_frame_gated.restype = C.c_int
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _cam(cam) -> _Camera:
    return _Camera(cam.fx, cam.fy, cam.cx, cam.cy, cam.baseline)


def _dtype_code(a: np.ndarray) -> int:
    if a.dtype == np.float32:
        return F32
    if a.dtype == np.float16:
        return F16
    if a.dtype == np.uint16:
        return U16X256
    raise TypeError(a.dtype)


def ingest(disp: np.ndarray) -> np.ndarray:
    """Integer disparity codes D = rint(256 d) (uint16 input: the raw code)."""
    disp = np.ascontiguousarray(disp)
    H, W = disp.shape
    D = np.zeros((H, W), np.int32)
    lib().orc_ingest(_ptr(disp), _dtype_code(disp), disp.strides[0], W, H, _ptr(D))
    return D


def denoise(D: np.ndarray, params: Params | None = None):
    """Denoised disparity d~ (px, FP64) and the 'fit determined' flags."""
    params = params or Params()
    D = np.ascontiguousarray(D, dtype=np.int32)
    H, W = D.shape
    den = np.zeros((H, W))
    ok = np.zeros((H, W), np.uint8)
    lib().orc_denoise(_ptr(D), W, H, C.byref(params.c()), _ptr(den), _ptr(ok))
    return den, ok


def star_offsets(dirs: int, steps: int):
    ou = np.zeros(dirs * steps, np.int32)
    ov = np.zeros(dirs * steps, np.int32)
    lib().orc_star_offsets(dirs, steps, _ptr(ou), _ptr(ov))
    return ou.reshape(dirs, steps), ov.reshape(dirs, steps)


def st_edges(D: np.ndarray, cam, t: float) -> np.ndarray:
    """ST edge map: |5-point depth Laplacian| > t (metres), or an invalid
    4-neighbour (Sec. III-D, simple thresholding)."""
    D = np.ascontiguousarray(D, dtype=np.int32)
    H, W = D.shape
    E = np.zeros((H, W), np.uint8)
    lib().orc_st_edges(_ptr(D), W, H, C.byref(_cam(cam)), float(t), _ptr(E))
    return E.astype(bool)


def support_mask(D: np.ndarray, u: int, v: int, params: Params | None = None, cam=None):
    """Boolean (2R+1)^2 grid of the offsets in the support of pixel (u, v)
    (the ST support needs the camera for its edge map)."""
    params = params or Params()
    D = np.ascontiguousarray(D, dtype=np.int32)
    H, W = D.shape
    R = params.r_affine if params.support == FIXED else params.steps
    incl = np.zeros((2 * R + 1, 2 * R + 1), np.uint8)
    E = np.ascontiguousarray(st_edges(D, cam, params.st_t), np.uint8) if params.support == STAR_ST else None
    lib().orc_support_mask(_ptr(D), W, H, u, v, C.byref(params.c()), _ptr(E) if E is not None else None,
                           _ptr(incl))
    return incl.astype(bool)


def affine_normals(D: np.ndarray, den: np.ndarray, cam, params: Params | None = None,
                   diag: bool = False):
    """Unit camera-facing normals [H, W, 3], mask [H, W] (and per-pixel
    diagnostics N, alpha, beta, gamma, det, g_u, g_v when diag=True)."""
    params = params or Params()
    D = np.ascontiguousarray(D, dtype=np.int32)
    den = np.ascontiguousarray(den, dtype=np.float64)
    H, W = D.shape
    nrm = np.zeros((H, W, 3))
    mask = np.zeros((H, W), np.uint8)
    dg = np.zeros((H, W, 8)) if diag else None
    lib().orc_affine_normals(_ptr(D), _ptr(den), W, H, C.byref(_cam(cam)), C.byref(params.c()),
                             _ptr(nrm), _ptr(mask), _ptr(dg) if diag else None)
    return (nrm, mask, dg) if diag else (nrm, mask)


def components(D: np.ndarray, params: Params | None = None):
    """Min-index component labels (int32, -1 invalid) and the component count."""
    params = params or Params()
    D = np.ascontiguousarray(D, dtype=np.int32)
    H, W = D.shape
    labels = np.zeros((H, W), np.int32)
    n = lib().orc_components(_ptr(D), W, H, C.byref(params.c()), _ptr(labels))
    return labels, n


def points(den: np.ndarray, mask: np.ndarray, cam):
    den = np.ascontiguousarray(den, dtype=np.float64)
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    H, W = den.shape
    pts = np.zeros((H, W, 3))
    lib().orc_points(_ptr(den), _ptr(mask), W, H, C.byref(_cam(cam)), _ptr(pts))
    return pts


@dataclass
class Frame:
    den: np.ndarray
    normals: np.ndarray
    points: np.ndarray
    labels: np.ndarray
    mask: np.ndarray
    n_components: int


def set_threads(n: int) -> int:
    """Threads of the oracle's parallel loops (n <= 0: unchanged); returns
    the count in effect."""
    return int(lib().orc_set_threads(int(n)))


def learned_radius() -> int:
    """Radius of the full window fitted at pixels the learned gate certifies."""
    return int(lib().orc_learned_radius())


def run_frame(disp: np.ndarray, cam, params: Params | None = None, gate=None) -> Frame:
    """The whole chain on one disparity map (float32, float16 or uint16 d*256).
    gate (bool [H, W], optional): the learned gate's decisions; certified
    pixels take the un-gated 5x5 denoise and the full (2 learned_radius() + 1)^2
    affine window."""
    params = params or Params()
    disp = np.ascontiguousarray(disp)
    H, W = disp.shape
    den = np.zeros((H, W))
    nrm = np.zeros((H, W, 3))
    pts = np.zeros((H, W, 3))
    labels = np.zeros((H, W), np.int32)
    mask = np.zeros((H, W), np.uint8)
    g = None if gate is None else np.ascontiguousarray(gate, np.uint8)
    n = lib().orc_run_frame_gated(_ptr(disp), _dtype_code(disp), disp.strides[0], W, H,
                                  C.byref(_cam(cam)), C.byref(params.c()),
                                  _ptr(g) if g is not None else None, _ptr(den), _ptr(nrm),
                                  _ptr(pts), _ptr(labels), _ptr(mask))
    return Frame(den, nrm, pts, labels, mask, n)
