"""ctypes binding of the serving runtime (include/sn_serve.h), same names as
the C ABI, plus a small `Server` holder.  Argument marshalling only: the
scheduler, slots, graphs and streams live in libsn.so."""
from __future__ import annotations

import ctypes as C

import numpy as np

from .sn import SnError, lib, sn_camera, sn_params, default_params, SN_OK


class sn_server_camera(C.Structure):
    _fields_ = [("W", C.c_int), ("H", C.c_int), ("cam", sn_camera), ("params", sn_params),
                ("rate_hz", C.c_double), ("gate_weights", C.c_void_p), ("gate_weights_bytes", C.c_size_t)]


class sn_server_config(C.Structure):
    _fields_ = [("n_cameras", C.c_int), ("cameras", C.POINTER(sn_server_camera)),
                ("memory_budget", C.c_size_t), ("max_slots_per_camera", C.c_int),
                ("n_streams", C.c_int), ("results_to_host", C.c_int), ("queue_depth", C.c_int)]


class sn_serve_result(C.Structure):
    _fields_ = [("tag", C.c_uint64), ("camera", C.c_int), ("slot", C.c_int), ("latency_ms", C.c_double),
                ("normals", C.c_void_p), ("points", C.c_void_p), ("labels", C.c_void_p),
                ("mask", C.c_void_p), ("num_components", C.c_int32)]


class sn_serve_sim(C.Structure):
    _fields_ = [("duration_s", C.c_double), ("rate_scale", C.c_double), ("seed", C.c_uint64),
                ("frames", C.POINTER(C.c_void_p)), ("pool_size", C.POINTER(C.c_int)),
                ("max_pool", C.c_int), ("frame_pitch", C.POINTER(C.c_size_t))]


class sn_serve_stats(C.Structure):
    _fields_ = [("offered_mpix_s", C.c_double), ("sustained_mpix_s", C.c_double),
                ("p50_ms", C.c_double), ("p99_ms", C.c_double), ("max_ms", C.c_double),
                ("submitted", C.c_longlong), ("completed", C.c_longlong), ("refused", C.c_longlong),
                ("wall_s", C.c_double)]


_vp = C.c_void_p
for _name, _args, _res in [
        ("sn_server_create", [C.POINTER(sn_server_config), C.POINTER(_vp)], C.c_int),
        ("sn_server_destroy", [_vp], C.c_int),
        ("sn_server_slots", [_vp, C.c_int], C.c_int),
        ("sn_server_submit", [_vp, C.c_int, _vp, C.c_size_t, C.c_uint64], C.c_int),
        ("sn_server_poll", [_vp, C.POINTER(sn_serve_result), C.c_int], C.c_int),
        ("sn_server_release", [_vp, C.c_int, C.c_int], C.c_int),
        ("sn_server_simulate", [_vp, C.POINTER(sn_serve_sim), C.POINTER(sn_serve_stats)], C.c_int),
        ("sn_server_check", [_vp], C.c_int)]:
    _f = getattr(lib, _name)
    _f.argtypes = _args
    _f.restype = _res

EXPORTS = ("sn_server_create", "sn_server_destroy", "sn_server_slots", "sn_server_submit",
           "sn_server_poll", "sn_server_release", "sn_server_simulate", "sn_server_check")


def _check(st, what):
    if st != SN_OK:
        raise SnError(st, what)


_weight_buffers = []   # gate-weight blobs handed to servers (kept alive for the process)


def camera(W, H, cam, rate_hz=0.0, gate_weights=None, **params) -> sn_server_camera:
    """One camera of a server.  learned=1 attaches the gate weights
    (gate_weights: path or bytes; default: the packaged trained weights)."""
    p = default_params(**params)
    ptr, size = None, 0
    if p.learned:
        from . import gate
        blob = gate_weights if isinstance(gate_weights, (bytes, bytearray)) else \
            open(gate_weights or gate.DEFAULT_WEIGHTS, "rb").read()
        buf = C.create_string_buffer(bytes(blob), len(blob))
        _weight_buffers.append(buf)
        ptr, size = C.cast(buf, C.c_void_p), len(blob)
    return sn_server_camera(W, H, sn_camera(cam.fx, cam.fy, cam.cx, cam.cy, cam.baseline), p, rate_hz, ptr, size)


class Server:
    """Owns one sn_server.  `frames` (simulation pools) must be pinned host
    arrays that outlive the server's use of them."""

    def __init__(self, cameras, memory_budget=2 << 30, max_slots_per_camera=4, n_streams=4,
                 results_to_host=False, queue_depth=64):
        self._cams = (sn_server_camera * len(cameras))(*cameras)
        cfg = sn_server_config(len(cameras), self._cams, memory_budget, max_slots_per_camera,
                               n_streams, int(results_to_host), queue_depth)
        self.handle = _vp()
        _check(lib.sn_server_create(C.byref(cfg), C.byref(self.handle)), "sn_server_create")
        self.cameras = cameras
        self.results_to_host = results_to_host
        self._keep = []

    def close(self):
        if self.handle:
            lib.sn_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def slots(self, cam: int) -> int:
        return lib.sn_server_slots(self.handle, cam)

    def submit(self, cam: int, host_frame, tag: int) -> int:
        """host_frame: a pinned torch tensor [H, W] (kept alive here until polled)."""
        self._keep.append(host_frame)
        return lib.sn_server_submit(self.handle, cam, _vp(host_frame.data_ptr()),
                                    host_frame.stride(0) * host_frame.element_size(), tag)

    def poll(self, max_results: int = 64):
        buf = (sn_serve_result * max_results)()
        n = lib.sn_server_poll(self.handle, buf, max_results)
        return [buf[i] for i in range(n)]

    def release(self, cam: int, slot: int):
        _check(lib.sn_server_release(self.handle, cam, slot), "sn_server_release")

    def result_arrays(self, r: sn_serve_result):
        """Copies of a polled result's host outputs (results_to_host only)."""
        cam = self.cameras[r.camera]
        W, H = cam.W, cam.H
        snorm = cam.params.normal_fmt == 1

        def arr(ptr, ctype, count):
            return np.ctypeslib.as_array(C.cast(ptr, C.POINTER(ctype)), shape=(count,)).copy()
        if snorm:
            nrm = arr(r.normals, C.c_int16, H * W * 4).reshape(H, W, 4)
        else:
            nrm = arr(r.normals, C.c_float, 3 * H * W).reshape(3, H, W)
        pts = arr(r.points, C.c_float, 3 * H * W).reshape(3, H, W)
        lab = arr(r.labels, C.c_int32, H * W).reshape(H, W)
        msk = arr(r.mask, C.c_uint8, H * W).reshape(H, W)
        return dict(normals=nrm, points=pts, labels=lab, mask=msk, n_components=int(r.num_components))

    def simulate(self, pools, duration_s, rate_scale=1.0, seed=0) -> dict:
        """pools: per camera a list of pinned torch tensors [H, W]."""
        max_pool = max(len(p) for p in pools)
        frames = (_vp * (len(pools) * max_pool))()
        for c, pool in enumerate(pools):
            for i, t in enumerate(pool):
                frames[c * max_pool + i] = t.data_ptr()
        sizes = (C.c_int * len(pools))(*[len(p) for p in pools])
        pitches = (C.c_size_t * len(pools))(*[p[0].stride(0) * p[0].element_size() for p in pools])
        sim = sn_serve_sim(duration_s, rate_scale, seed, frames, sizes, max_pool, pitches)
        st = sn_serve_stats()
        _check(lib.sn_server_simulate(self.handle, C.byref(sim), C.byref(st)), "sn_server_simulate")
        return {k: getattr(st, k) for k, _ in sn_serve_stats._fields_}

    def check(self):
        _check(lib.sn_server_check(self.handle), "sn_server_check")
