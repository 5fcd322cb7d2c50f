"""Serving runtime (include/sn_serve.h) on the GPU.

* every result computed in a mix of cameras and resolutions (plain FP32,
  uint16 in / snorm16 out, and the learned FP16 chain), with several
  requests in flight on several streams, is bit-identical to the same frame
  run alone through sn_run_frame;
* admission: a camera whose slots are all held queues its requests and
  refuses (SN_EBUSY) beyond the queue depth; releasing a slot drains the queue;
* the simulated camera set of the serving workload (2x 640x480 at 120 Hz,
  4x 1482x994 at 30 Hz, 2x 2048x1024 at 30 Hz, Poisson arrivals) completes
  every request.
"""
import time

import numpy as np
import pytest
import torch

from scenes import make_scene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2504_15121_gb300 as P
    return P


def pinned(arr):
    a = np.ascontiguousarray(arr)
    t = torch.from_numpy(a.view(np.int16) if a.dtype == np.uint16 else a)
    return t.pin_memory()


def alone(P, scene, disp_np, **params):
    pipe = P.Pipeline(scene.camera, scene.W, scene.H, **params)
    try:
        d = pipe.upload(disp_np)
        out = pipe.buffers()
        pipe.run_frame(d, out, write_den=False)
        torch.cuda.synchronize()
        return dict(normals=out.normals.cpu().numpy(), points=out.points.cpu().numpy(),
                    labels=out.labels.cpu().numpy(), mask=out.mask.cpu().numpy(),
                    n_components=int(out.num_components.item()))
    finally:
        pipe.close()


def wait_results(srv, n, timeout=60.0):
    got = []
    t0 = time.time()
    while len(got) < n and time.time() - t0 < timeout:
        got += srv.poll()
        time.sleep(0.001)
    return got


def test_results_alone_equal_mixed(P):
    from paper_2504_15121_gb300 import serve
    specs = [("planes_640x480", {}), ("mixed_1482x994", {}),
             ("driving_2048x1024", dict(in_dtype=P.sn.SN_IN_U16X256, normal_fmt=P.sn.SN_NORMALS_SNORM16X4)),
             ("mixed_1482x994", dict(learned=1, in_dtype=P.sn.SN_IN_F16, normal_fmt=P.sn.SN_NORMALS_SNORM16X4))]
    frames = {}
    cams = []
    for ci, (name, params) in enumerate(specs):
        frames[ci] = [make_scene(name, frame=10 + k) for k in range(2)]
        s = frames[ci][0]
        cams.append(serve.camera(s.W, s.H, s.camera, **params))
    srv = serve.Server(cams, memory_budget=3 << 30, max_slots_per_camera=2, n_streams=3,
                       results_to_host=True, queue_depth=16)
    try:
        host = {}
        tag = 0
        for k in range(2):
            for ci, (name, params) in enumerate(specs):
                s = frames[ci][k]
                arr = s.disp_u16 if params.get("in_dtype") == P.sn.SN_IN_U16X256 else \
                    s.disp.astype(np.float16) if params.get("in_dtype") == P.sn.SN_IN_F16 else s.disp
                host[tag] = (ci, s, arr, params)
                assert srv.submit(ci, pinned(arr), tag) == P.sn.SN_OK
                tag += 1
        results = wait_results(srv, tag)
        assert len(results) == tag
        for r in results:
            ci, s, arr, params = host[r.tag]
            got = srv.result_arrays(r)
            want = alone(P, s, arr, **params)
            for key in ("normals", "points", "labels", "mask", "n_components"):
                assert np.array_equal(got[key], want[key]), (r.tag, key)
            assert r.latency_ms > 0
            srv.release(r.camera, r.slot)
        srv.check()
    finally:
        srv.close()


def test_admission_queue_and_backpressure(P):
    from paper_2504_15121_gb300 import serve
    s = make_scene("planes_320x240", frame=0)
    srv = serve.Server([serve.camera(s.W, s.H, s.camera)], memory_budget=1 << 30, max_slots_per_camera=1,
                       n_streams=1, results_to_host=True, queue_depth=2)
    try:
        assert srv.slots(0) == 1
        f = pinned(s.disp)
        assert srv.submit(0, f, 0) == P.sn.SN_OK
        first = wait_results(srv, 1)
        assert len(first) == 1                      # the only slot is now held
        codes = [srv.submit(0, f, 1 + i) for i in range(4)]
        assert codes[:2] == [P.sn.SN_OK, P.sn.SN_OK] and codes[2:] == [P.sn.SN_EBUSY] * 2
        time.sleep(0.05)
        assert srv.poll() == []                     # queued, not admitted
        srv.release(first[0].camera, first[0].slot)
        nxt = wait_results(srv, 1)
        assert [r.tag for r in nxt] == [1]
        srv.release(nxt[0].camera, nxt[0].slot)
        last = wait_results(srv, 1)
        assert [r.tag for r in last] == [2]
        srv.release(last[0].camera, last[0].slot)
        srv.check()
    finally:
        srv.close()


def serving_cameras(P, serve, **params):
    """The serving workload's camera set and pinned frame pools."""
    spec = [("planes_640x480", 120.0)] * 2 + [("mixed_1482x994", 30.0)] * 4 + [("driving_2048x1024", 30.0)] * 2
    scenes = {}
    cams, pools = [], []
    u16 = params.get("in_dtype") == P.sn.SN_IN_U16X256
    f16 = params.get("in_dtype") == P.sn.SN_IN_F16
    for ci, (name, rate) in enumerate(spec):
        if name not in scenes:
            scenes[name] = [make_scene(name, frame=20 + k) for k in range(2)]
        ss = scenes[name]
        cams.append(serve.camera(ss[0].W, ss[0].H, ss[0].camera, rate_hz=rate, **params))
        pick = (lambda s: s.disp_u16 if s.disp_u16 is not None else np.rint(s.disp * 256).astype(np.uint16)) if u16 \
            else (lambda s: s.disp.astype(np.float16)) if f16 else (lambda s: s.disp)
        pools.append([pinned(pick(s)) for s in ss])
    return cams, pools


def test_learned_camera_needs_weights(P):
    from paper_2504_15121_gb300 import serve
    s = make_scene("planes_320x240", frame=0)
    cam = serve.camera(s.W, s.H, s.camera, learned=1)
    cam.gate_weights = None
    cam.gate_weights_bytes = 0
    with pytest.raises(P.sn.SnError) as ei:
        serve.Server([cam], memory_budget=1 << 30, max_slots_per_camera=1, n_streams=1)
    assert ei.value.status == P.sn.SN_EINVAL


def test_simulated_camera_set(P):
    from paper_2504_15121_gb300 import serve
    cams, pools = serving_cameras(P, serve)
    srv = serve.Server(cams, memory_budget=4 << 30, max_slots_per_camera=4, n_streams=4, queue_depth=64)
    try:
        st = srv.simulate(pools, duration_s=1.5, rate_scale=1.0, seed=3)
        print(st)
        assert st["refused"] == 0 and st["completed"] == st["submitted"] > 500
        assert 0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
        srv.check()
    finally:
        srv.close()
