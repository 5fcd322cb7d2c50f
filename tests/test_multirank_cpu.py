"""Multi-rank host logic of bench.py on CPU: two gloo ranks, as torchrun
launches them for --gpus 2 (replicas only: frames are independent, so the
only cross-rank traffic is the barrier and the max-over-ranks time).

* the job time is the slowest rank's, on every rank;
* whole-job throughput counts every rank's pixels over that time;
* replicas render disjoint seeded frames;
* the reference arm does its work on rank 0 only.
"""
import os
import socket

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms = bench.max_over_ranks(10.0 + 3.0 * rank, dist)      # rank 1 is slower
        value = bench.whole_job_mpix(world, 1000000, ms)
        scenes = bench.make_inputs(1, rank)
        dist.barrier()
        q.put((rank, ms, value, float(np.asarray(scenes[0].disp, np.float64).sum())))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, ms0, v0, s0), (r1, ms1, v1, s1) = out
    assert ms0 == ms1 == 13.0                       # the slowest rank's time everywhere
    assert v0 == v1 == pytest.approx(2 * 1e6 / 0.013 / 1e6)
    assert s0 != s1                                 # disjoint frames


def test_single_process_has_no_reduction():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.5, None) == 7.5
    assert bench.whole_job_mpix(1, 2_097_152, 1000.0) == pytest.approx(2.097152)


def test_reference_arm_other_ranks_do_nothing(monkeypatch):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    args = bench.argparse.Namespace(steps=1, warmup=0, gpus=2)
    assert bench.run_reference(args) is None        # returns at once: no oracle work


def test_compare_at_equal_error_picks_fastest_as_accurate_plain():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    plain = {
        "fast_but_worse": {"value": 30000.0, "gt_error_deg": 20.0, "pixels": 1000},
        "accurate_slow": {"value": 2000.0, "gt_error_deg": 11.0, "pixels": 1000},
        "accurate_fast": {"value": 8000.0, "gt_error_deg": 12.0, "pixels": 995},
        "accurate_few_pixels": {"value": 50000.0, "gt_error_deg": 5.0, "pixels": 400},
    }
    r = bench.compare_at_equal_error(plain, 12000.0, 13.0, 1000)
    # the cheaper-but-worse setting and the one that drops most pixels do not count
    assert r["fastest_plain_as_accurate"] == "accurate_fast"
    assert r["vs_that_plain"] == pytest.approx(1.5)
    none = bench.compare_at_equal_error(plain, 12000.0, 1.0, 1000)
    assert none["fastest_plain_as_accurate"] is None and none["vs_that_plain"] is None
    # also near edges: only settings no worse there either
    for k, e in (("fast_but_worse", 30.0), ("accurate_slow", 9.0), ("accurate_fast", 25.0),
                 ("accurate_few_pixels", 1.0)):
        plain[k]["edge_band_error_deg"] = e
    r = bench.compare_at_equal_error(plain, 12000.0, 13.0, 1000, edge_err=10.0)
    assert r["fastest_plain_as_accurate"] == "accurate_fast"
    assert r["fastest_plain_as_accurate_also_near_edges"] == "accurate_slow"
    assert r["vs_that_plain_also_near_edges"] == pytest.approx(6.0)


def test_near_edge_band():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    prim = np.zeros((20, 30), np.int32)
    prim[:, 12:] = 1                       # one vertical edge between columns 11 and 12
    prim[15:, :] = 2                       # one horizontal edge between rows 14 and 15
    e = bench.near_edge(prim, 3)
    assert np.array_equal(np.where(e[0])[0], np.arange(8, 16))        # columns 11, 12 +- 3
    assert np.array_equal(np.where(e[:, 0])[0], np.arange(11, 19))    # rows 14, 15 +- 3
    assert not e[5, 0] and not e[5, 29]
