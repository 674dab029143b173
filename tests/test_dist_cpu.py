"""Multi-process host logic of bench.py on the CPU (gloo, world size 2): the
rendezvous, the barrier, the max-over-ranks timing, per-rank seeds and the
whole-job rate; the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import bench
    r, w, local = bench.dist_env()
    ok = bench.dist_init(w, "gloo")
    bench.barrier(ok)
    mx = bench.max_over_ranks(1.5 + r, ok)
    ref = bench.run_reference(type("A", (), {"steps": 1, "warmup": 0, "gpus": w})(), r, w) if r != 0 else None
    q.put((r, w, local, ok, mx, bench.rank_seed(r), ref, bench.rank_frames(1000, r, w)))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_rank_gloo_host_logic():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, l0, ok0, mx0, s0, _, f0), (r1, w1, l1, ok1, mx1, s1, ref1, f1) = out
    assert (r0, r1, w0, w1, l0, l1) == (0, 1, 2, 2, 0, 1)
    assert ok0 and ok1
    assert mx0 == mx1 == 2.5  # the slowest rank's time
    assert s0 != s1  # each rank draws its own frames
    assert ref1 is None  # only rank 0 runs the reference arm
    assert f0 == (0, 1000) and f1 == (1000, 2000)  # contiguous slices of one 2000-frame job


def test_whole_job_rate_is_weak_scaling():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.whole_job_rate(1000, 1, 0.5) == 2000
    assert bench.whole_job_rate(1000, 4, 0.5) == 8000


def test_frame_range_tiles_the_frames_once():
    sys.path.insert(0, ROOT)
    from paper_2204_13622_gb300 import binding
    for T, W in [(10, 3), (7, 7), (5, 8), (1 << 20, 8), (0, 2)]:
        ranges = [binding.frame_range(T, r, W) for r in range(W)]
        assert ranges[0][0] == 0 and ranges[-1][1] == T
        for (a0, a1), (b0, b1) in zip(ranges, ranges[1:]):
            assert a1 == b0 and a0 <= a1
        sizes = [b - a for a, b in ranges]
        assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        binding.frame_range(10, 2, 2)
