"""Multi-rank timing logic of bench.py on CPU: two gloo ranks, each with its own timed
duration, agree on the slowest one, and the whole-job rate counts every rank's units."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as tmp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.max_over_ranks(1.0 + 2.0 * rank, dist, torch.device("cpu"))
    rate = bench.whole_job_rate(100, world, 4, t)
    out.put((rank, t, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [3.0, 3.0]
    assert all(abs(r[2] - 100 * 2 * 4 / 3.0) < 1e-12 for r in res)


def test_single_rank_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(2.5, None, None) == 2.5
    assert bench.whole_job_rate(10, 1, 3, 2.0) == 15.0


def test_level_traffic_record_matches_kernel_sources():
    """The stored ncu DRAM traffic of the level kernel is reported only for the kernel
    sources it was captured on and for launch shapes that have a capture."""
    sys.path.insert(0, ROOT)
    import bench
    import mch_inputs as mi
    wl = mi.workload(bench.WORKLOAD)
    rec = bench.LEVEL_TRAFFIC[bench.WORKLOAD]
    # the committed record belongs to the committed level-kernel sources
    assert rec["sha256_16"] == bench._sources_hash()
    shapes = [(wl.n_level(k + 1), v) for k, v in enumerate((2, 5, 9, 5))]
    mean, per = bench._level_traffic(wl, [v for _, v in shapes])
    assert per == [rec["bytes_per_launch"][s] for s in shapes]
    assert abs(mean - sum(per) / len(per)) < 1e-6
    # a shape without a capture gives no traffic
    assert bench._level_traffic(wl, [0, 0, 0, 0]) == (None, None)
    # another source hash (an edited kernel) gives none either
    saved = rec["sha256_16"]
    try:
        rec["sha256_16"] = "0" * 16
        assert bench._level_traffic(wl, [v for _, v in shapes]) == (None, None)
    finally:
        rec["sha256_16"] = saved
