"""The N > 1 bench path on CPU: two gloo ranks (one process each) check the whole-job reduction
the GPU ranks use -- independent replica content per rank, the slowest rank's time, and the job
rate over all ranks' frames."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        local = [1.5, 2.5][rank]                     # the ranks' own timed seconds
        slow = bench.max_over_ranks(local, world, device="cpu")
        rate = bench.job_rate(10, world, 1920 * 1080, slow)
        seeds = [None] * world
        dist.all_gather_object(seeds, bench.replica_seed(rank))
        out.put((rank, slow, rate, seeds))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_like_the_gpu_bench():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slow, rate, seeds in res:
        assert slow == 2.5                            # both ranks agree on the slowest time
        assert abs(rate - 10 * 2 * 1920 * 1080 / 2.5 / 1e6) < 1e-9
        assert len(set(seeds)) == 2                   # independent replicas


def test_single_rank_is_the_identity():
    import bench
    assert bench.max_over_ranks(3.25, 1) == 3.25
    assert bench.job_rate(4, 1, 100, 2.0) == 4 * 100 / 2.0 / 1e6
