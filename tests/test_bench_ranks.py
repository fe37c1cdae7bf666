"""bench.py's multi-rank aggregation on CPU with two gloo ranks: step times
are the slowest rank's (element-wise maximum), and the whole-job value is
the flops of all ranks over that time."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank-dependent times: rank 0 slower in the first, rank 1 in the second
        got = bench.max_over_ranks([3.0 - rank, 5.0 + 2 * rank], device="cpu")
        dist.barrier()
        out.put((rank, got, bench.whole_job_tflops(2.0e12, world, got[0])))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_max_over_ranks_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=240) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, value in res:
        assert got == [3.0, 7.0], (rank, got)
        # 2 ranks x 2e12 flops over the slowest rank's 3 ms
        assert value == pytest.approx(2 * 2.0e12 / 3.0e-3 / 1e12)


def test_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([1.5, 2.5], device="cpu") == [1.5, 2.5]
    assert bench.whole_job_tflops(1.0e12, 1, 1.0) == pytest.approx(1000.0)
