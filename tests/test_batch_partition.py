"""Splitting a batch of independent products over GPUs (fmm_batch_partition):
longest-processing-time by flops.  Host logic, checked on CPU: a partition
of all products, deterministic, the largest share within the LPT bound of
the best possible (brute force on small batches), and two gloo ranks that
each compute it on their own agree on the assignment and each take the
products of their own part."""
import itertools
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def api():
    sys.path.insert(0, ROOT)
    from paper_1507_00687_gb300 import build
    build.build()
    from paper_1507_00687_gb300 import api as A
    return A


def _flops(d):
    return [2.0 * m * k * n for m, k, n in d]


def test_partition_covers_every_product_once_and_is_deterministic(api):
    from paper_1507_00687_gb300 import inputs
    dims = inputs.log_uniform_dims(512, 512, 4096, 128, seed=1507 + 4000).tolist()
    for parts in (1, 2, 3, 8):
        p = api.partition_batch(dims, parts)
        assert len(p) == parts
        allidx = sorted(i for part in p for i in part)
        assert allidx == list(range(len(dims)))
        assert p == api.partition_batch(dims, parts)
        f = _flops(dims)
        loads = [sum(f[i] for i in part) for part in p]
        # LPT: the largest share exceeds the mean by at most the largest product
        assert max(loads) <= sum(f) / parts + max(f) + 1e-6


def test_partition_within_lpt_bound_of_optimum(api):
    g = np.random.default_rng(5)
    for trial in range(30):
        n = int(g.integers(3, 10))
        dims = [tuple(int(x) for x in g.integers(1, 9, size=3) * 128) for _ in range(n)]
        f = _flops(dims)
        for parts in (2, 3):
            p = api.partition_batch(dims, parts)
            lpt = max(sum(f[i] for i in part) for part in p)
            best = min(max(sum(f[i] for i in range(n) if a[i] == q) for q in range(parts))
                       for a in itertools.product(range(parts), repeat=n))
            assert lpt <= (4.0 / 3.0 - 1.0 / (3 * parts)) * best + 1e-6, (dims, parts)


def test_partition_order_and_ties(api):
    # Longest processing time first, equal flop counts in index order, each
    # product to the least-loaded part with ties to the lowest part: four
    # equal products alternate 0, 1, 0, 1; a large product goes first and
    # alone, the small ones then fill the other part before sharing.
    assert api.partition_batch([(256, 256, 256)] * 4, 2) == [[0, 2], [1, 3]]
    assert api.partition_batch([(256, 256, 256)] * 3, 3) == [[0], [1], [2]]
    dims = [(128, 128, 128), (512, 512, 512), (128, 128, 128), (128, 128, 128)]
    assert api.partition_batch(dims, 2) == [[1], [0, 2, 3]]


def test_partition_rejects_bad_arguments(api):
    from paper_1507_00687_gb300 import _native as N
    import ctypes as C
    assert N.lib().fmm_batch_partition(None, None, None, 3, 2, None) == 1
    z = (C.c_int64 * 1)(4)
    out = (C.c_int32 * 1)()
    assert N.lib().fmm_batch_partition(z, z, z, 1, 0, out) == 1
    assert N.lib().fmm_batch_partition(z, z, z, 1, 1, out) == 0 and out[0] == 0


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    from paper_1507_00687_gb300 import api, inputs
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dims = inputs.log_uniform_dims(64, 512, 4096, 128, seed=77).tolist()
        mine = api.partition_batch(dims, world)[rank]
        # every rank's own view of the whole assignment, gathered for comparison
        views = [None] * world
        dist.all_gather_object(views, (rank, api.partition_batch(dims, world), mine))
        mine_flops = torch.tensor([sum(2.0 * m * k * n for m, k, n in (dims[i] for i in mine))], dtype=torch.float64)
        total = mine_flops.clone()
        dist.all_reduce(total)
        out.put((rank, views, float(mine_flops), float(total)))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_gloo_ranks_agree_on_the_split():
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
    (_, views0, f0, total), (_, views1, f1, total1) = res
    assert views0 == views1  # both ranks hold the same assignment
    (r0, full0, mine0), (r1, full1, mine1) = views0
    assert full0 == full1 and mine0 == full0[0] and mine1 == full0[1]
    assert not set(mine0) & set(mine1) and len(mine0) + len(mine1) == 64
    assert total == total1 == f0 + f1
