"""The multi-rank (torchrun) path of bench.py on CPU with the gloo backend,
world size 2: per-rank seeded shards of the workload (weak scaling), a
max-over-ranks timing reduction as the only collective, and rank-0-only
output of the reference arm."""
import io
import os
import contextlib
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        wl = bench.rank_workload("thick_oxide", rank, n_stacks=4)
        ms = bench.max_over_ranks(1.0 + rank, "cpu")
        # every rank sees the slowest rank's time
        buf = io.StringIO()
        with contextlib.redirect_stdout(buf):
            args = type("A", (), {"workload": "film_1l", "steps": 1, "warmup": 0})()
            if rank == 1:
                bench.run_reference(args)      # non-zero ranks print nothing
        out.put((rank, ms, wl.params[:10].tolist(), buf.getvalue()))
    finally:
        dist.destroy_process_group()


def test_two_rank_sharding_and_timing_reduction():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, ms0, p0, o0), (r1, ms1, p1, o1) = res
    assert ms0 == ms1 == 2.0
    assert not np.allclose(p0, p1)          # independent parameter samples per rank
    assert o1 == ""


def test_single_process_reduction_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, "cpu") == 3.5
