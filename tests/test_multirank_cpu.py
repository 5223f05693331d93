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


def _strong_worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    import oracle
    from paper_2509_06924_gb300 import shard
    from paper_2509_06924_gb300 import workloads as W
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        name, S = "uneven", 24
        mine = bench.rank_workload(name, rank, S, scaling="strong", world=world)
        full = W.make_workload(name, n_stacks=S)
        idx = shard.workload_partition(full, world)[rank]
        ll, g = oracle.batch("grad", mine.n_layers, mine.params, mine.dataset, mine.q_off, mine.q, mine.dq,
                             mine.r_obs, mine.r_err, mine.n_quad, n_threads=1)
        total = bench.sum_over_ranks(float(mine.evals), "cpu")
        gathered = [None] * world
        dist.all_gather_object(gathered, (idx.tolist(), ll.tolist(), g.tolist()))
        out.put((rank, total, gathered))
    finally:
        dist.destroy_process_group()


def test_two_rank_strong_split_reassembles_the_single_rank_result():
    """--scaling strong: the ranks' cost-balanced shares cover the batch once,
    the evaluation total is the batch's, and the shares' log-likelihoods and
    gradients, put back in stack order, equal one evaluation of the whole
    batch (the oracle stands in for the device path on CPU)."""
    import oracle
    from paper_2509_06924_gb300 import workloads as W
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_strong_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    full = W.make_workload("uneven", n_stacks=24)
    assert res[0][1] == res[1][1] == float(full.evals)
    gathered = res[0][2]
    ll = np.full(full.n_stacks, np.nan)
    g = np.full(full.params.size, np.nan)
    po = full.par_off
    seen = []
    for idx, l_r, g_r in gathered:
        seen += idx
        off = 0
        for j, s in enumerate(idx):
            ll[s] = l_r[j]
            n = po[s + 1] - po[s]
            g[po[s]:po[s + 1]] = g_r[off:off + n]
            off += n
    assert sorted(seen) == list(range(full.n_stacks))
    ll_ref, g_ref = oracle.batch("grad", full.n_layers, full.params, full.dataset, full.q_off, full.q, full.dq,
                                 full.r_obs, full.r_err, full.n_quad, n_threads=1)
    np.testing.assert_array_equal(ll, ll_ref)
    np.testing.assert_array_equal(g, g_ref)
