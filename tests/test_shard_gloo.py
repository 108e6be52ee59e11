"""Sharded listing on CPU ranks (gloo, world_size 2): each rank lists a
contiguous range of seed ranks of near-equal work, and a sum all-reduce of
(count, hash, probes) gives the full listing's values.  The listing on each
rank is the oracle (this is a test of the host-side split and combine; the
GPU ranks call tl_list_triangles_range with the same ranges)."""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_2203_04774_gb300 import shard, synth


def _graph():
    n = 3000
    e = synth.chung_lu(n, 14, 2.3, 77)
    off, _ = synth.simple_csr(n, e)
    return n, e, synth.order_degree(off)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n, e, rank_v = _graph()
        g = oracle.Graph(n, e)
        g.order_apply(rank_v)
        out_off, out_adj = g.csr(0)
        in_off, in_adj = g.csr(1)
        res = {}
        for alg in (oracle.APP, oracle.APM, oracle.AMM):
            work = shard.seed_work(out_off, out_adj, in_off, in_adj, alg)
            b, en = shard.balanced_ranges(work, world)[rank]
            _, c, h, p = g.list(alg, oracle.LITERAL, b, en, store=False)
            # the hash is summed mod 2^64: int64 addition wraps the same way
            t = torch.tensor([c, np.uint64(h).astype(np.int64), p, int(work[b:en].sum())],
                             dtype=torch.int64)
            dist.all_reduce(t, op=dist.ReduceOp.SUM)
            res[alg] = [int(v) for v in t]
        q.put((rank, res))
    finally:
        dist.destroy_process_group()


def test_seed_work_sums_to_cost_and_ranges_partition():
    n, e, r = _graph()
    g = oracle.Graph(n, e)
    g.order_apply(r)
    out_off, out_adj = g.csr(0)
    in_off, in_adj = g.csr(1)
    for alg in (oracle.APP, oracle.APM, oracle.AMM):
        w = shard.seed_work(out_off, out_adj, in_off, in_adj, alg)
        assert int(w.sum()) == g.cost(alg)  # Property 1, vertex by vertex summed
        for parts in (1, 2, 3, 7, 64):
            rg = shard.balanced_ranges(w, parts)
            assert rg[0][0] == 0 and rg[-1][1] == n
            assert all(rg[i][1] == rg[i + 1][0] for i in range(parts - 1))
            sums = [int(w[b:en].sum()) for b, en in rg]
            assert max(sums) <= int(w.sum()) / parts + int(w.max())
            # each range's probes are its work
            b, en = rg[parts // 2]
            assert g.list(alg, oracle.LITERAL, b, en, store=False)[3] == sums[parts // 2]


def test_two_gloo_ranks_combine_to_the_full_listing():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    n, e, r = _graph()
    g = oracle.Graph(n, e)
    g.order_apply(r)
    for alg in (oracle.APP, oracle.APM, oracle.AMM):
        _, c, h, p = g.list(alg, store=False)
        want = [c, int(np.uint64(h).astype(np.int64)), p, g.cost(alg)]
        assert out[0][alg] == want and out[1][alg] == want
        assert shard.combine([(c, h)]) == (c, h)


def test_balanced_ranges_edge_cases():
    # more parts than vertices, all-zero work, one heavy vertex: still a
    # partition of [0, n) into contiguous (possibly empty) ranges
    for work in (np.zeros(5, np.int64), np.array([0, 0, 100, 0], np.int64),
                 np.ones(3, np.int64), np.zeros(0, np.int64)):
        n = len(work)
        for parts in (1, 2, 7):
            rg = shard.balanced_ranges(work, parts)
            assert len(rg) == parts and rg[0][0] == 0 and rg[-1][1] == n
            assert all(b <= e for b, e in rg)
            assert all(rg[i][1] == rg[i + 1][0] for i in range(parts - 1))
            assert sum(int(work[b:e].sum()) for b, e in rg) == int(work.sum())
    with pytest.raises(ValueError):
        shard.balanced_ranges(np.ones(4), 0)
    # the combine wraps the hash sum mod 2^64
    assert shard.combine([(1, (1 << 64) - 1), (2, 5)]) == (3, 4)
