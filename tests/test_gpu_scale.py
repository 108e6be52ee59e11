"""Full-size listing of the largest configuration: Chung-Lu, n = 10^8 vertices,
exponent 2.2, average degree 40 (about 2 * 10^9 edges), seed 4, generated on
the device, in the launch configuration of the benchmark (1 GiB chunks, the
library's count + hash consumer).

Compared with the CPU oracle's listing of the same graph
(tests/golden/chunglu1e8.json, written by tests/golden/make_chunglu1e8.py
from oracle/ alone): the number of edges after cleaning, the triangle count
and the 64-bit set hash of A++ and A+- under the degree ordering, and the
costs C++ and C+- of that ordering, which by Property 1 are also the probe
counts.  The triangle set does not depend on the ordering, so the Split and
core orderings (computed on the device) must give the same count and hash.
Beside that, properties that hold at any size:
  * the membership tests performed equal C++ resp. C+- (Property 1);
  * a sample of listed triangles are triangles of the raw edge list (all
    three edges found in a sorted copy of the input), with a < b < c and no
    duplicates.
"""
import ctypes
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

N, AVG, GAMMA_EXP, SEED = 100_000_000, 40, 2.2, 4
CHUNK = 1 << 30
SAMPLE = 1 << 20
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "chunglu1e8.json")


def _golden():
    with open(GOLDEN) as f:
        d = json.load(f)
    assert (d["n"], d["avg_degree"], d["exponent"], d["seed"]) == (N, AVG, GAMMA_EXP, SEED)
    return d


@pytest.fixture(scope="module")
def env():
    import __graft_entry__
    __graft_entry__.build()
    import torch

    import paper_2203_04774_gb300 as tl
    torch.cuda.set_device(0)
    if torch.cuda.get_device_properties(0).total_memory < 200 * (1 << 30):
        pytest.skip("needs a GPU with >= 200 GiB")
    return tl, torch


def _list(tl, torch, g, alg, keep_sample=False):
    """List with the library's count + hash consumer; optionally copy the first
    SAMPLE triangles of chunk 0 to the device memory of a torch tensor."""
    ch = tl.CountHash()
    sample = []

    def consumer(ptr, n, idx, user):
        if keep_sample and idx == 0:
            k = min(n, SAMPLE)
            view = torch.as_tensor(tl._DevView(ptr, k), device="cuda")
            sample.append(view.clone())
        return tl.lib().tl_count_hash(ptr, n, idx, ctypes.cast(ch.user, ctypes.c_void_p))

    try:
        nt, probes = tl.tl_list_triangles_range(g, alg, 0, N, CHUNK, consumer, None)
        st = tl.tl_last_list_stats(g)
        return nt, int(ch.state.count), int(ch.state.hash), probes, st, (sample[0] if sample else None)
    finally:
        ch.release()


def test_chung_lu_1e8_vertices_2e9_edges(env):
    tl, torch = env
    from paper_2203_04774_gb300.synth import device as dev
    gold = _golden()
    want = (gold["triangles"], int(gold["hash"], 16))
    edges = dev.chung_lu_device(N, AVG, GAMMA_EXP, SEED)
    assert edges.shape[0] == gold["pairs"]
    g = tl.tl_graph_load(N, edges)
    try:
        n, m = tl.tl_graph_size(g)
        assert n == N and m == gold["m"]
        results = {}
        rank = torch.empty(N, dtype=torch.int32, device="cuda")
        tl.tl_order_compute(g, tl.TL_ORDER_DEGREE, rank)
        tl.tl_order_apply(g, rank)
        assert tl.tl_cost(g, tl.TL_APP) == gold["C_pp"]
        assert tl.tl_cost(g, tl.TL_APM) == gold["C_pm"]
        for alg in (tl.TL_APP, tl.TL_APM):
            nt, cnt, h, probes, st, smp = _list(tl, torch, g, alg, keep_sample=alg == tl.TL_APP)
            assert probes == tl.tl_cost(g, alg)  # Property 1
            assert nt == cnt and st["chunks"] > 1
            results[("degree", alg)] = (nt, h)
            if smp is not None:
                sample = smp
        for kind, name, alg in ((tl.TL_ORDER_SPLIT, "split", tl.TL_APM),
                                (tl.TL_ORDER_CORE, "core", tl.TL_APP)):
            tl.tl_order_compute(g, kind, rank)
            tl.tl_order_apply(g, rank)
            nt, cnt, h, probes, st, _ = _list(tl, torch, g, alg)
            assert probes == tl.tl_cost(g, alg)
            results[(name, alg)] = (nt, h)
        for key, got in results.items():
            assert got == want, (key, got, want)
    finally:
        tl.tl_graph_free(g)
        del rank
    # sampled triangles are triangles of the raw input
    s = sample.to(torch.int64)
    assert bool((s[:, 0] < s[:, 1]).all()) and bool((s[:, 1] < s[:, 2]).all())
    assert torch.unique(s, dim=0).shape[0] == s.shape[0]
    a, b = edges[:, 0].to(torch.int64), edges[:, 1].to(torch.int64)
    del edges
    keys = torch.minimum(a, b) * N + torch.maximum(a, b)
    del a, b
    keys, _ = torch.sort(keys)
    for i, j in ((0, 1), (0, 2), (1, 2)):
        q = s[:, i] * N + s[:, j]
        pos = torch.searchsorted(keys, q).clamp_(max=keys.numel() - 1)
        assert bool((keys[pos] == q).all()), (i, j)
