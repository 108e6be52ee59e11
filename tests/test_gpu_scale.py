"""Full-size listing of the largest configuration: Chung-Lu, n = 10^8 vertices,
exponent 2.2, average degree 40 (about 2 * 10^9 edges), seed 4, generated on
the device.

The oracle cannot hold this graph, so the CUDA path is checked through
properties that hold at any size, each computed by independent means:
  * A++ and A+- (different probe sets, different tiers) list the same number
    of triangles with the same order-free set hash;
  * so do two different orderings (degree and Split, both computed on the
    device), i.e. two different DAGs;
  * the membership tests performed equal C++ resp. C+- (Property 1);
  * a sample of listed triangles are triangles of the raw edge list (all
    three edges found in a sorted copy of the input), with a < b < c and no
    duplicates.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

N, AVG, GAMMA_EXP, SEED = 100_000_000, 40, 2.2, 4
CHUNK = 1 << 30
SAMPLE = 1 << 20


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
    edges = dev.chung_lu_device(N, AVG, GAMMA_EXP, SEED)
    g = tl.tl_graph_load(N, edges)
    try:
        n, m = tl.tl_graph_size(g)
        assert n == N and 1.5e9 < m <= edges.shape[0]
        results = {}
        rank = torch.empty(N, dtype=torch.int32, device="cuda")
        tl.tl_order_compute(g, tl.TL_ORDER_DEGREE, rank)
        tl.tl_order_apply(g, rank)
        for alg in (tl.TL_APP, tl.TL_APM):
            nt, cnt, h, probes, st, smp = _list(tl, torch, g, alg, keep_sample=alg == tl.TL_APP)
            assert probes == tl.tl_cost(g, alg)  # Property 1
            assert nt == cnt and st["chunks"] > 1
            results[("degree", alg)] = (nt, h)
            if smp is not None:
                sample = smp
        tl.tl_order_compute(g, tl.TL_ORDER_SPLIT, rank)
        tl.tl_order_apply(g, rank)
        nt, cnt, h, probes, st, _ = _list(tl, torch, g, tl.TL_APM)
        assert probes == tl.tl_cost(g, tl.TL_APM)
        results[("split", tl.TL_APM)] = (nt, h)
        assert len(set(results.values())) == 1, results
        assert results[("degree", tl.TL_APP)][0] > 1e9
    finally:
        tl.tl_graph_free(g)
        del rank
    # sampled triangles are triangles of the raw input
    s = sample.to(torch.int64)
    assert bool((s[:, 0] < s[:, 1]).all()) and bool((s[:, 1] < s[:, 2]).all())
    key = s[:, 0] * N * N + s[:, 1] * N + s[:, 2]
    assert torch.unique(key).numel() == s.shape[0]
    a, b = edges[:, 0].to(torch.int64), edges[:, 1].to(torch.int64)
    del edges
    keys = torch.minimum(a, b) * N + torch.maximum(a, b)
    del a, b
    keys, _ = torch.sort(keys)
    for i, j in ((0, 1), (0, 2), (1, 2)):
        q = s[:, i] * N + s[:, j]
        pos = torch.searchsorted(keys, q).clamp_(max=keys.numel() - 1)
        assert bool((keys[pos] == q).all()), (i, j)
