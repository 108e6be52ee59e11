"""Disjoint unions (batched listing) vs the CPU oracle run on each graph alone.

A union of k graphs must list, for every part, exactly the triangles that part
has alone under its own ordering (no edge joins two parts), with the part's
costs and probe counts; tl_count_hash_parts must give each part the (count,
hash) of the graph alone.  Every call goes through the C ABI.
"""
import numpy as np
import pytest

import oracle
import paper_2203_04774_gb300 as tl
from paper_2203_04774_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    torch.cuda.set_device(0)


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _wheel(k):
    spokes = np.stack([np.zeros(k, np.uint32), np.arange(1, k + 1, dtype=np.uint32)], 1)
    rim = np.stack([np.arange(1, k + 1, dtype=np.uint32),
                    np.r_[np.arange(2, k + 1), 1].astype(np.uint32)], 1)
    return k + 1, np.concatenate([spokes, rim])


def _parts_small():
    """(n, edges) of assorted small graphs, including degenerate ones."""
    dup = np.array([[0, 1], [1, 0], [1, 2], [2, 2], [2, 0], [0, 2], [3, 3], [2, 3], [3, 1]],
                   np.uint32)
    return [
        (5, synth.complete(5)),
        (300, synth.chung_lu(300, 10, 2.5, 7)),
        (50, synth.gnp(50, 0.2, 3)),
        (1, np.zeros((0, 2), np.uint32)),          # a single vertex
        (21, synth.star(21)),                       # triangle-free
        (10, np.zeros((0, 2), np.uint32)),          # no edges
        (4, dup),                                   # loops, duplicates, both directions
        (9, synth.complete_bipartite(4, 5)),        # triangle-free
        (30, synth.complete(30)),                   # T = C(30, 3) = 4060
        (7, synth.fig3_graph()),
    ]


def _vbase(sizes):
    vb = np.zeros(len(sizes) + 1, np.int64)
    np.cumsum(sizes, out=vb[1:])
    return vb


def _demux(t, vb):
    """Union triples -> list of per-part canonical triple arrays with local ids."""
    t = np.asarray(t, np.int64).reshape(-1, 3)
    p = np.searchsorted(vb, t[:, 0], side="right") - 1
    assert np.all(np.searchsorted(vb, t[:, 2], side="right") - 1 == p), "a triple spans parts"
    return [oracle.canonical((t[p == i] - vb[i]).astype(np.uint32)) for i in range(len(vb) - 1)]


def _check_union(u, parts, ranks, algs_by_part, chunk_bytes=tl.TL_MIN_CHUNK_BYTES):
    """List the union (one range per run of equal algorithms) and compare every
    part with the oracle on that graph alone under the same local ordering."""
    sizes = [n for n, _ in parts]
    vb = _vbase(sizes)
    refs = []
    for (n, e), r in zip(parts, ranks):
        ref = oracle.Graph(n, e)
        ref.order_apply(r)
        refs.append(ref)
    for alg in (tl.TL_APP, tl.TL_APM, tl.TL_AMM):
        assert u.cost(alg) == sum(ref.cost(alg) for ref in refs)
    # runs of consecutive parts with the same algorithm -> one range call each
    runs, i = [], 0
    while i < len(parts):
        j = i
        while j < len(parts) and algs_by_part[j] == algs_by_part[i]:
            j += 1
        runs.append((i, j, algs_by_part[i]))
        i = j
    got = [None] * len(parts)
    counts = np.zeros(len(parts), np.uint64)
    hashes = np.zeros(len(parts), np.uint64)
    for i, j, alg in runs:
        t, nt, probes, _ = u.list_collect(alg, chunk_bytes, int(vb[i]), int(vb[j]))
        assert nt == len(t)
        assert probes == sum(refs[q].cost(alg) for q in range(i, j))  # Property 1, per part
        per = _demux(t, vb)
        for q in range(len(parts)):
            if i <= q < j:
                got[q] = per[q]
            else:
                assert len(per[q]) == 0
        nt2, c, h, probes2 = u.list_count_hash_parts(alg, sizes, chunk_bytes, int(vb[i]),
                                                     int(vb[j]))
        assert (nt2, probes2) == (nt, probes)
        counts[i:j] = c[i:j]
        hashes[i:j] = h[i:j]
        assert not np.any(c[:i]) and not np.any(c[j:])
    for q, ref in enumerate(refs):
        rt, rc, rh, rp = ref.list(algs_by_part[q])
        assert np.array_equal(got[q], oracle.canonical(rt)), q
        assert (int(counts[q]), int(hashes[q])) == (rc, rh), q


def test_load_parts_identity_and_degree_orderings():
    parts = _parts_small()
    sizes = [n for n, _ in parts]
    ms = [len(e) for _, e in parts]
    e_all = np.concatenate([e for _, e in parts]).astype(np.uint32)
    u = tl.Graph.load_parts(sizes, ms, _dev(e_all))
    assert u.n == sum(sizes)
    assert u.m == sum(oracle.Graph(n, e).m for n, e in parts)
    ident = [synth.order_identity(n) for n in sizes]
    for alg in (tl.TL_APP, tl.TL_APM, tl.TL_AMM):
        _check_union(u, parts, ident, [alg] * len(parts))
    # device orderings of a union are computed part by part
    vb = _vbase(sizes)
    for kind, host in ((tl.TL_ORDER_DEGREE, lambda n, e, off: synth.order_degree(off)),
                       (tl.TL_ORDER_SPLIT, lambda n, e, off: synth.order_split(off)),
                       (tl.TL_ORDER_CORE, lambda n, e, off: oracle.core_order_levels(n, e))):
        rank_u = u.order_compute(kind).cpu().numpy().astype(np.int64)
        local = []
        for i, (n, e) in enumerate(parts):
            off, _ = synth.simple_csr(n, e)
            r = rank_u[vb[i]:vb[i + 1]] - vb[i]
            assert np.array_equal(r, host(n, e, off)), (kind, i)
            local.append(r.astype(np.uint32))
        u.order_apply(_dev(rank_u.astype(np.uint32)))
        _check_union(u, parts, local, [tl.TL_APP] * 5 + [tl.TL_APM] * 5)
    u.free()


def test_load_parts_host_edges():
    parts = _parts_small()
    sizes = [n for n, _ in parts]
    e_all = np.concatenate([e for _, e in parts]).astype(np.uint32)
    u = tl.Graph.load_parts(sizes, [len(e) for _, e in parts], e_all)  # host pointer
    ident = [synth.order_identity(n) for n in sizes]
    _check_union(u, parts, ident, [tl.TL_APM] * len(parts))
    u.free()


def test_union_of_loaded_graphs_each_with_its_own_ordering():
    parts = _parts_small()
    graphs = [tl.Graph(n, _dev(e)) for n, e in parts]
    kinds = ["random", "degree", "core", "identity", "degree", "random", "core", "split",
             "random", "check"]
    ranks = []
    for (n, e), kind in zip(parts, kinds):
        off, adj = synth.simple_csr(n, e)
        ranks.append({"random": lambda: synth.order_random(n, 5),
                      "degree": lambda: synth.order_degree(off),
                      "core": lambda: synth.order_core(off, adj),
                      "identity": lambda: synth.order_identity(n),
                      "split": lambda: synth.order_split(off),
                      "check": lambda: synth.order_check(off, adj)}[kind]())
    # explicit ranks
    u = tl.Graph.union(graphs, [_dev(r) for r in ranks])
    algs = [tl.TL_APP, tl.TL_APM] * 5
    _check_union(u, parts, ranks, algs)
    u.free()
    # current orderings: apply to half of the graphs, the rest stay on the identity
    for i in range(0, len(graphs), 2):
        graphs[i].order_apply(_dev(ranks[i]))
    cur = [ranks[i] if i % 2 == 0 else synth.order_identity(parts[i][0])
           for i in range(len(parts))]
    u = tl.Graph.union(graphs)
    _check_union(u, parts, cur, [tl.TL_APP] * len(parts))
    u.free()
    # mixing explicit and current (None) entries
    mixed = [_dev(ranks[i]) if i % 3 == 0 else None for i in range(len(parts))]
    want = [ranks[i] if i % 3 == 0 else cur[i] for i in range(len(parts))]
    u = tl.Graph.union(graphs, mixed)
    _check_union(u, parts, want, [tl.TL_APM] * len(parts))
    u.free()
    for g in graphs:
        g.free()


def test_union_each_part_same_alone_and_in_the_mix():
    """The batched result of every part equals the library's own result for
    that graph listed alone, and the oracle's."""
    rng = np.random.default_rng(9)
    parts = []
    for i in range(40):
        n = int(rng.integers(50, 3000))
        parts.append((n, synth.chung_lu(n, float(rng.uniform(4, 30)),
                                        float(rng.uniform(2.1, 3.0)), 1000 + i)))
    graphs = [tl.Graph(n, _dev(e)) for n, e in parts]
    ranks = [g.order_compute(tl.TL_ORDER_DEGREE) for g in graphs]
    algs = [tl.TL_APP if i % 3 else tl.TL_APM for i in range(len(parts))]
    order = np.argsort(algs, kind="stable")  # A++ parts first, then A+-
    graphs_o = [graphs[i] for i in order]
    u = tl.Graph.union(graphs_o, [ranks[i] for i in order])
    sizes = [parts[i][0] for i in order]
    vb = _vbase(sizes)
    n_app = int(np.sum(np.array(algs) == tl.TL_APP))
    c = np.zeros(len(parts), np.uint64)
    h = np.zeros(len(parts), np.uint64)
    for alg, i, j in ((tl.TL_APP, 0, n_app), (tl.TL_APM, n_app, len(parts))):
        _, cc, hh, _ = u.list_count_hash_parts(alg, sizes, x_begin=int(vb[i]),
                                               x_end=int(vb[j]))
        c[i:j], h[i:j] = cc[i:j], hh[i:j]
    for pos, i in enumerate(order):
        g = graphs[i]
        g.order_apply(ranks[i])
        nt, cnt, hsh, _ = g.list_count_hash(algs[i])
        assert (int(c[pos]), int(h[pos])) == (cnt, hsh), i
        ref = oracle.Graph(*parts[i])
        ref.order_apply(ranks[i].cpu().numpy())
        _, rc, rh, _ = ref.list(algs[i], store=False)
        assert (cnt, hsh) == (rc, rh), i
    u.free()
    for g in graphs:
        g.free()


def test_union_many_parts_every_tier():
    """Hundreds of parts of uneven size; a wheel (hub of degree 5000) and a
    60,000-vertex power-law part bring tasks to the mid and large listing
    kernels: per-part (count, hash) vs the oracle."""
    rng = np.random.default_rng(4)
    parts = []
    for i in range(300):
        n = int(np.exp(rng.uniform(np.log(20), np.log(4000))))
        parts.append((n, synth.chung_lu(n, float(rng.uniform(4, 40)),
                                        float(rng.uniform(2.1, 3.0)), 2000 + i)))
    parts.insert(17, _wheel(5000))
    parts.insert(200, (60000, synth.chung_lu(60000, 24, 2.1, 21)))
    sizes = [n for n, _ in parts]
    e_all = np.concatenate([e for _, e in parts]).astype(np.uint32)
    u = tl.Graph.load_parts(sizes, [len(e) for _, e in parts], _dev(e_all))
    rank_u = u.order_compute(tl.TL_ORDER_DEGREE)
    u.order_apply(rank_u)
    vb = _vbase(sizes)
    rank_np = rank_u.cpu().numpy().astype(np.int64)
    seen = np.zeros(tl.TL_KERNELS, np.int64)
    for alg in (tl.TL_APP, tl.TL_APM, tl.TL_AMM):
        nt, c, h, probes = u.list_count_hash_parts(alg, sizes)
        seen += np.array(tl.tl_last_list_stats(u.h)["tasks"]) > 0
        tot_probes = 0
        for i, (n, e) in enumerate(parts):
            ref = oracle.Graph(n, e)
            ref.order_apply((rank_np[vb[i]:vb[i + 1]] - vb[i]).astype(np.uint32))
            _, rc, rh, rp = ref.list(alg, store=False)
            assert (int(c[i]), int(h[i])) == (rc, rh), (alg, i)
            tot_probes += rp
        assert probes == tot_probes and nt == int(c.sum())
    assert np.all(seen > 0), seen
    u.free()


def test_union_invalid_inputs():
    with pytest.raises(tl.TLError) as ei:
        tl.Graph.load_parts([3, 2], [1, 1], _dev(np.array([[0, 2], [0, 2]], np.uint32)))
    assert ei.value.status == tl.TL_EINVAL  # id 2 >= n of part 1
    with pytest.raises(tl.TLError) as ei:
        tl.Graph.load_parts([3, 0], [1, 0], _dev(np.array([[0, 2]], np.uint32)))
    assert ei.value.status == tl.TL_EINVAL  # empty part
    a = tl.Graph(4, _dev(synth.complete(4)))
    b = tl.Graph(3, _dev(synth.complete(3)))
    bad = _dev(np.array([0, 1, 3], np.uint32))  # not a permutation of [0, 3)
    with pytest.raises(tl.TLError) as ei:
        tl.Graph.union([a, b], [None, bad])
    assert ei.value.status == tl.TL_EINVAL
    swap = _dev(np.array([1, 0, 2], np.uint32))
    u = tl.Graph.union([a, b], [None, swap])
    assert u.list_count_hash(tl.TL_APP)[0] == 4 + 1
    u.free()
    a.free()
    b.free()


def test_union_of_ordered_graphs_concatenates_their_dags():
    """When every part holds its DAG and no rank is given, the union's DAG is
    assembled by concatenation; it must equal byte for byte the DAG built by
    relabel-and-sort from the same per-part orderings."""
    parts = _parts_small()
    graphs = [tl.Graph(n, _dev(e)) for n, e in parts]
    ranks = []
    for (n, e), g in zip(parts, graphs):
        off, _ = synth.simple_csr(n, e)
        r = synth.order_degree(off) if n % 2 else synth.order_random(n, n)
        g.order_apply(_dev(r))
        ranks.append(r)
    fast = tl.Graph.union(graphs)                         # concatenated DAGs
    slow = tl.Graph.union(graphs, [_dev(r) for r in ranks])  # relabel + sort
    for d in (0, 1):
        fo, fa = fast.csr(d)
        so, sa = slow.csr(d)
        assert np.array_equal(fo, so) and np.array_equal(fa, sa), d
    for alg in (tl.TL_APP, tl.TL_APM, tl.TL_AMM):
        assert fast.cost(alg) == slow.cost(alg)
    _check_union(fast, parts, ranks, [tl.TL_APP, tl.TL_APM, tl.TL_AMM] * 3 + [tl.TL_APP])
    # the union's own orderings still work (its edge set is concatenated too)
    r = fast.order_compute(tl.TL_ORDER_DEGREE)
    fast.order_apply(r)
    assert fast.list_count_hash(tl.TL_APM)[0] == slow.list_count_hash(tl.TL_APM)[0]
    fast.free()
    slow.free()
    for g in graphs:
        g.free()
