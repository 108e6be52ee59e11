"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test would fail under a plausible mistake in the oracle: a dropped
term of the cost, a swapped N+ / N- (A++ would then count C+- probes), a
wrong orientation (triangle counts off on graphs with triangles), a missed
dedup (duplicated triangles), a wrong id translation (brute-force mismatch).
"""
import itertools
import os

import numpy as np
import pytest

import oracle
from paper_2203_04774_gb300 import synth
from tests import _pins

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _fig3_lines():
    rows = []
    with open(os.path.join(GOLD, "fig3.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split(None, 3))
    return rows


def _as_set(t):
    return set(map(tuple, oracle.canonical(t).tolist()))


# ---- values printed in the paper -----------------------------------------

def test_fig3_printed_costs():
    g = oracle.Graph(7, synth.fig3_graph())
    for kind, seq, val, cite in _fig3_lines():
        if kind != "cost_pm":
            continue
        g.order_apply(synth.rank_from_sequence(seq))
        assert g.cost(oracle.APM) == int(val), (seq, cite)


def test_fig3_printed_optimum_is_global_minimum():
    """Fig. 3 caption: the optimal C+- of this graph is 3.  Brute force over
    all 7! orderings."""
    want = [int(v) for k, s, v, c in _fig3_lines() if k == "optimum_pm"][0]
    g = oracle.Graph(7, synth.fig3_graph())
    best = None
    for perm in itertools.permutations(range(7)):
        g.order_apply(np.array(perm, dtype=np.uint32))
        c = g.cost(oracle.APM)
        best = c if best is None else min(best, c)
    assert best == want


def test_fig3_triangles_brute_force():
    e = synth.fig3_graph()
    g = oracle.Graph(7, e)
    tri = _pins.brute_force_triangles(7, e)
    assert [tuple("abcdefg"[i] for i in t) for t in tri] == [
        ("a", "b", "e"), ("a", "d", "e"), ("b", "c", "g")]
    for alg in (oracle.APP, oracle.APM, oracle.AMM):
        t, cnt, _, _ = g.list(alg)
        assert _as_set(t) == set(tri) and cnt == 3


def test_split_worked_example():
    """Sec. 3.3.3: delta = (e,b,g,a,f,d,c) (C+- = 7) gives (e,g,f,c,d,a,b) (C+- = 4)."""
    row = [r for r in _fig3_lines() if r[0] == "split"][0]
    src, dst = row[1].split("->")
    delta = np.array(["abcdefg".index(ch) for ch in src])
    rank = synth.order_split(delta=delta)
    assert np.array_equal(rank, synth.rank_from_sequence(dst))
    g = oracle.Graph(7, synth.fig3_graph())
    g.order_apply(synth.rank_from_sequence(src))
    assert g.cost(oracle.APM) == 7
    g.order_apply(rank)
    assert g.cost(oracle.APM) == 4


def test_neigh_move_of_fig3():
    """Fig. 3: Neigh moves a from the first slot to just after e, C+- 9 -> 6."""
    row = [r for r in _fig3_lines() if r[0] == "neigh_move"][0]
    before, after = row[1].split(":")[1].split("->")[0], row[1].split("->")[1]
    off, adj = synth.simple_csr(7, synth.fig3_graph())
    r0 = synth.rank_from_sequence(row[1].split(":")[0])
    r1 = synth.orderings.neigh_move_one(off, adj, r0, "abcdefg".index(before))
    assert np.array_equal(r1, synth.rank_from_sequence(after))


# ---- closed forms ----------------------------------------------------------

@pytest.mark.parametrize("n", [3, 4, 7, 30])
def test_complete_graph_closed_forms(n):
    cpp, cpm, tri = _pins.kn_costs(n)
    g = oracle.Graph(n, synth.complete(n))
    for rank in (synth.order_identity(n), synth.order_random(n, 7), np.arange(n)[::-1].copy()):
        g.order_apply(rank)
        assert g.cost(oracle.APP) == cpp
        assert g.cost(oracle.APM) == cpm
        assert g.cost(oracle.AMM) == cpp  # d-_v = rank of v, as d+ mirrored
        for alg in (oracle.APP, oracle.APM, oracle.AMM):
            for mode in (oracle.LITERAL, oracle.SETS):
                _, cnt, _, probes = g.list(alg, mode, store=False)
                assert cnt == tri
    if n == 30:
        assert (cpp, cpm, tri) == (8555, 4060, 4060)


def test_star_costs():
    n = 12
    g = oracle.Graph(n, synth.star(n, hub=0))
    last = np.array([n - 1] + list(range(n - 1)), dtype=np.uint32)  # hub ranked last
    g.order_apply(last)
    assert (g.cost(oracle.APP), g.cost(oracle.APM), g.cost(oracle.AMM)) == (n - 1, 0, (n - 1) ** 2)
    g.order_apply(synth.order_identity(n))  # hub first
    assert (g.cost(oracle.APP), g.cost(oracle.APM), g.cost(oracle.AMM)) == ((n - 1) ** 2, 0, n - 1)


@pytest.mark.parametrize("d", [1, 2, 3, 4])
def test_ld_gadget(d):
    """Appendix B: e_d, v_1..v_d, K_d..K_0 has C++ = C_d, optimal (brute
    force for d <= 2); triangle count of L_d."""
    e, ids = synth.ld_gadget(d)
    n = 2 * d + 2
    g = oracle.Graph(n, e)
    seq = [ids["e"]] + ids["v"] + ids["K"][::-1]
    rank = np.empty(n, dtype=np.uint32)
    rank[np.array(seq)] = np.arange(n)
    g.order_apply(rank)
    assert g.cost(oracle.APP) == _pins.ld_closed_form(d)
    _, cnt, _, _ = g.list(oracle.APP, store=False)
    assert cnt == _pins.ld_triangles(d) == len(_pins.brute_force_triangles(n, e))
    if d <= 2:
        best = min(_cost_of(g, p, oracle.APP) for p in itertools.permutations(range(n)))
        assert best == _pins.ld_closed_form(d)


def _cost_of(g, perm, alg):
    g.order_apply(np.array(perm, dtype=np.uint32))
    return g.cost(alg)


def test_nae3sat_gadget():
    """Appendix A: every ordering of G_phi has C+- >= 2 * #clauses (each
    clause's middle literal has one predecessor and one successor in its
    triangle plus its variable); the ordering built from a NAE assignment
    reaches it exactly.  Also the 1-clause case by brute force."""
    clauses = [(0, 1, 2), (1, 2, 3), (0, 2, 3)]
    nv = 4
    e, info = synth.nae3sat_gadget(clauses, nv)
    n = info["n"]
    g = oracle.Graph(n, e)
    assign = {0: True, 1: False, 2: True, 3: False}  # NAE-satisfies all three clauses
    true_vars = [i for i in range(nv) if assign[i]]
    false_vars = [i for i in range(nv) if not assign[i]]
    F, A, T = [], [], []
    for j, cl in enumerate(clauses):
        lits = [nv + 3 * j + a for a in range(3)]
        vals = [assign[v] for v in cl]
        f = vals.index(False)
        t = vals.index(True)
        a = ({0, 1, 2} - {f, t}).pop()
        F.append(lits[f]); A.append(lits[a]); T.append(lits[t])
    seq = true_vars + F + A + T + false_vars
    rank = np.empty(n, dtype=np.uint32)
    rank[np.array(seq)] = np.arange(n)
    g.order_apply(rank)
    assert g.cost(oracle.APM) == 2 * len(clauses)
    _, cnt, _, _ = g.list(oracle.APM, store=False)
    assert cnt == len(clauses)
    for s in range(20):
        g.order_apply(synth.order_random(n, 1000 + s))
        assert g.cost(oracle.APM) >= 2 * len(clauses)
    e1, info1 = synth.nae3sat_gadget([(0, 1, 2)], 3)
    g1 = oracle.Graph(info1["n"], e1)
    assert min(_cost_of(g1, p, oracle.APM) for p in itertools.permutations(range(6))) == 2


@pytest.mark.parametrize("shape", ["bipartite", "tree", "star"])
def test_triangle_free(shape):
    if shape == "bipartite":
        n, e = 13, synth.complete_bipartite(6, 7)
    elif shape == "tree":
        n, e = 200, synth.random_tree(200, 5)
    else:
        n, e = 50, synth.star(50, 17)
    g = oracle.Graph(n, e)
    for rank in (synth.order_identity(n), synth.order_random(n, 3)):
        g.order_apply(rank)
        for alg in (oracle.APP, oracle.APM, oracle.AMM):
            for mode in (oracle.LITERAL, oracle.SETS):
                _, cnt, h, _ = g.list(alg, mode, store=False)
                assert cnt == 0 and h == 0


# ---- brute force on small random graphs ------------------------------------

def _orderings(n, e):
    off, adj = synth.simple_csr(n, e)
    yield "identity", synth.order_identity(n)
    yield "random", synth.order_random(n, 11)
    yield "degree", synth.order_degree(off)
    yield "core", synth.order_core(off, adj)
    yield "split", synth.order_split(off)
    yield "check", synth.order_check(off, adj)


@pytest.mark.parametrize("seed", list(range(100, 120)))
def test_gnp_brute_force(seed):
    n = 50
    e = synth.gnp(n, 0.2, seed)
    want = set(_pins.brute_force_triangles(n, e))
    g = oracle.Graph(n, e)
    for name, rank in _orderings(n, e):
        g.order_apply(rank)
        for alg in (oracle.APP, oracle.APM, oracle.AMM):
            for mode in (oracle.LITERAL, oracle.SETS):
                t, cnt, h, probes = g.list(alg, mode)
                assert cnt == len(want), (name, alg, mode)
                assert _as_set(t) == want, (name, alg, mode)
                assert h == oracle.hash_triples(oracle.canonical(t))


def test_k30_brute_force():
    n = 30
    e = synth.complete(n)
    want = set(_pins.brute_force_triangles(n, e))
    assert len(want) == 4060
    g = oracle.Graph(n, e)
    for alg in (oracle.APP, oracle.APM, oracle.AMM):
        t, cnt, _, _ = g.list(alg)
        assert _as_set(t) == want


def test_duplicates_loops_and_directions_are_merged():
    """Sec. 4.1: loops removed; a pair in either or both directions kept once."""
    base = synth.gnp(40, 0.25, 7)
    noisy = np.concatenate([base, base[:, ::-1], base[:50], np.array([[3, 3], [9, 9]], np.uint32)])
    g0, g1 = oracle.Graph(40, base), oracle.Graph(40, noisy)
    assert g0.m == g1.m == len(_pins.simple_edge_set(base))
    for alg in (oracle.APP, oracle.APM, oracle.AMM):
        a = g0.list(alg)
        b = g1.list(alg)
        assert a[1:] == b[1:]


def test_degrees_closed_forms():
    """Degree (Sec. 1.3) of the cleaned graph: n-1 in K_n, n-1 / 1 in a star,
    unchanged by loops, duplicates and reversed pairs; the sum is 2m."""
    assert oracle.Graph(9, synth.complete(9)).degrees().tolist() == [8] * 9
    d = oracle.Graph(7, synth.star(7, hub=3)).degrees().tolist()
    assert d == [1, 1, 1, 6, 1, 1, 1]
    base = synth.gnp(30, 0.3, 5)
    noisy = np.concatenate([base, base[:, ::-1], base[:20], np.array([[4, 4]], np.uint32)])
    g = oracle.Graph(30, noisy)
    E = _pins.simple_edge_set(base)
    want = np.zeros(30, np.int64)
    for a, b in E:
        want[a] += 1
        want[b] += 1
    assert g.degrees().tolist() == want.tolist() and int(g.degrees().sum()) == 2 * g.m


def test_lazy_dag_and_concurrent_listing():
    """The DAG is built on first use; listings of disjoint seed ranges run
    from several threads at once add up to the whole listing."""
    from concurrent.futures import ThreadPoolExecutor
    n = 2000
    e = synth.chung_lu(n, 16, 2.2, 11)
    g = oracle.Graph(n, e)
    whole = g.list(oracle.APM, store=False)  # identity ordering, built here
    assert g.cost(oracle.APM) == whole[3]
    cuts = np.linspace(0, n, 9).astype(int).tolist()
    with ThreadPoolExecutor(4) as ex:
        parts = list(ex.map(lambda r: g.list(oracle.APM, oracle.LITERAL, r[0], r[1], store=False),
                            zip(cuts, cuts[1:])))
    assert sum(p[1] for p in parts) == whole[1]
    assert sum(p[2] for p in parts) % (1 << 64) == whole[2]
    assert sum(p[3] for p in parts) == whole[3]


# ---- Property 1 and invariants -------------------------------------------

@pytest.mark.parametrize("seed", [1, 2, 3])
def test_property1_probes_equal_cost(seed):
    """Property 1: the inner test runs sum_(u,w) d+_u = C++ times in A++ and
    sum_(u,v) d+_v = C+- times in A+-."""
    n = 400
    e = synth.chung_lu(n, 12, 2.3, seed)
    g = oracle.Graph(n, e)
    for name, rank in _orderings(n, e):
        g.order_apply(rank)
        for alg in (oracle.APP, oracle.APM, oracle.AMM):
            _, _, _, probes = g.list(alg, oracle.LITERAL, store=False)
            assert probes == g.cost(alg), (name, alg)


def test_invariants_across_orderings_and_algorithms():
    n = 2000
    e = synth.chung_lu(n, 16, 2.2, 9)
    g = oracle.Graph(n, e)
    m = g.m
    ref = None
    for name, rank in _orderings(n, e):
        g.order_apply(rank)
        off_o, adj_o = g.csr(0)
        off_i, adj_i = g.csr(1)
        dp, dm = np.diff(off_o.astype(np.int64)), np.diff(off_i.astype(np.int64))
        assert dp.sum() == dm.sum() == m
        assert g.cost(oracle.APP) >= m
        assert g.cost(oracle.APP) == int((dp * dp).sum())
        # N- is the transpose of N+ and every row is strictly increasing
        src = np.repeat(np.arange(n), dp)
        assert np.all(adj_o > src)
        fw = set(zip(src.tolist(), adj_o.tolist()))
        bw = set(zip(adj_i.tolist(), np.repeat(np.arange(n), dm).tolist()))
        assert fw == bw
        for off, adj in ((off_o, adj_o), (off_i, adj_i)):
            for x in range(0, n, 97):
                row = adj[off[x]:off[x + 1]]
                assert np.all(np.diff(row.astype(np.int64)) > 0)
        for alg in (oracle.APP, oracle.APM, oracle.AMM):
            t, cnt, h, _ = g.list(alg)
            c = oracle.canonical(t)
            assert len({tuple(r) for r in c.tolist()}) == cnt  # no duplicates
            per_vertex = np.bincount(c.ravel(), minlength=n)
            assert per_vertex.sum() == 3 * cnt
            key = (cnt, h)
            ref = key if ref is None else ref
            assert key == ref, (name, alg)
    # every reported triple is a triangle of the graph
    E = _pins.simple_edge_set(e)
    for a, b, c in oracle.canonical(t).tolist()[:2000]:
        assert (a, b) in E and (a, c) in E and (b, c) in E


def test_seed_ranges_partition_the_listing():
    n = 3000
    g = oracle.Graph(n, synth.chung_lu(n, 20, 2.5, 4))
    g.order_apply(synth.order_degree(synth.simple_csr(n, synth.chung_lu(n, 20, 2.5, 4))[0]))
    for alg in (oracle.APP, oracle.APM, oracle.AMM):
        _, cnt, h, p = g.list(alg, store=False)
        cuts = [0, 17, 900, 2999, n]
        parts = [g.list(alg, seed_begin=a, seed_end=b, store=False) for a, b in zip(cuts, cuts[1:])]
        assert sum(x[1] for x in parts) == cnt
        assert sum(x[2] for x in parts) % (1 << 64) == h
        assert sum(x[3] for x in parts) == p


def test_invalid_inputs_rejected():
    with pytest.raises(oracle.OracleError):
        oracle.Graph(5, np.array([[0, 5]], np.uint32))
    g = oracle.Graph(5, np.array([[0, 1], [1, 2], [0, 2]], np.uint32))
    with pytest.raises(oracle.OracleError):
        g.order_apply(np.array([0, 1, 1, 3, 4], np.uint32))
    with pytest.raises(oracle.OracleError):
        g.order_apply(np.array([0, 1, 2, 3, 5], np.uint32))
    # the failed calls left the previous (identity) ordering in force
    assert g.cost(oracle.APP) == 2 * 2 + 1 * 1  # identity: d+ = (2, 1, 0, 0, 0)


# ---- the set hash ----------------------------------------------------------

def test_mix64_published_vectors():
    """splitmix64 with state 0 outputs 0xe220a8397b1dcdaf, 0x6e789e6aa1b965f4,
    0x06c45d188009454f (its i-th output is the finaliser of i * GAMMA)."""
    G = 0x9E3779B97F4A7C15
    M = (1 << 64) - 1
    assert oracle.mix64(G) == 0xE220A8397B1DCDAF
    assert oracle.mix64((2 * G) & M) == 0x6E789E6AA1B965F4
    assert oracle.mix64((3 * G) & M) == 0x06C45D188009454F


def test_set_hash_is_order_free_and_sensitive():
    t = oracle.canonical(np.array(_pins.brute_force_triangles(30, synth.complete(30))))
    h = oracle.hash_triples(t)
    rng = np.random.default_rng(0)
    assert oracle.hash_triples(t[rng.permutation(len(t))]) == h
    assert oracle.hash_triples(t[:-1]) != h
    t2 = t.copy()
    t2[5] = (t2[5][0], t2[5][1], t2[5][2] + 1) if t2[5][2] < 29 else t2[5]
    assert oracle.hash_triples(t2) != h
    # all 4060 per-triple values distinct
    per = [oracle.hash_triples(t[i:i + 1]) for i in range(len(t))]
    assert len(set(per)) == len(per)


def test_core_numbers_closed_forms_and_brute_force():
    """Coreness (Sec. 1.3): K_n -> n-1, trees and stars -> 1, a cycle -> 2,
    isolated vertices -> 0; K_5 joined to a path -> 4 on the clique, 1 on the
    path; and on small random graphs, the definition checked by brute force
    (c_v = the largest k whose k-core, found by deleting vertices of degree
    < k until none is left, contains v)."""
    assert list(oracle.core_numbers(6, synth.complete(6))) == [5] * 6
    assert list(oracle.core_numbers(20, synth.random_tree(20, 3))) == [1] * 20
    assert list(oracle.core_numbers(9, synth.star(9))) == [1] * 9
    cyc = np.stack([np.arange(7), (np.arange(7) + 1) % 7], 1)
    assert list(oracle.core_numbers(7, cyc)) == [2] * 7
    assert list(oracle.core_numbers(4, np.zeros((0, 2), np.uint32))) == [0] * 4
    path = np.array([[4, 5], [5, 6], [6, 7]])
    c = oracle.core_numbers(8, np.concatenate([synth.complete(5), path]))
    assert list(c) == [4] * 5 + [1] * 3

    def brute(n, e):
        nb = [set() for _ in range(n)]
        for a, b in e:
            if a != b:
                nb[a].add(b)
                nb[b].add(a)
        core = [0] * n
        for k in range(1, n):
            alive = set(range(n))
            changed = True
            while changed:
                changed = False
                for v in list(alive):
                    if len(nb[v] & alive) < k:
                        alive.discard(v)
                        changed = True
            for v in alive:
                core[v] = k
        return core

    for seed in range(6):
        e = synth.gnp(25, 0.25, 40 + seed)
        assert list(oracle.core_numbers(25, e)) == brute(25, e.tolist()), seed


def test_core_order_levels_is_a_degeneracy_ordering():
    """The level-synchronous core ordering: a permutation along which the
    coreness never decreases and every vertex has at most c_v later
    neighbours (d+_v <= c_v); its maximum d+ is the degeneracy max_v c_v.
    Worked cases: on K_5 plus a pendant path the path goes first (level 1)
    and the clique last; on a star the leaves are taken in one round before
    the hub's degree falls, so the hub comes last."""
    cases = [(8, np.concatenate([synth.complete(5), np.array([[4, 5], [5, 6], [6, 7]])])),
             (9, synth.star(9))]
    for seed in range(8):
        n = 60 + 20 * seed
        cases.append((n, synth.chung_lu(n, 8, 2.3, 70 + seed)))
    for n, e in cases:
        r = oracle.core_order_levels(n, e).astype(np.int64)
        assert sorted(r.tolist()) == list(range(n))
        c = oracle.core_numbers(n, e)
        inv = np.argsort(r)
        assert np.all(np.diff(c[inv]) >= 0)
        off, adj = synth.simple_csr(n, e)
        src = np.repeat(np.arange(n), np.diff(off.astype(np.int64)))
        later = r[adj.astype(np.int64)] > r[src]
        dplus = np.bincount(src[later], minlength=n)
        assert np.all(dplus <= c)
        assert dplus.max(initial=0) == c.max(initial=0)
    r = oracle.core_order_levels(8, cases[0][1])
    assert sorted(r[5:].tolist()) == [0, 1, 2] and sorted(r[:5].tolist()) == [3, 4, 5, 6, 7]
    r = oracle.core_order_levels(9, synth.star(9))
    assert r[0] == 8


def test_amm_is_app_on_the_reversed_ordering():
    """A-- (seed edge S2) is the mirror image of A++ (seed edge L): reversing
    the ordering swaps N+ and N-, so C--(pi) = C++(reversed pi) and both list
    the same triangles with the same number of tests (the footnote of Sec. 2.1
    calls their complexities equivalent)."""
    for seed in range(5):
        n = 400
        e = synth.chung_lu(n, 12, 2.3, 90 + seed)
        g = oracle.Graph(n, e)
        r = synth.order_random(n, seed)
        g.order_apply(r)
        t_mm, c_mm, h_mm, p_mm = g.list(oracle.AMM)
        cost_mm = g.cost(oracle.AMM)
        g.order_apply((n - 1 - r.astype(np.int64)).astype(np.uint32))
        t_pp, c_pp, h_pp, p_pp = g.list(oracle.APP)
        assert cost_mm == g.cost(oracle.APP) == p_mm == p_pp
        assert (c_mm, h_mm) == (c_pp, h_pp)
        assert np.array_equal(oracle.canonical(t_mm), oracle.canonical(t_pp))
