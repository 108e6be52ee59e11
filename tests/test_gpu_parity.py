"""CUDA path vs the CPU oracle, element by element (triangle sets are exact).

Every call goes through the C ABI (libtl.so) via the thin ctypes binding.
"""
import numpy as np
import pytest

import oracle
import paper_2203_04774_gb300 as tl
from paper_2203_04774_gb300 import synth
from tests import _pins

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


def _orderings(n, e, which=("identity", "random", "degree", "core", "split", "check")):
    off, adj = synth.simple_csr(n, e)
    table = {
        "identity": lambda: synth.order_identity(n),
        "random": lambda: synth.order_random(n, 11),
        "degree": lambda: synth.order_degree(off),
        "core": lambda: synth.order_core(off, adj),
        "split": lambda: synth.order_split(off),
        "check": lambda: synth.order_check(off, adj),
        "neigh": lambda: synth.order_neigh(off, adj)[0],
        "neigh_c++": lambda: synth.order_neigh(off, adj, objective="C++")[0],
    }
    for name in which:
        yield name, table[name]()


def _compare(n, e, orderings, algs=(tl.TL_APP, tl.TL_APM, tl.TL_AMM), chunk_bytes=tl.TL_MIN_CHUNK_BYTES,
             host_edges=False):
    g = tl.Graph(n, e if host_edges else _dev(e))
    ref = oracle.Graph(n, e)
    assert g.m == ref.m
    for name, rank in orderings:
        g.order_apply(_dev(rank))
        ref.order_apply(rank)
        for d in (0, 1):
            off_g, adj_g = g.csr(d)
            off_r, adj_r = ref.csr(d)
            assert np.array_equal(off_g, off_r), (name, d)
            assert np.array_equal(adj_g, adj_r), (name, d)
        for alg in algs:
            assert g.cost(alg) == ref.cost(alg), (name, alg)
            t, nt, probes, _ = g.list_collect(alg, chunk_bytes)
            rt, rc, rh, rp = ref.list(alg)
            assert nt == rc == len(t), (name, alg)
            assert probes == rp == ref.cost(alg), (name, alg)  # Property 1
            assert np.array_equal(oracle.canonical(t), oracle.canonical(rt)), (name, alg)
            assert oracle.hash_triples(t) == rh
    g.free()


def test_fig3_graph_every_ordering_in_the_paper():
    e = synth.fig3_graph()
    seqs = ["abcdefg", "bcdeafg", "egfacdb", "ebgafdc", "egfcdab"]
    g = tl.Graph(7, _dev(e))
    for seq, cpm in zip(seqs, [9, 6, 3, 7, 4]):  # values printed with Fig. 3 and in Sec. 3.3.3
        g.order_apply(_dev(synth.rank_from_sequence(seq)))
        assert g.cost(tl.TL_APM) == cpm
    _compare(7, e, [(s, synth.rank_from_sequence(s)) for s in seqs])


@pytest.mark.parametrize("seed", list(range(100, 120)))
def test_gnp_vs_oracle_and_brute_force(seed):
    n = 50
    e = synth.gnp(n, 0.2, seed)
    _compare(n, e, _orderings(n, e))
    g = tl.Graph(n, _dev(e))
    t, nt, _, _ = g.list_collect(tl.TL_APP)
    assert set(map(tuple, oracle.canonical(t).tolist())) == set(_pins.brute_force_triangles(n, e))


@pytest.mark.parametrize("n", [3, 30, 32, 33, 34, 100])
def test_complete_graphs(n):
    cpp, cpm, tri = _pins.kn_costs(n)
    e = synth.complete(n)
    g = tl.Graph(n, _dev(e))
    for rank in (synth.order_identity(n), synth.order_random(n, 3)):
        g.order_apply(_dev(rank))
        # C-- of K_n equals C++ (d-_v = rank of v, mirrored)
        assert (g.cost(tl.TL_APP), g.cost(tl.TL_APM), g.cost(tl.TL_AMM)) == (cpp, cpm, cpp)
        for alg in (tl.TL_APP, tl.TL_APM, tl.TL_AMM):
            t, nt, probes, _ = g.list_collect(alg)
            assert nt == tri and probes == (cpm if alg == tl.TL_APM else cpp)
            assert len(set(map(tuple, t.tolist()))) == tri


@pytest.mark.parametrize("shape", ["bipartite", "tree", "star"])
def test_triangle_free(shape):
    n, e = {"bipartite": (60, synth.complete_bipartite(25, 35)),
            "tree": (5000, synth.random_tree(5000, 5)),
            "star": (4000, synth.star(4000, 17))}[shape]
    _compare(n, e, _orderings(n, e, ("identity", "random", "degree")))


@pytest.mark.parametrize("d", [1, 2, 5, 12])
def test_ld_gadget(d):
    e, ids = synth.ld_gadget(d)
    n = 2 * d + 2
    seq = [ids["e"]] + ids["v"] + ids["K"][::-1]
    rank = np.empty(n, dtype=np.uint32)
    rank[np.array(seq)] = np.arange(n)
    g = tl.Graph(n, _dev(e))
    g.order_apply(_dev(rank))
    assert g.cost(tl.TL_APP) == _pins.ld_closed_form(d)
    assert g.list_collect(tl.TL_APP)[1] == _pins.ld_triangles(d)


def test_config1_chung_lu_full_set():
    """Chung-Lu n=10^4, average degree 20, exponent 2.5, seed 1, degree
    ordering, A++ (plus A+- and other orderings): full set compare."""
    n = 10000
    e = synth.chung_lu(n, 20, 2.5, 1)
    _compare(n, e, _orderings(n, e, ("degree", "core", "random", "split", "check", "neigh",
                                     "neigh_c++")))


def test_host_edges_and_host_rank():
    n = 3000
    e = synth.chung_lu(n, 16, 2.2, 6)
    g = tl.Graph(n, e)  # host pointer
    off, _ = synth.simple_csr(n, e)
    rank = synth.order_degree(off)
    g.order_apply(rank)  # host pointer
    ref = oracle.Graph(n, e)
    ref.order_apply(rank)
    for alg in (tl.TL_APP, tl.TL_APM, tl.TL_AMM):
        t, nt, _, _ = g.list_collect(alg)
        assert np.array_equal(oracle.canonical(t), oracle.canonical(ref.list(alg)[0]))


def test_duplicates_loops_reversed_pairs():
    n = 400
    base = synth.chung_lu(n, 12, 2.4, 3)
    noisy = np.concatenate([base, base[:, ::-1], base[: len(base) // 3],
                            np.stack([np.arange(n), np.arange(n)], 1).astype(np.uint32)])
    _compare(n, noisy, _orderings(n, noisy, ("degree", "random")))


def test_edge_cases_empty_and_tiny():
    import torch
    for n, e in [(1, np.zeros((0, 2), np.uint32)), (5, np.zeros((0, 2), np.uint32)),
                 (3, np.array([[1, 1], [2, 2]], np.uint32)), (2, np.array([[0, 1]], np.uint32)),
                 (3, np.array([[0, 1], [1, 2], [2, 0]], np.uint32))]:
        g = tl.Graph(n, e)
        for alg in (tl.TL_APP, tl.TL_APM, tl.TL_AMM):
            t, nt, probes, calls = g.list_collect(alg)
            want = len(_pins.brute_force_triangles(n, e))
            assert nt == want == len(t)
        g.free()


def test_invalid_inputs():
    e = np.array([[0, 1], [1, 2], [0, 2]], np.uint32)
    with pytest.raises(tl.TLError) as ei:
        tl.Graph(3, np.array([[0, 3]], np.uint32))
    assert ei.value.status == tl.TL_EINVAL
    g = tl.Graph(3, _dev(e))
    before = g.csr(0)
    for bad in ([0, 1, 1], [0, 1, 3]):
        with pytest.raises(tl.TLError) as ei:
            g.order_apply(_dev(np.array(bad, np.uint32)))
        assert ei.value.status == tl.TL_EINVAL
    after = g.csr(0)  # previous ordering still in force
    assert np.array_equal(before[0], after[0]) and np.array_equal(before[1], after[1])
    with pytest.raises(tl.TLError) as ei:
        tl.tl_list_triangles(g.h, tl.TL_APP, 1 << 20)
    assert ei.value.status == tl.TL_EINVAL  # chunk below the minimum
    with pytest.raises(tl.TLError) as ei:
        tl.tl_list_triangles_range(g.h, tl.TL_APP, 2, 1)
    assert ei.value.status == tl.TL_EINVAL
    for bad in ({"narrow_max_p": 257}, {"warp_work": 255}, {"large_max": 1024},
                {"narrow_keep_mib": 4097}, {"narrow_cold_first": 2}, {"large_hash_max_p": 16385}):
        with pytest.raises(tl.TLError) as ei:
            tl.tl_set_tuning(g.h, bad)
        assert ei.value.status == tl.TL_EINVAL, bad
        assert tl.tl_get_tuning(g.h) == tl.tl_default_tuning()  # split unchanged


def test_many_chunks_k300():
    """4,455,100 triangles of K_300 through 12 MiB chunks (1,048,576 triples
    each): several overflow/resume rounds, no triangle lost or repeated."""
    n = 300
    e = synth.complete(n)
    g = tl.Graph(n, _dev(e))
    g.order_apply(_dev(synth.order_random(n, 5)))
    for alg in (tl.TL_APP, tl.TL_APM, tl.TL_AMM):
        t, nt, probes, calls = g.list_collect(alg, tl.TL_MIN_CHUNK_BYTES)
        assert nt == len(t) == 300 * 299 * 298 // 6
        assert calls >= 5
        assert len(np.unique(oracle.canonical(t), axis=0)) == nt
        assert oracle.hash_triples(t) == oracle.Graph(n, e).list(alg, store=False)[2]


def test_seed_ranges_partition():
    n = 10000
    e = synth.chung_lu(n, 20, 2.5, 1)
    off, _ = synth.simple_csr(n, e)
    rank = synth.order_degree(off)
    g = tl.Graph(n, _dev(e))
    g.order_apply(_dev(rank))
    ref = oracle.Graph(n, e)
    ref.order_apply(rank)
    for alg in (tl.TL_APP, tl.TL_APM, tl.TL_AMM):
        cuts = [0, 1, 777, 5000, 9990, n]
        parts = []
        for a, b in zip(cuts, cuts[1:]):
            t, nt, probes, _ = g.list_collect(alg, x_begin=a, x_end=b)
            rt, rc, rh, rp = ref.list(alg, seed_begin=a, seed_end=b)
            assert nt == rc and probes == rp
            assert np.array_equal(oracle.canonical(t), oracle.canonical(rt))
            parts.append(t)
        allt = np.concatenate(parts)
        assert len(np.unique(oracle.canonical(allt), axis=0)) == len(allt)


def test_count_hash_consumer_matches_oracle():
    n = 10000
    e = synth.chung_lu(n, 20, 2.5, 1)
    off, _ = synth.simple_csr(n, e)
    rank = synth.order_degree(off)
    g = tl.Graph(n, _dev(e))
    g.order_apply(_dev(rank))
    ref = oracle.Graph(n, e)
    ref.order_apply(rank)
    for alg in (tl.TL_APP, tl.TL_APM, tl.TL_AMM):
        nt, cnt, h, probes = g.list_count_hash(alg)
        _, rc, rh, rp = ref.list(alg, store=False)
        assert (nt, cnt, h, probes) == (rc, rc, rh, rp)


@pytest.mark.parametrize("offset", [0, 1, 2, 3, 5])
def test_count_hash_any_alignment_and_length(offset):
    """The consumer reads 16-byte groups when it can; any start triple and
    any length gives the oracle's count and hash."""
    import torch
    rng = np.random.default_rng(offset)
    t = np.sort(rng.integers(0, 1 << 31, size=(100_003, 3), dtype=np.uint32), axis=1)
    dev = torch.from_numpy(t.view(np.int32)).cuda()
    for n in (0, 1, 7, 4096, len(t) - offset):
        sub = t[offset:offset + n]
        ch = tl.CountHash()
        try:
            rc = tl.lib().tl_count_hash(dev.data_ptr() + 12 * offset, n, 0, ch.user)
            assert rc == 0
            assert (int(ch.state.count), int(ch.state.hash)) == (n, oracle.hash_triples(sub))
        finally:
            ch.release()


def test_every_tier_runs_and_matches():
    """Chung-Lu graph plus a wheel (hub joined to a 5000-cycle): probe sets of
    every size, so all five listing kernels (small, medium, narrow, mid,
    large with the shared-memory bitmap) get tasks; full set compare with the
    oracle."""
    n = 60000
    base = synth.chung_lu(n, 24, 2.1, 21)
    k = 5000
    spokes = np.stack([np.zeros(k, np.uint32), np.arange(1, k + 1, dtype=np.uint32)], 1)
    rim = np.stack([np.arange(1, k + 1, dtype=np.uint32),
                    np.r_[np.arange(2, k + 1), 1].astype(np.uint32)], 1)
    e = np.concatenate([base, spokes, rim])
    off, adj = synth.simple_csr(n, e)
    seen = np.zeros(tl.TL_KERNELS, dtype=np.int64)
    g = tl.Graph(n, _dev(e))
    ref = oracle.Graph(n, e)
    for name, rank in [("degree", synth.order_degree(off)), ("identity", synth.order_identity(n)),
                       ("random", synth.order_random(n, 4))]:
        g.order_apply(_dev(rank))
        ref.order_apply(rank)
        for alg in (tl.TL_APP, tl.TL_APM, tl.TL_AMM):
            t, nt, probes, _ = g.list_collect(alg)
            st = tl.tl_last_list_stats(g.h)
            seen += np.array(st["tasks"]) > 0
            rt, rc, rh, rp = ref.list(alg)
            assert (nt, probes) == (rc, rp), (name, alg)
            assert sum(st["kernel_probes"]) == rp and sum(st["kernel_triangles"]) == rc
            assert np.array_equal(oracle.canonical(t), oracle.canonical(rt)), (name, alg)
    assert np.all(seen > 0), seen


@pytest.mark.parametrize("large_hash_max_p", [16384, 0])
def test_large_n_hash_probe_path(large_hash_max_p):
    """n above the shared-memory bitmap limit (1,572,864 ranks): the large
    kernel probes with a shared-memory hash table, and with binary search for
    probe sets too large for it (a star-like hub with 40,000 neighbours); with
    large_hash_max_p = 0 every large vertex takes the filter + global table."""
    n = 2_000_000
    e1 = synth.chung_lu(n, 4, 2.1, 12)
    hub = np.stack([np.zeros(40000, np.uint32), np.arange(1, 40001, dtype=np.uint32)], 1)
    ring = np.stack([np.arange(1, 40000, dtype=np.uint32), np.arange(2, 40001, dtype=np.uint32)], 1)
    # a second hub with 150,000 neighbours: beyond the global hash table too
    h2 = 1_000_000
    leaves = np.arange(h2 + 1, h2 + 150_001, dtype=np.uint32)
    hub2 = np.stack([np.full_like(leaves, h2), leaves], 1)
    ring2 = np.stack([leaves[:-1], leaves[1:]], 1)
    e = np.concatenate([e1, hub, ring, hub2, ring2])
    off, _ = synth.simple_csr(n, e)
    orders = [("degree", synth.order_degree(off)), ("identity", synth.order_identity(n)),
              ("reverse", (n - 1 - np.arange(n)).astype(np.uint32))]
    g = tl.Graph(n, _dev(e))
    tl.tl_set_tuning(g.h, {"large_hash_max_p": large_hash_max_p})
    ref = oracle.Graph(n, e)
    for name, rank in orders:
        g.order_apply(_dev(rank))
        ref.order_apply(rank)
        # A-- only where the 150,000-neighbour hub is not last among its
        # neighbours (else C-- >= 150,000^2 tests for the oracle)
        algs = (tl.TL_APP, tl.TL_APM) + ((tl.TL_AMM,) if name == "identity" else ())
        for alg in algs:
            nt, cnt, h, probes = g.list_count_hash(alg)
            _, rc, rh, rp = ref.list(alg, store=False)
            assert (nt, h, probes) == (rc, rh, rp), (name, alg)


@pytest.mark.parametrize("kind", ["degree", "split"])
def test_device_orderings_match_host(kind):
    """tl_order_compute (degree ordering of Sec. 2.2, Split of Sec. 3.3.3) is
    bit-identical to the host orderings, ties by id included."""
    import torch
    for n, e in [(7, synth.fig3_graph()), (3000, synth.chung_lu(3000, 12, 2.3, 8)),
                 (5000, synth.complete_bipartite(10, 4990)), (4000, synth.star(4000, 11)),
                 (1, np.zeros((0, 2), np.uint32))]:
        off, _ = synth.simple_csr(n, e)
        want = synth.order_degree(off) if kind == "degree" else synth.order_split(off)
        g = tl.Graph(n, _dev(e))
        k = tl.TL_ORDER_DEGREE if kind == "degree" else tl.TL_ORDER_SPLIT
        assert np.array_equal(tl.tl_order_compute(g.h, k), want), (n, kind)
        dev_rank = torch.empty(n, dtype=torch.int32, device="cuda")
        tl.tl_order_compute(g.h, k, dev_rank)
        assert np.array_equal(dev_rank.cpu().numpy().view(np.uint32), want)
        g.order_apply(dev_rank)  # usable directly as an ordering
        ref = oracle.Graph(n, e)
        ref.order_apply(want)
        assert g.cost(tl.TL_APP) == ref.cost(tl.TL_APP)
        g.free()


def test_device_core_ordering_matches_oracle():
    """TL_ORDER_CORE is the level-synchronous core ordering, rank for rank
    (oracle.core_order_levels); it is a degeneracy ordering (coreness
    non-decreasing, d+_v <= c_v) and lists the same triangles."""
    k = 3000
    spokes = np.stack([np.zeros(k, np.uint32), np.arange(1, k + 1, dtype=np.uint32)], 1)
    rim = np.stack([np.arange(1, k + 1, dtype=np.uint32),
                    np.r_[np.arange(2, k + 1), 1].astype(np.uint32)], 1)
    cases = [(7, synth.fig3_graph()), (3000, synth.chung_lu(3000, 12, 2.3, 8)),
             (20000, synth.chung_lu(20000, 30, 2.1, 9)), (40, synth.complete(40)),
             (4000, synth.star(4000, 11)), (1, np.zeros((0, 2), np.uint32)),
             (50, np.zeros((0, 2), np.uint32)), (k + 1, np.concatenate([spokes, rim])),
             (5000, synth.complete_bipartite(10, 4990))]
    for n, e in cases:
        want = oracle.core_order_levels(n, e)
        g = tl.Graph(n, _dev(e))
        got = g.order_compute(tl.TL_ORDER_CORE).cpu().numpy().view(np.uint32)
        assert np.array_equal(got, want), n
        c = oracle.core_numbers(n, e)
        assert np.all(np.diff(c[np.argsort(got)]) >= 0)
        off, adj = synth.simple_csr(n, e)
        src = np.repeat(np.arange(n), np.diff(off.astype(np.int64)))
        r = got.astype(np.int64)
        dplus = np.bincount(src[r[adj.astype(np.int64)] > r[src]], minlength=n)
        assert np.all(dplus <= c)
        g.order_apply(_dev(got))
        ref = oracle.Graph(n, e)
        ref.order_apply(want)
        for alg in (tl.TL_APP, tl.TL_APM, tl.TL_AMM):
            assert g.cost(alg) == ref.cost(alg)
            nt, _, h, _ = g.list_count_hash(alg)
            _, rc, rh, _ = ref.list(alg, store=False)
            assert (nt, h) == (rc, rh)
        g.free()


def test_device_generator_on_gpu_matches_host():
    from paper_2203_04774_gb300.synth import device as dev
    e = synth.chung_lu(50000, 20, 2.2, 4)
    t = dev.chung_lu_device(50000, 20, 2.2, 4, device="cuda", block=1 << 16)
    assert np.array_equal(e, t.cpu().numpy().view(np.uint32))


@pytest.mark.parametrize("tuning", [
    {"warp_work": 256, "narrow_piece": 1024, "mid_piece": 1024, "large_per_p": 1,
     "large_min": 1024, "large_max": 1024},
    {"warp_work": 1024, "narrow_piece": 1 << 20, "mid_piece": 1 << 22, "large_per_p": 4096,
     "large_min": 1 << 16, "large_max": 1 << 26},
    {"small_max_p": 4, "medium_max_p": 40, "narrow_max_p": 16, "mid_max_p": 100},
    {"small_max_p": 0, "medium_max_p": 0, "narrow_max_p": 0, "mid_max_p": 0},
    # L2 priorities of the narrow kernel's short steps: about half of the
    # scanned CSR kept (evict_last), the rest evict_first; all kept
    {"small_max_p": 0, "medium_max_p": 0, "narrow_keep_mib": 1, "narrow_cold_first": 1},
    {"small_max_p": 0, "medium_max_p": 0, "narrow_keep_mib": 4096},
    {"mid_max_p": 300, "large_hash_max_p": 0},
])
def test_tuning_changes_speed_not_results(tuning):
    """The work split (tl_set_tuning) changes task shapes only: extreme piece
    sizes, warp-task sizes and probe-set thresholds (down to every vertex in
    the large kernel) list the oracle's triangle set with probes = C++ / C+- /
    C-- (Property 1); so do the narrow kernel's L2 load priorities."""
    n = 30000
    e = np.concatenate([synth.chung_lu(n, 30, 2.1, 31), synth.complete(90)])
    rank = synth.order_degree(synth.simple_csr(n, e)[0])
    g = tl.Graph(n, _dev(e))
    g.order_apply(_dev(rank))
    ref = oracle.Graph(n, e)
    ref.order_apply(rank)
    tl.tl_set_tuning(g.h, tuning)
    assert tl.tl_get_tuning(g.h) == dict(tl.tl_default_tuning(), **tuning)
    for alg in (tl.TL_APP, tl.TL_APM, tl.TL_AMM):
        t, nt, probes, _ = g.list_collect(alg, tl.TL_MIN_CHUNK_BYTES)
        rt, rc, rh, rp = ref.list(alg)
        assert (nt, probes) == (rc, rp), alg
        assert probes == g.cost(alg), alg
        assert np.array_equal(oracle.canonical(t), oracle.canonical(rt)), alg
    tl.tl_set_tuning(g.h, None)
    assert tl.tl_get_tuning(g.h) == tl.tl_default_tuning()
    g.free()
