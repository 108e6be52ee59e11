"""The seeded input generators and the host orderings."""
import numpy as np
import pytest

import oracle
from paper_2203_04774_gb300 import synth


def test_counter_streams_are_chunk_independent():
    a = synth.counter_u64(5, 3, 1000)
    b = np.concatenate([synth.counter_u64(5, 3, 400), synth.counter_u64(5, 3, 600, start=400)])
    assert np.array_equal(a, b)
    assert not np.array_equal(a, synth.counter_u64(5, 4, 1000))
    assert not np.array_equal(a, synth.counter_u64(6, 3, 1000))
    u = synth.counter_uniform(1, 0, 100000)
    assert 0.0 <= u.min() and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.01


def test_chung_lu_shape_and_determinism():
    e = synth.chung_lu(10000, 20, 2.5, 1)
    assert e.shape == (100000, 2) and e.dtype == np.uint32 and e.max() < 10000
    assert np.array_equal(e, synth.chung_lu(10000, 20, 2.5, 1))
    w = synth.chung_lu_weights(10000, 20, 2.5)
    assert w.max() <= np.sqrt(10000 * 20) * (1 + 1e-12)  # capped at sqrt of the pre-cap sum
    off, _ = synth.simple_csr(10000, e)
    deg = np.diff(off)
    assert deg[:10].mean() > 5 * deg.mean()  # low ids are the hubs


def test_rmat_shape():
    e = synth.rmat(10, 16, 0.57, 0.19, 0.19, 2)
    assert e.shape == (16 << 10, 2) and e.max() < 1024
    # quadrant (0,0) is the most likely: low ids dominate
    assert (e < 512).mean() > 0.6


def _coreness(n, off, adj):
    """Coreness by repeated peeling (Sec. 1.3 definition): plain and slow."""
    deg = np.diff(off).astype(np.int64)
    alive = np.ones(n, bool)
    core = np.zeros(n, np.int64)
    k = 0
    while alive.any():
        changed = True
        while changed:
            changed = False
            for v in np.nonzero(alive & (deg <= k))[0]:
                alive[v] = False
                core[v] = k
                changed = True
                for u in adj[off[v]:off[v + 1]]:
                    if alive[u]:
                        deg[u] -= 1
        k += 1
    return core


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_orderings_are_permutations_with_their_defining_property(seed):
    n = 600
    e = synth.chung_lu(n, 10, 2.3, seed)
    off, adj = synth.simple_csr(n, e)
    deg = np.diff(off)
    ident = np.arange(n)
    ranks = {
        "identity": synth.order_identity(n),
        "random": synth.order_random(n, seed),
        "degree": synth.order_degree(off),
        "core": synth.order_core(off, adj),
        "split": synth.order_split(off),
        "check": synth.order_check(off, adj),
        "neigh": synth.order_neigh(off, adj)[0],
    }
    for name, r in ranks.items():
        assert np.array_equal(np.sort(r), ident), name
    seq = np.argsort(ranks["degree"])
    assert np.all(np.diff(deg[seq]) >= 0)
    core = _coreness(n, off, adj)
    seq = np.argsort(ranks["core"])
    assert np.all(np.diff(core[seq]) >= 0)


def test_neigh_and_check_lower_cpm():
    n = 3000
    e = synth.chung_lu(n, 16, 2.3, 8)
    off, adj = synth.simple_csr(n, e)
    g = oracle.Graph(n, e)
    g.order_apply(synth.order_degree(off))
    c_deg = g.cost(oracle.APM)
    rank, trace = synth.order_neigh(off, adj)
    assert trace[0] == c_deg
    assert all(b <= a for a, b in zip(trace, trace[1:]))
    g.order_apply(rank)
    assert g.cost(oracle.APM) == trace[-1] < c_deg
    g.order_apply(synth.order_check(off, adj))
    c_check = g.cost(oracle.APM)
    g.order_apply(synth.order_random(n, 1))
    assert c_check < g.cost(oracle.APM)


def test_device_generator_matches_host_generator():
    """The torch (device) Chung-Lu generator draws exactly the host edges;
    checked here with torch on the CPU."""
    torch = pytest.importorskip("torch")
    from paper_2203_04774_gb300.synth import device as dev
    e = synth.chung_lu(20000, 16, 2.2, 7)
    t = dev.chung_lu_device(20000, 16, 2.2, 7, device="cpu", block=30000)
    assert t.dtype == torch.int32
    assert np.array_equal(e, t.numpy().view(np.uint32))
    assert np.array_equal(synth.counter_uniform(3, 1, 1000, start=77),
                          dev.counter_uniform_t(3, 1, 1000, 77, "cpu").numpy())


def _place(rank, u, nb_sorted, p):
    """Ordering with u removed and put back just after nb_sorted[p-1]
    (p = 0: just before nb_sorted[0]); rank order of the others unchanged."""
    seq = [v for v in np.argsort(rank, kind="stable") if v != u]
    at = seq.index(nb_sorted[0]) if p == 0 else seq.index(nb_sorted[p - 1]) + 1
    seq.insert(at, u)
    out = np.empty(len(rank), dtype=np.uint32)
    out[np.array(seq)] = np.arange(len(rank), dtype=np.uint32)
    return out


@pytest.mark.parametrize("objective,alg", [("C+-", oracle.APM), ("C++", oracle.APP)])
def test_neigh_move_takes_the_cheapest_slot(objective, alg):
    """One Neigh move (Algorithm 3) against brute force: every slot of the
    moved vertex among its neighbours is tried and its cost computed by the
    oracle; the move lands on a cheapest one, the current slot on a tie, else
    the smallest."""
    rng = np.random.default_rng(11)
    moved = 0
    for trial in range(12):
        n = 14
        e = np.array([(a, b) for a in range(n) for b in range(a + 1, n) if rng.random() < 0.35],
                     dtype=np.uint32)
        off, adj = synth.simple_csr(n, e)
        g = oracle.Graph(n, e)
        rank = rng.permutation(n).astype(np.uint32)
        for u in range(n):
            nb = adj[off[u]:off[u + 1]]
            if len(nb) == 0:
                continue
            nb_sorted = sorted(nb, key=lambda v: rank[v])
            pcur = sum(rank[v] < rank[u] for v in nb)
            costs = []
            for p in range(len(nb) + 1):
                g.order_apply(_place(rank, u, nb_sorted, p))
                costs.append(g.cost(alg))
            best = min(costs)
            want_p = pcur if costs[pcur] == best else costs.index(best)
            got = synth.orderings.neigh_move_one(off, adj, rank, u, objective)
            g.order_apply(got)
            assert g.cost(alg) == best
            assert np.array_equal(got, rank if want_p == pcur else _place(rank, u, nb_sorted, want_p))
            moved += want_p != pcur
    assert moved > 20


def test_neigh_for_cpp_lowers_cpp_and_reaches_the_star_bound():
    n = 3000
    e = synth.chung_lu(n, 16, 2.3, 8)
    off, adj = synth.simple_csr(n, e)
    g = oracle.Graph(n, e)
    g.order_apply(synth.order_degree(off))
    c_deg = g.cost(oracle.APP)
    rank, trace = synth.order_neigh(off, adj, objective="C++")
    assert np.array_equal(np.sort(rank), np.arange(n))
    assert trace[0] == c_deg
    assert all(b <= a for a, b in zip(trace, trace[1:]))
    g.order_apply(rank)
    assert g.cost(oracle.APP) == trace[-1] < c_deg
    # a star with its hub first has C++ = (n-1)^2; every edge adds at least
    # one to C++ (C++ >= m), and Neigh brings it down to that bound
    k = 200
    star = np.array([(0, v) for v in range(1, k)], dtype=np.uint32)
    off, adj = synth.simple_csr(k, star)
    hub_first = np.arange(k, dtype=np.uint32)
    rank, trace = synth.order_neigh(off, adj, start=hub_first, objective="C++")
    assert trace[0] == (k - 1) ** 2 and trace[-1] == k - 1
    g = oracle.Graph(k, star)
    g.order_apply(rank)
    assert g.cost(oracle.APP) == k - 1
