"""The request server (tl_server_*): every request's result equals the graph's
own result alone and the oracle's, however requests are batched together;
admission by footprint; argument errors.  Every call goes through the C ABI."""
import threading

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


@pytest.fixture(scope="module")
def pool():
    """24 graphs of uneven size, two orderings each (degree; random or core),
    with the oracle's (count, hash) for every (graph, ordering, algorithm)."""
    rng = np.random.default_rng(5)
    graphs = []
    for i in range(24):
        n = int(np.exp(rng.uniform(np.log(30), np.log(20000))))
        e = synth.chung_lu(n, float(rng.uniform(4, 40)), float(rng.uniform(2.1, 3.0)), 500 + i)
        off, adj = synth.simple_csr(n, e)
        orders = [synth.order_degree(off),
                  synth.order_core(off, adj) if i % 2 else synth.order_random(n, i)]
        want = {}
        ref = oracle.Graph(n, e)
        for o, r in enumerate(orders):
            ref.order_apply(r)
            for alg in (tl.TL_APP, tl.TL_APM, tl.TL_AMM):
                _, c, h, _ = ref.list(alg, store=False)
                want[(o, alg)] = (c, h)
        graphs.append((n, e, orders, want))
    return graphs


def _register(srv, pool):
    ids = []
    for n, e, orders, _ in pool:
        g = tl.Graph(n, _dev(e))
        gid = srv.add_graph(g)
        oids = [srv.add_ordering(gid, _dev(r)) for r in orders]
        ids.append((gid, oids))
    return ids


def _requests(pool, count, seed):
    rng = np.random.default_rng(seed)
    algs = (tl.TL_APP, tl.TL_APM, tl.TL_AMM)
    return [(int(rng.integers(len(pool))), int(rng.integers(2)), algs[int(rng.integers(3))])
            for _ in range(count)]


def _run(srv, ids, reqs):
    rids = [srv.submit(ids[p][0], ids[p][1][o], a) for p, o, a in reqs]
    return [srv.wait(r) for r in rids]


@pytest.mark.parametrize("max_batch,workers", [(64, 2), (1, 1), (7, 3)])
def test_every_request_matches_the_oracle_in_any_mix(pool, max_batch, workers):
    srv = tl.Server(64 << 30, max_batch=max_batch, workers=workers)
    ids = _register(srv, pool)
    reqs = _requests(pool, 150, 1)
    res = _run(srv, ids, reqs)
    for (p, o, a), r in zip(reqs, res):
        assert r["status"] == tl.TL_OK
        assert (r["triangles"], r["hash"]) == pool[p][3][(o, a)], (p, o, a)
        assert r["t_submit_ns"] <= r["t_admit_ns"] <= r["t_done_ns"]
        assert 1 <= r["batch_size"] <= max_batch
    sizes = [r["batch_size"] for r in res]
    if max_batch > 1:
        assert max(sizes) > 1  # requests submitted together were listed together
    srv.close()


def test_concurrent_clients(pool):
    srv = tl.Server(64 << 30, max_batch=32, workers=2)
    ids = _register(srv, pool)
    out, errors = {}, []

    def client(c):
        try:
            reqs = _requests(pool, 40, 100 + c)
            out[c] = (reqs, _run(srv, ids, reqs))
        except BaseException as e:  # surfaced below
            errors.append(e)

    threads = [threading.Thread(target=client, args=(c,)) for c in range(4)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    for reqs, res in out.values():
        for (p, o, a), r in zip(reqs, res):
            assert (r["status"], r["triangles"], r["hash"]) == (tl.TL_OK,) + pool[p][3][(o, a)]
    srv.close()


def test_admission_by_footprint(pool):
    # a budget that holds one batch of the largest graph's request but not
    # more: requests still all finish (they wait for memory), in order
    probe = tl.Server(64 << 30, max_batch=64, workers=2)
    ids = _register(probe, pool)
    big = int(np.argmax([p[0] for p in pool]))
    req_bytes, batch_bytes = probe.footprint(ids[big][0])
    probe.close()
    srv = tl.Server(batch_bytes + req_bytes, max_batch=64, workers=2)
    ids = _register(srv, pool)
    reqs = _requests(pool, 60, 2) + [(big, 0, tl.TL_APP)] * 3
    res = _run(srv, ids, reqs)
    for (p, o, a), r in zip(reqs, res):
        assert (r["status"], r["triangles"], r["hash"]) == (tl.TL_OK,) + pool[p][3][(o, a)]
    for r in res[-3:]:
        assert r["batch_size"] == 1  # the largest request fills the budget alone
    srv.close()
    # a budget below one request of the largest graph: that request fails with
    # TL_ENOMEM, smaller ones are served
    srv = tl.Server(batch_bytes + req_bytes - 1, max_batch=64, workers=2)
    ids = _register(srv, pool)
    small = int(np.argmin([p[0] for p in pool]))
    res = _run(srv, ids, [(big, 0, tl.TL_APM), (small, 1, tl.TL_APP)])
    assert res[0]["status"] == tl.TL_ENOMEM
    assert (res[1]["status"], res[1]["triangles"]) == (tl.TL_OK, pool[small][3][(1, tl.TL_APP)][0])
    srv.close()


def test_server_argument_errors(pool):
    srv = tl.Server(8 << 30, max_batch=4, workers=1)
    n, e, orders, _ = pool[0]
    g = tl.Graph(n, _dev(e))
    gid = srv.add_graph(g)
    bad = orders[0].copy()
    bad[0] = bad[1]
    with pytest.raises(tl.TLError) as ei:
        srv.add_ordering(gid, _dev(bad))
    assert ei.value.status == tl.TL_EINVAL
    oid = srv.add_ordering(gid, orders[0])  # host pointer
    with pytest.raises(tl.TLError):
        srv.submit(gid + 1, oid, tl.TL_APP)
    with pytest.raises(tl.TLError):
        srv.submit(gid, oid + 1, tl.TL_APP)
    with pytest.raises(tl.TLError):
        srv.wait(12345)
    r = srv.wait(srv.submit(gid, oid, tl.TL_APP))
    assert (r["triangles"], r["hash"]) == pool[0][3][(0, tl.TL_APP)]
    srv.close()


def test_one_waiter_per_request(pool):
    """Two threads wait for the same request: one gets its result, the other
    TL_EINVAL (the id is either being waited for or already consumed)."""
    srv = tl.Server(8 << 30, max_batch=4, workers=1)
    n, e, orders, want = pool[-1]
    g = tl.Graph(n, _dev(e))
    gid = srv.add_graph(g)
    oid = srv.add_ordering(gid, _dev(orders[0]))
    rid = srv.submit(gid, oid, tl.TL_APM)
    got, errs = [], []

    def waiter():
        try:
            got.append(srv.wait(rid))
        except tl.TLError as ex:
            errs.append(ex.status)

    threads = [threading.Thread(target=waiter) for _ in range(2)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert errs == [tl.TL_EINVAL] and len(got) == 1
    assert (got[0]["triangles"], got[0]["hash"]) == want[(0, tl.TL_APM)]
    srv.close()


def test_tuning_table_by_profile(pool):
    """With a table of work splits the server picks, per algorithm group of a
    batch, the entry nearest to the group's work profile: results stay the
    oracle's, and a one-request batch takes the entry autotune.nearest picks
    for that graph alone."""
    import torch

    from paper_2203_04774_gb300 import autotune

    def entry(alg, p_bin, tuning):
        p = np.zeros(tl.TL_PROFILE_BINS_P)
        w = np.zeros(tl.TL_PROFILE_BINS_W)
        p[p_bin] = 1.0
        w[12] = 1.0
        return {"alg": alg, "tuning": tuning,
                "profile": {"p": p.tolist(), "w": w.tolist(), "m": 1 << 16, "n": 1 << 12}}
    table = [entry("A++", 3, {"warp_work": 256, "narrow_piece": 1024}),
             entry("A++", 9, {"mid_max_p": 64, "large_per_p": 1, "large_min": 1024,
                              "large_max": 4096}),
             entry("A+-", 5, {"narrow_max_p": 16, "small_max_p": 4}),
             entry("A--", 2, {"medium_max_p": 0})]
    srv = tl.Server(64 << 30, max_batch=1, workers=1)
    srv.set_tuning_table(table)
    ids = _register(srv, pool)
    reqs = _requests(pool, 60, 7)
    res = _run(srv, ids, reqs)
    for (p, o, a), r in zip(reqs, res):
        n, e, orders, want = pool[p]
        assert (r["triangles"], r["hash"]) == want[(o, a)]
        g = tl.Graph(n, _dev(e))
        g.order_apply(torch.from_numpy(orders[o]).cuda())
        _, chosen = autotune.lookup(g.h, a, table)
        assert r["tuning_entry"] == (table.index(chosen) if chosen else -1), (p, o, a)
        g.free()
    srv.set_tuning_table(None)
    r2 = _run(srv, ids, reqs[:10])
    assert all(x["tuning_entry"] == -1 for x in r2)
    srv.close()
