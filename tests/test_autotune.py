"""The autotuner of the work split: table lookup by work profile (CPU), and
on the GPU the profile's total (the cost, by Property 1), a tuning search
that keeps the triangle count, and the looked-up split applied to a graph."""
import numpy as np
import pytest

import paper_2203_04774_gb300 as tl
from paper_2203_04774_gb300 import autotune


def _prof(p_bin, w_bin, m):
    p = np.zeros(tl.TL_PROFILE_BINS_P)
    w = np.zeros(tl.TL_PROFILE_BINS_W)
    p[p_bin] = 1.0
    w[w_bin] = 1.0
    return {"p": p.tolist(), "w": w.tolist(), "m": m, "n": m // 10, "work": 1}


def test_nearest_entry_by_profile_and_size():
    table = [
        {"alg": "A+-", "profile": _prof(6, 14, 1 << 30), "tuning": {"warp_work": 1024}},
        {"alg": "A+-", "profile": _prof(12, 20, 1 << 24), "tuning": {"mid_piece": 1 << 18}},
        {"alg": "A++", "profile": _prof(6, 14, 1 << 30), "tuning": {"large_per_p": 16}},
    ]
    assert autotune.nearest(_prof(6, 14, 1 << 29), tl.TL_APM, table)[0] == {"warp_work": 1024}
    assert autotune.nearest(_prof(11, 20, 1 << 24), tl.TL_APM, table)[0] == {"mid_piece": 1 << 18}
    assert autotune.nearest(_prof(6, 14, 1 << 29), tl.TL_APP, table)[0] == {"large_per_p": 16}
    assert autotune.nearest(_prof(6, 14, 1 << 29), tl.TL_AMM, table) == ({}, None)
    assert autotune.distance(_prof(3, 3, 100), _prof(3, 3, 100)) == 0.0


def test_committed_table_is_well_formed():
    defaults = set(tl.Tuning().as_dict())
    for e in autotune.load_table():
        assert e["alg"] in ("A++", "A+-", "A--")
        assert set(e["tuning"]) <= defaults
        assert len(e["profile"]["p"]) == tl.TL_PROFILE_BINS_P
        assert len(e["profile"]["w"]) == tl.TL_PROFILE_BINS_W
        assert abs(sum(e["profile"]["p"]) - 1) < 1e-9 and e["ms"] <= e["default_ms"]


@pytest.mark.gpu
def test_profile_search_and_apply_on_the_gpu():
    import torch

    import oracle
    from paper_2203_04774_gb300 import synth
    torch.cuda.set_device(0)
    n = 40000
    e = synth.chung_lu(n, 24, 2.2, 12)
    rank = synth.order_degree(synth.simple_csr(n, e)[0])
    g = tl.Graph(n, torch.from_numpy(e).cuda())
    g.order_apply(torch.from_numpy(rank).cuda())
    ref = oracle.Graph(n, e)
    ref.order_apply(rank)
    for alg in (tl.TL_APP, tl.TL_APM):
        h = tl.tl_work_profile(g.h, alg)
        assert int(h.sum()) == ref.cost(alg)  # the profile holds every test (Property 1)
        half = tl.tl_work_profile(g.h, alg, 0, n // 2)
        assert int(half.sum()) == ref.list(alg, seed_begin=0, seed_end=n // 2, store=False)[3]
        entry = autotune.tune(g.h, alg, chunk_bytes=tl.TL_MIN_CHUNK_BYTES)
        assert entry["triangles"] == ref.list(alg, store=False)[1]
        assert entry["ms"] <= entry["default_ms"]
        got = autotune.apply(g.h, alg, [entry])
        assert got == entry["tuning"]
        assert tl.tl_get_tuning(g.h) == dict(tl.tl_default_tuning(), **entry["tuning"])
        _, nt, probes, _ = g.list_collect(alg)
        assert (nt, probes) == (entry["triangles"], ref.cost(alg))
    g.free()
