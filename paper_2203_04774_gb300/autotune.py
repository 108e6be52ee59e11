"""Autotuner of the listing's work split, picked per work profile.

The work split (``tl_tuning``: which kernel takes each B vertex, the piece
and task sizes) changes the speed of a listing, never its triangles or probe
count.  The best split depends on how the listing's work is distributed over
probe-set sizes, so a graph is described by its *work profile*
(``tl_work_profile``): the share of the membership tests (the cost of
Sec. 3.1, by Property 1) held by B vertices of each bit length of p (the
probe-set size) and of W (the vertex's tests).

* ``tune(g, alg)`` measures: a coordinate search from the defaults, one field
  at a time over its candidate values, each candidate timed by the listing
  kernels' CUDA-event time (``tl_last_list_stats``), keeping the fastest.
* A table (``tuning_table.json`` beside this file) holds tuned entries of
  measured workloads: the profile, the size, the tuning and both times.
* ``lookup(g, alg)`` returns the tuning of the nearest entry (L1 distance of
  the two profile marginals plus the difference of log2 m over 8) and
  ``apply`` sets it on the graph.

``python -m paper_2203_04774_gb300.autotune --out PATH WORKLOAD...`` builds
table entries for the seeded workloads named (rmat20, chunglu1e8, batch4096)
on the current GPU.
"""
from __future__ import annotations

import json
import math
import os
import statistics

import numpy as np

from . import (TL_AMM, TL_APM, TL_APP, tl_default_tuning, tl_graph_size, tl_last_list_stats,
               tl_list_triangles, tl_set_tuning, tl_work_profile)

TABLE_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning_table.json")
ALG_NAMES = {TL_APP: "A++", TL_APM: "A+-", TL_AMM: "A--"}

# Candidate values of each field, searched in this order.
CANDIDATES = [
    ("warp_work", [4096, 2048, 1024, 512]),
    ("narrow_piece", [1 << 14, 1 << 16, 1 << 18]),
    ("large_per_p", [64, 16, 256]),
    ("mid_piece", [1 << 16, 1 << 18]),
    ("narrow_max_p", [256, 128]),
    ("mid_max_p", [2048, 1024]),
    ("medium_max_p", [1024, 256]),
    ("narrow_keep_mib", [0, 64]),
    ("narrow_cold_first", [0, 1]),
    ("large_hash_max_p", [16384, 0]),
]


def profile(g, alg: int, x_begin: int = 0, x_end: int | None = None) -> dict:
    """The work profile as shares: by bit length of p and by bit length of W."""
    h = tl_work_profile(g, alg, x_begin, x_end).astype(np.float64)
    tot = h.sum()
    n, m = tl_graph_size(g)
    if tot == 0:
        zp, zw = np.zeros(h.shape[0]), np.zeros(h.shape[1])
        return {"p": zp.tolist(), "w": zw.tolist(), "work": 0, "n": n, "m": m}
    return {"p": (h.sum(axis=1) / tot).tolist(), "w": (h.sum(axis=0) / tot).tolist(),
            "work": int(tot), "n": n, "m": m}


def distance(a: dict, b: dict) -> float:
    dp = float(np.abs(np.asarray(a["p"]) - np.asarray(b["p"])).sum())
    dw = float(np.abs(np.asarray(a["w"]) - np.asarray(b["w"])).sum())
    dm = abs(math.log2(max(a["m"], 1)) - math.log2(max(b["m"], 1))) / 8.0
    return dp + dw + dm


def time_listing(g, alg: int, tuning: dict | None, reps: int = 1,
                 chunk_bytes: int = 1 << 30) -> tuple[float, int]:
    """Median listing-kernel milliseconds under `tuning` (None: defaults),
    and the triangle count (the same under every tuning)."""
    tl_set_tuning(g, None)
    if tuning:
        tl_set_tuning(g, tuning)
    ms, count = [], None
    for _ in range(reps):
        nt = tl_list_triangles(g, alg, chunk_bytes)
        ms.append(sum(tl_last_list_stats(g)["kernel_ms"]))
        if count is not None and nt != count:
            raise RuntimeError("the triangle count changed between runs")
        count = nt
    return statistics.median(ms), count


def tune(g, alg: int, reps: int = 1, chunk_bytes: int = 1 << 30, log=None) -> dict:
    """Coordinate search of the work split for this graph and algorithm;
    returns a table entry.  The graph is left with the defaults."""
    best = {}
    base_ms, count = time_listing(g, alg, None, reps, chunk_bytes)
    best_ms = base_ms
    trials = [({}, base_ms)]
    defaults = tl_default_tuning()
    for field, values in CANDIDATES:
        for v in values:
            if v == best.get(field, defaults[field]):
                continue
            trial = dict(best, **{field: v})
            ms, c = time_listing(g, alg, trial, reps, chunk_bytes)
            if c != count:
                raise RuntimeError(f"tuning {trial} changed the triangle count")
            trials.append((trial, ms))
            if log:
                log(f"[autotune] {ALG_NAMES[alg]} {trial}: {ms:.1f} ms")
            if ms < best_ms:
                best_ms, best = ms, trial
    tl_set_tuning(g, None)
    return {"alg": ALG_NAMES[alg], "profile": profile(g, alg), "tuning": best,
            "ms": best_ms, "default_ms": base_ms, "triangles": count,
            "trials": [[t, round(ms, 3)] for t, ms in trials]}


def load_table(path: str = TABLE_PATH) -> list:
    if not os.path.exists(path):
        return []
    with open(path) as f:
        return json.load(f)["entries"]


def lookup(g, alg: int, table: list | None = None, x_begin: int = 0,
           x_end: int | None = None) -> tuple[dict, dict | None]:
    """(tuning, entry) of the table entry nearest to this listing's profile
    for the same algorithm; ({}, None) when the table has none."""
    table = load_table() if table is None else table
    return nearest(profile(g, alg, x_begin, x_end), alg, table)


def nearest(prof: dict, alg: int, table: list) -> tuple[dict, dict | None]:
    """(tuning, entry) of the entry of `table` for `alg` nearest to `prof`."""
    cands = [e for e in table if e["alg"] == ALG_NAMES[alg]]
    if not cands:
        return {}, None
    e = min(cands, key=lambda e: distance(prof, e["profile"]))
    return dict(e["tuning"]), e


def apply(g, alg: int, table: list | None = None) -> dict:
    """Set the looked-up tuning on g (the defaults when nothing matches)."""
    tuning, _ = lookup(g, alg, table)
    tl_set_tuning(g, None)
    if tuning:
        tl_set_tuning(g, tuning)
    return tuning


# ---- building table entries for the seeded workloads -------------------------

def _workload_graph(name: str):
    """A loaded, degree-ordered graph of a seeded workload (device inputs)."""
    import torch

    from . import (TL_ORDER_DEGREE, tl_graph_load, tl_graph_load_parts, tl_order_apply,
                   tl_order_compute)
    from . import synth
    from .synth import device as sdev
    if name == "rmat20":
        e = torch.from_numpy(synth.rmat(20, 16, 0.57, 0.19, 0.19, 2)).cuda()
        n = 1 << 20
        g = tl_graph_load(n, e)
    elif name == "chunglu1e8":
        n = 100_000_000
        e = sdev.chung_lu_device(n, 40, 2.2, 4)
        g = tl_graph_load(n, e)
    elif name == "batch4096":
        fam = synth.chung_lu_family(4096, (1000, 200000), (8, 64), (2.1, 3.0), 3)
        parts = [sdev.chung_lu_device(int(fam["n"][i]), float(fam["deg"][i]),
                                      float(fam["gamma"][i]), int(fam["seeds"][i]))
                 for i in range(4096)]
        e = torch.cat(parts)
        del parts
        n = int(fam["n"].sum())
        g = tl_graph_load_parts(fam["n"], fam["pairs"], e)
    else:
        raise ValueError(f"unknown workload {name}")
    del e
    rank = torch.empty(n, dtype=torch.int32, device="cuda")
    tl_order_compute(g, TL_ORDER_DEGREE, rank)
    tl_order_apply(g, rank)
    return g


def main(argv=None):
    import argparse
    import sys

    from . import tl_graph_free
    ap = argparse.ArgumentParser(description="tune the work split of seeded workloads")
    ap.add_argument("workloads", nargs="+", choices=["rmat20", "chunglu1e8", "batch4096"])
    ap.add_argument("--algs", default="0,1", help="0: A++, 1: A+-, 2: A--")
    ap.add_argument("--reps", type=int, default=1)
    ap.add_argument("--out", required=True)
    args = ap.parse_args(argv)
    entries = []
    for name in args.workloads:
        g = _workload_graph(name)
        try:
            for alg in [int(a) for a in args.algs.split(",")]:
                e = tune(g, alg, args.reps, log=lambda *a: print(*a, file=sys.stderr, flush=True))
                e["workload"] = name
                entries.append(e)
        finally:
            tl_graph_free(g)
    with open(args.out, "w") as f:
        json.dump({"entries": entries}, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
