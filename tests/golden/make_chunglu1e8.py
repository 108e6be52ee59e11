#!/usr/bin/env python3
"""Writes tests/golden/chunglu1e8.json: the CPU oracle's listing of the
largest workload, a Chung-Lu graph with n = 10^8 vertices, exponent 2.2,
average degree 40 and seed 4 (about 2 * 10^9 undirected edges), under the
degree ordering (non-decreasing degree, ties by id; Sec. 2.2).

Only the oracle (oracle/) and the seeded input generator run here.  The
oracle's outer loop over seed vertices is split into disjoint rank ranges
listed concurrently on all host cores: the iterations of the outer loop are
independent (Algorithms 1 and 2 of Sec. 2.1), so the ranges' counts, set
hashes and probe counts add up to those of the whole listing (pinned by
test_seed_ranges_partition_the_listing and
test_lazy_dag_and_concurrent_listing).

Recorded: m (edges after the cleaning of Sec. 4.1), the triangle count T
and set hash H of Algorithm 1 (A++) and of Algorithm 2 (A+-), their probe
counts, and the costs C++ and C+- of the ordering (Sec. 3.1; Property 1
makes probes equal cost).  The triangle set does not depend on the
ordering, so (T, H) hold for every ordering.

Usage: python tests/golden/make_chunglu1e8.py [--n N --out PATH] (a smaller
n writes a file of the same form for a quick trial).  Needs about 40 GB of
host memory at n = 10^8.
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import sys
import time
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2203_04774_gb300 import synth  # noqa: E402


def log(*a):
    print(f"[{time.strftime('%H:%M:%S')}]", *a, file=sys.stderr, flush=True)


def list_parallel(g, alg, n, threads, weight, parts=4096):
    """(count, hash, probes) of the whole listing as the sum over disjoint
    seed-rank ranges.  The ranges hold about equal shares of `weight` (a
    per-rank estimate of the work) and the heaviest go first, so that no
    single range keeps one thread busy after the others are done."""
    cum = np.cumsum(weight, dtype=np.float64)
    cuts = np.searchsorted(cum, np.linspace(0, cum[-1], parts + 1)[1:-1], side="right")
    cuts = np.unique(np.concatenate([[0], cuts, [n]])).astype(np.int64)
    ranges = list(zip(cuts[:-1].tolist(), cuts[1:].tolist()))
    share = [cum[b - 1] - (cum[a - 1] if a else 0.0) for a, b in ranges]
    ranges = [r for _, r in sorted(zip(share, ranges), reverse=True)]
    done = [0]
    t0 = time.time()

    def one(r):
        out = g.list(alg, oracle.LITERAL, int(r[0]), int(r[1]), store=False)
        done[0] += 1
        if done[0] % 256 == 0:
            log(f"  alg {alg}: {done[0]}/{len(ranges)} ranges, {time.time() - t0:.0f} s")
        return out[1:]

    with ThreadPoolExecutor(threads) as ex:
        res = list(ex.map(one, ranges))
    count = sum(r[0] for r in res)
    hsh = sum(r[1] for r in res) % (1 << 64)
    probes = sum(r[2] for r in res)
    return count, hsh, probes, time.time() - t0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=100_000_000)
    ap.add_argument("--avg-degree", type=float, default=40)
    ap.add_argument("--exponent", type=float, default=2.2)
    ap.add_argument("--seed", type=int, default=4)
    ap.add_argument("--threads", type=int, default=os.cpu_count())
    ap.add_argument("--out", default=os.path.join(HERE, "chunglu1e8.json"))
    args = ap.parse_args()
    n = args.n
    t_all = time.time()
    log(f"drawing Chung-Lu n={n} d={args.avg_degree} gamma={args.exponent} seed={args.seed}")
    e = synth.chung_lu(n, args.avg_degree, args.exponent, args.seed, threads=args.threads)
    pairs = int(e.shape[0])
    log(f"{pairs} pairs; loading into the oracle")
    g = oracle.Graph(n, e)
    del e
    m = g.m
    log(f"m = {m}; degree ordering")
    deg = g.degrees()
    rank = synth.order_degree_from_degrees(deg)
    g.order_apply(rank)
    del rank
    # per-rank work estimate: under the degree ordering the vertex at rank r
    # has the r-th smallest degree d, and its work grows about as d^2
    weight = np.sort(deg).astype(np.float64) ** 2 + 1.0
    del deg
    c_pp, c_pm = g.cost(oracle.APP), g.cost(oracle.APM)
    log(f"C++ = {c_pp}, C+- = {c_pm}")
    res = {}
    for alg, name in ((oracle.APP, "A++"), (oracle.APM, "A+-")):
        cnt, hsh, probes, dt = list_parallel(g, alg, n, args.threads, weight)
        log(f"{name}: T = {cnt}, H = {hsh:#018x}, probes = {probes}, {dt:.0f} s")
        res[name] = {"triangles": cnt, "hash": f"{hsh:#018x}", "probes": probes,
                     "seconds": round(dt, 1)}
    assert res["A++"]["triangles"] == res["A+-"]["triangles"]
    assert res["A++"]["hash"] == res["A+-"]["hash"]
    assert res["A++"]["probes"] == c_pp and res["A+-"]["probes"] == c_pm  # Property 1
    out = {
        "workload": "Chung-Lu power-law graph (synth.chung_lu)",
        "n": n, "avg_degree": args.avg_degree, "exponent": args.exponent, "seed": args.seed,
        "pairs": pairs, "m": m,
        "ordering": "degree (non-decreasing, ties by id; Sec. 2.2)",
        "C_pp": c_pp, "C_pm": c_pm,
        "triangles": res["A++"]["triangles"], "hash": res["A++"]["hash"],
        "listings": res,
        "hash_definition": "sum over triangles a<b<c (original ids) of "
                           "mix(mix(mix(a+G)+b+G)+c+G) mod 2^64, G = 0x9e3779b97f4a7c15, "
                           "mix = splitmix64 finaliser",
        "produced_by": "tests/golden/make_chunglu1e8.py (oracle/ only, literal Algorithms 1 "
                       "and 2 over disjoint seed-rank ranges)",
        "host": {"machine": platform.machine(), "cpus": os.cpu_count(),
                 "threads": args.threads, "numpy": np.__version__},
        "seconds_total": round(time.time() - t_all, 1),
    }
    with open(args.out, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    log(f"wrote {args.out} in {time.time() - t_all:.0f} s")


if __name__ == "__main__":
    main()
