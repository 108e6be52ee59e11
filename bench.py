#!/usr/bin/env python3
"""Benchmark of the triangle-listing hot path on one GB300 (one JSON line).

Headline workload (the paper's largest scale): a Chung-Lu power-law graph
with n = 10^8 vertices, exponent 2.2, average degree 40, seed 4 (2 * 10^9
pairs, about 1.99 * 10^9 undirected edges after cleaning), generated on the
device, degree ordering (ties by id) computed on the device before timing.
One step runs the whole path once: graph_load (a1) -> order_apply (a2-a5:
relabel, orient, CSR, cost) -> list_triangles A++ and list_triangles A+-
(a6-a9), each listing streamed in 1 GiB chunks to the library's device
count + hash consumer.

value: triangles listed per second of device time over the timed steps
(both algorithms list the same T triangles; a step lists 2T).  e2e: the
same step through the C ABI from pinned host buffers (edges and ranks
copied in every step, the count and hash read back), wall clock.
roofline: the listing kernels' algorithmic bytes 4 (C + m) + 12 T per
listing over their summed CUDA-event time.  cpu_baseline: the CPU oracle
(literal Algorithms 1 and 2, one thread) on a stated sample of seed ranks of
the same graph and ordering, built in a separate process while the GPU
runs.

With no --workload the line also carries the other workloads as
sub-objects: "rmat20" (R-MAT scale 20, with the per-ordering cost-vs-time
sweep), "batch4096" (4,096 graphs: one disjoint-union pass vs one pass per
graph) and "serve" (Poisson request stream: batched vs one request per
pass).  --workload X runs one of them alone as the line's headline.

--impl reference times the CPU oracle as the reference arm on the headline
workload (the reference is a paper; the oracle stands in for its code).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "triangles/s"
DEFAULT_CHUNK_MB = 1024
FALLBACK_HBM_GBS = 6800.0
NOMINAL_HBM_GBS = 8000.0  # the nominal HBM3e figure, reported beside the measured one
CHUNK_BYTES = DEFAULT_CHUNK_MB << 20

WORKLOADS = {
    "chunglu1e8": {"workload": "chunglu1e8-degree", "generator": "Chung-Lu", "n": 100_000_000,
                   "avg_degree": 40, "exponent": 2.2, "seed": 4,
                   "ordering": "degree (ties by id), computed on the device",
                   "algorithms": ["A++", "A+-"]},
    # the same family at n = 8e6 (1.6e8 pairs, a few GB on the device): the
    # small case for full profiler captures of the listing kernels
    "chunglu8e6": {"workload": "chunglu8e6-degree", "generator": "Chung-Lu", "n": 8_000_000,
                   "avg_degree": 40, "exponent": 2.2, "seed": 4,
                   "ordering": "degree (ties by id), computed on the device",
                   "algorithms": ["A++", "A+-"]},
    "rmat20": {"workload": "rmat20-degree", "generator": "R-MAT", "scale": 20, "edge_factor": 16,
               "abcd": [0.57, 0.19, 0.19, 0.05], "seed": 2, "ordering": "degree (ties by id)",
               "algorithms": ["A++", "A+-"]},
}
DATA = {"Chung-Lu": "synthetic (seeded Chung-Lu power-law graph generated on the device; the "
                    "paper's datasets are not available)",
        "R-MAT": "synthetic (seeded R-MAT; the paper's datasets are not available)"}

# The oracle sample of a workload: seed ranks [k n/16, k n/16 + n/(16 S)) for
# k = 0..15, both algorithms, literal form, one thread.  S is chosen per
# workload for about 1-3 s of CPU work per sample; cpu_baseline repeats the
# sample, the reference arm times one sample per step.
ORACLE_SAMPLE_DIV = {"chunglu1e8": 2048, "chunglu8e6": 256, "rmat20": 64}


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def code_only(src: str) -> str:
    """C++ source without comments, blank lines and trailing spaces."""
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    return "\n".join(line.rstrip() for line in src.splitlines() if line.strip())


def list_source_hash():
    """Hash of the listing kernels' code (list.cu + list.cuh, comments ignored):
    recorded DRAM counters are used only while it matches."""
    h = hashlib.sha256()
    for f in ("list.cu", "list.cuh"):
        with open(os.path.join(ROOT, "paper_2203_04774_gb300", "csrc", f)) as fh:
            h.update(code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def recorded_traffic(workload: str):
    """DRAM bytes per step of the listing kernels from the committed ncu
    summary of this workload, if it was taken on the current listing kernels
    (else None).  A summary of a smaller case of the same workload scales to
    the full one by its stated factor."""
    p = os.path.join(ROOT, "profiles", f"list_{workload}_traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
        if d.get("list_source_sha256_16") != list_source_hash():
            return None
        return int(d["dram_bytes_per_step"] * d.get("scale_to_workload", 1.0))
    except Exception:
        return None


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None
        self.out = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            if self.out:
                self.out.close()

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# ---- the CPU oracle: sampled listing (cpu_baseline and the reference arm) ----

def sample_ranges(n: int, div: int):
    """Seed-rank ranges [k n/16, k n/16 + n/(16 div)), k = 0..15."""
    step = n // 16
    width = max(1, step // div)
    return [(k * step, k * step + width) for k in range(16)]


def host_inputs(key: str, threads: int = 1):
    """(n, raw edge pairs, degree-ordering ranks) of a workload on the host,
    from the same seeded generators as the device path."""
    from paper_2203_04774_gb300 import synth
    wl = WORKLOADS[key]
    if wl["generator"] == "R-MAT":
        e = synth.rmat(wl["scale"], wl["edge_factor"], *wl["abcd"][:3], wl["seed"])
        n = 1 << wl["scale"]
        return n, e, synth.order_degree_from_degrees(synth.simple_degrees(n, e))
    n = wl["n"]
    e = synth.chung_lu(n, wl["avg_degree"], wl["exponent"], wl["seed"], threads=threads)
    return n, e, None


def oracle_graph(key: str, threads: int = 1):
    """The oracle's graph of a workload under the degree ordering, and the
    seconds taken to draw, load and order it."""
    import oracle
    from paper_2203_04774_gb300 import synth
    t0 = time.perf_counter()
    n, e, rank = host_inputs(key, threads)
    g = oracle.Graph(n, e)
    del e
    if rank is None:  # degrees of the cleaned graph, then the degree ordering
        rank = synth.order_degree_from_degrees(g.degrees())
    g.order_apply(rank)
    return g, n, time.perf_counter() - t0


def oracle_sample(g, n: int, div: int, threads: int = 1) -> int:
    """One sample: both algorithms (literal form) over the sample ranges;
    returns the triangles listed.  With threads > 1 the ranges, each cut
    into eight equal parts, are listed concurrently (the iterations of the
    outer loop of Algorithms 1 and 2 are independent; the oracle's listing
    is safe to call from several threads)."""
    import oracle
    tasks = []
    for alg in (oracle.APP, oracle.APM):
        for a, b in sample_ranges(n, div):
            if threads == 1:
                tasks.append((alg, a, b))
                continue
            cuts = np.linspace(a, b, 9).astype(np.int64)
            tasks += [(alg, int(c0), int(c1)) for c0, c1 in zip(cuts[:-1], cuts[1:]) if c1 > c0]

    def one(t):
        return g.list(t[0], oracle.LITERAL, t[1], t[2], store=False)[1]

    if threads == 1:
        return sum(one(t) for t in tasks)
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(threads) as ex:
        return sum(ex.map(one, tasks))


def oracle_threads(key: str) -> int:
    """Host threads of the oracle's timed sample: all cores for the 2e9-edge
    graph (its seed ranges listed concurrently), one for the others (the
    paper's single-threaded protocol)."""
    return (os.cpu_count() or 1) if key == "chunglu1e8" else 1


def sample_text(key: str, div: int, threads: int = 1) -> str:
    how = "one thread" if threads == 1 else f"{threads} threads listing parts of the ranges concurrently"
    return (f"CPU oracle, Algorithms 1 and 2 in the literal boolean-array form, {how}, "
            f"seed ranks [k n/16, k n/16 + n/{16 * div}) for k = 0..15 ({1 / div:.4g} of the "
            f"seed vertices) of the {WORKLOADS[key]['workload']} graph under the same degree "
            f"ordering; listing only (the graph is built first, untimed)")


def cpu_baseline_of(g, n: int, key: str, min_s: float = 10.0) -> dict:
    div = ORACLE_SAMPLE_DIV[key]
    threads = oracle_threads(key)
    tri, reps = 0, 0
    t0 = time.perf_counter()
    while reps == 0 or time.perf_counter() - t0 < min_s:
        tri += oracle_sample(g, n, div, threads)
        reps += 1
    dt = time.perf_counter() - t0
    return {"value": tri / dt, "unit": "triangles/s", "cores": threads, "kind": "oracle",
            "sample": sample_text(key, div, threads) +
                      f"; {reps} samples, {tri} triangles in {dt:.1f} s"}


def _oracle_worker(conn, key: str, threads: int):
    """Runs in a spawned process: build the oracle's graph of the workload
    (on the host, while the GPU runs); when the parent says the GPU work is
    done, time the sample and send the result."""
    try:
        g, n, build_s = oracle_graph(key, threads)
        if not conn.poll(7200):
            raise TimeoutError("no go-ahead from the bench within 7200 s")
        conn.recv()
        res = cpu_baseline_of(g, n, key)
        res["build_s"] = round(build_s, 1)
        conn.send(res)
    except BaseException as ex:  # report, never hang the parent
        conn.send({"unavailable": f"oracle worker failed: {type(ex).__name__}: {ex}"})
    finally:
        conn.close()


class OracleWorker:
    """The headline's cpu_baseline, computed in a spawned process started
    before the first CUDA call."""

    def __init__(self, key: str, threads: int = 8):
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        self.conn, child = ctx.Pipe(duplex=True)
        self.proc = ctx.Process(target=_oracle_worker, args=(child, key, threads), daemon=True)
        self.proc.start()
        child.close()

    def result(self, timeout_s: float = 1800.0) -> dict:
        """Called once the GPU work is done: lets the worker time its
        sample (the host cores are then free) and waits for it."""
        t0 = time.time()
        try:
            self.conn.send("go")
            if self.conn.poll(timeout_s):
                res = self.conn.recv()
            else:
                res = {"unavailable": f"oracle worker gave no result within {timeout_s:.0f} s"}
        except EOFError:
            res = {"unavailable": "oracle worker exited without a result"}
        self.proc.join(timeout=10)
        if self.proc.is_alive():
            self.proc.kill()
        res["waited_s"] = round(time.time() - t0, 1)
        return res


def run_reference(args, key: str):
    """The reference arm: the CPU oracle, one sample of the workload per
    step, on rank 0 only."""
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    g, n, build_s = oracle_graph(key, threads=os.cpu_count() or 1)
    div = ORACLE_SAMPLE_DIV[key]
    threads = oracle_threads(key)
    for _ in range(args.warmup):
        oracle_sample(g, n, div, threads)
    t0 = time.perf_counter()
    tri = sum(oracle_sample(g, n, div, threads) for _ in range(args.steps))
    dt = time.perf_counter() - t0
    value = tri / dt
    wl = WORKLOADS[key]
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "triangles/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": DATA[wl["generator"]],
        "config": dict(wl, n=n, m=g.m, chunk_bytes=CHUNK_BYTES,
                       l2="CPU run (no L2 flush)", oracle_build_s=round(build_s, 1)),
        "cpu_baseline": {"value": value, "unit": "triangles/s", "cores": threads, "kind": "oracle",
                         "sample": sample_text(key, div, threads) + "; one sample per step"},
        "e2e": {"value": value, "unit": "triangles/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0}}), flush=True)


# ---- one listing workload: load + order + A++ + A+- per step ------------------

def run_listing(args, key: str, steps: int, warmup: int, e2e: bool, orderings: bool,
                cpu: str | None, dist=None) -> dict:
    """Time `steps` whole-path steps of a workload; returns its JSON line.
    cpu: None (no baseline), "inline" (oracle timed here, after the GPU
    work) or an OracleWorker's result dict."""
    import torch

    import paper_2203_04774_gb300 as tl
    from paper_2203_04774_gb300 import autotune
    from paper_2203_04774_gb300.synth import device as sdev

    world, rank, local = dist_setup()
    wl = WORKLOADS[key]
    table = autotune.load_table()
    t0 = time.time()
    e_host = r_host = None
    if wl["generator"] == "Chung-Lu":
        n = wl["n"]
        e_dev = sdev.chung_lu_device(n, wl["avg_degree"], wl["exponent"], wl["seed"])
        g = tl.tl_graph_load(n, e_dev)
        try:
            r_dev = torch.empty(n, dtype=torch.int32, device="cuda")
            tl.tl_order_compute(g, tl.TL_ORDER_DEGREE, r_dev)
        finally:
            tl.tl_graph_free(g)
        if e2e:  # the same inputs in pinned host memory
            e_host = torch.empty(e_dev.shape, dtype=e_dev.dtype, pin_memory=True)
            e_host.copy_(e_dev)
            r_host = torch.empty(r_dev.shape, dtype=r_dev.dtype, pin_memory=True)
            r_host.copy_(r_dev)
    else:
        n, e, rnk = host_inputs(key)
        e_dev = torch.from_numpy(e).cuda()
        r_dev = torch.from_numpy(rnk.view(np.int32)).cuda()
        if e2e:
            e_host = torch.from_numpy(e).pin_memory()
            r_host = torch.from_numpy(rnk.view(np.int32)).pin_memory()
    torch.cuda.synchronize()
    log(f"[bench] {key}: inputs ready in {time.time() - t0:.1f}s: n={n} pairs={e_dev.shape[0]}")
    stream = torch.cuda.Stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    # the consumer reduces each chunk on its own stream, overlapping the
    # listing kernel that fills the other chunk buffer
    cstream = torch.cuda.Stream()
    ch = tl.CountHash(cstream.cuda_stream)
    ch_ptr = tl.tl_count_hash_ptr()

    phase_names = ["graph_load", "order_apply", "list_A++", "list_A+-", "graph_free"]
    phase_ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(phase_names) + 1)]
    phase_ms = {k: [] for k in phase_names}

    def step(edges, ranks):
        phase_ev[0].record(stream)
        g = tl.tl_graph_load(n, edges, stream.cuda_stream)
        phase_ev[1].record(stream)
        try:
            tl.tl_order_apply(g, ranks)
            phase_ev[2].record(stream)
            m = tl.tl_graph_size(g)[1]
            costs = [tl.tl_cost(g, a) for a in (tl.TL_APP, tl.TL_APM)]
            out = []
            for i, a in enumerate((tl.TL_APP, tl.TL_APM)):
                # the work split picked by the autotuner for this listing's
                # work profile (a profile kernel and a table lookup, timed)
                autotune.apply(g, a, table)
                ch.reset()
                nt = tl.tl_list_triangles(g, a, CHUNK_BYTES, ch_ptr, ch.user)
                phase_ev[3 + i].record(stream)
                out.append((nt, int(ch.state.count), int(ch.state.hash),
                            tl.tl_last_list_stats(g)))
            return m, costs, out
        finally:
            tl.tl_graph_free(g)
            phase_ev[5].record(stream)
            phase_ev[5].synchronize()
            for i, k in enumerate(phase_names):
                phase_ms[k].append(phase_ev[i].elapsed_time(phase_ev[i + 1]))

    def barrier():
        torch.cuda.synchronize()
        if dist:
            dist.barrier()

    for _ in range(warmup):
        step(e_dev, r_dev)
    # timed region (device), L2 flushed before every step
    clocks = Clocks(local)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    launches0 = tl.tl_kernel_launches()
    results = []
    barrier()
    clocks.start()
    for i in range(steps):
        flush.zero_()
        torch.cuda.synchronize()
        ev[i][0].record(stream)
        results.append(step(e_dev, r_dev))
        ev[i][1].record(stream)
    barrier()
    clk = clocks.stop()
    launches = tl.tl_kernel_launches() - launches0
    timed_phase_ms = {k: statistics.median(v[-steps:]) for k, v in phase_ms.items()}
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    if dist:
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    m, costs, out = results[-1]
    T = out[0][0]
    assert all(o[0] == T and o[1] == T for r in results for o in r[2]), "triangle counts differ"
    assert len({o[2] for r in results for o in r[2]}) == 1, "set hashes differ"
    tri_per_step = sum(o[0] for o in out)
    value = tri_per_step * steps * world / (total_ms / 1e3)

    # roofline of the listing kernels (both algorithms, all launches)
    list_ms = statistics.mean(sum(sum(o[3]["kernel_ms"]) for o in r[2]) for r in results)
    alg_bytes = sum(4 * (c + m) + 12 * T for c in costs)
    peak, peak_kind = read_peaks()
    achieved = alg_bytes / (list_ms / 1e3) / 1e9

    # end to end through the C ABI from pinned host buffers
    e2e_ms = []
    for _ in range(max(2, min(steps, 5)) if e2e else 0):
        flush.zero_()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        step(e_host, r_host)
        torch.cuda.synchronize()
        e2e_ms.append((time.perf_counter() - t1) * 1e3)
    e2e_value = tri_per_step * len(e2e_ms) / (sum(e2e_ms) / 1e3) if e2e_ms else None

    per_ordering = None
    if rank == 0 and orderings:
        e_np = e_dev.cpu().numpy().view(np.uint32)
        per_ordering = ordering_sweep(tl, n, e_np, e_dev, stream)
    ch.release()
    del e_dev, r_dev, e_host, r_host, flush
    torch.cuda.empty_cache()

    cpu_res = None
    if rank == 0 and world == 1 and cpu == "inline":
        g_or, n_or, _ = oracle_graph(key)
        cpu_res = cpu_baseline_of(g_or, n_or, key)
        del g_or
    elif isinstance(cpu, dict):
        cpu_res = cpu
    return {
        "metric": METRIC, "value": value, "unit": "triangles/s", "n_gpus": world,
        "steps": steps, "warmup": warmup, "ms_per_step": total_ms / steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": DATA[wl["generator"]],
        "config": dict(wl, n=n, m=m, triangles=T, C_pp=costs[0], C_pm=costs[1],
                       chunk_bytes=CHUNK_BYTES,
                       l2="inputs larger than L2, and a 256 MiB buffer written before each step",
                       parallelism="replicas" if world > 1 else "1 GPU"),
        "oriented_edges_per_s": m * 2 * steps * world / (total_ms / 1e3),
        "e2e": {"value": e2e_value, "unit": "triangles/s",
                "h2d_bytes_per_step": h2d_bytes(key, n) if e2e else None,
                "d2h_bytes_per_step": 2 * 16},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": recorded_traffic(key),
                     "nominal_peak": NOMINAL_HBM_GBS,
                     "frac_of_nominal": achieved / NOMINAL_HBM_GBS,
                     "kernel": "k_list_warp<64|2048> + k_list_cta<32|256|1024> (A++ and A+-)",
                     "algorithmic_bytes_per_step": alg_bytes, "kernel_ms_per_step": list_ms,
                     "compulsory_bytes_per_step": len(costs) * (8 * m + 12 * T),
                     "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)"},
        "list_stats": {a: r[3] for a, r in zip(("A++", "A+-"), out)},
        "work_split": "autotuned per work profile (paper_2203_04774_gb300/tuning_table.json)",
        "phase_ms_median": timed_phase_ms,
        "gpu_launches": launches,
        "clocks": clk,
        "cpu_baseline": cpu_res,
        "per_ordering": per_ordering,
    }


def h2d_bytes(key: str, n: int) -> int:
    """Host-to-device bytes of one e2e step: the raw pairs and the ranks."""
    wl = WORKLOADS[key]
    pairs = (wl["edge_factor"] << wl["scale"]) if wl["generator"] == "R-MAT" else \
        int(round(wl["n"] * wl["avg_degree"] / 2.0))
    return pairs * 8 + n * 4


# ---- many graphs: batched listing and serving ------------------------------

BATCH = {"workload": "batch4096-chunglu-degree-A++", "generator": "Chung-Lu family",
         "graphs": 4096, "n_range": [1000, 200000], "n_distribution": "log-uniform",
         "avg_degree_range": [8, 64], "exponent_range": [2.1, 3.0], "seed": 3,
         "ordering": "degree (ties by id), computed on the device", "algorithms": ["A++"]}


def run_batch(args, steps: int, warmup: int) -> dict:
    """Many independent graphs: one disjoint-union pass vs one pass per graph.

    A step takes the 4096 edge lists (device resident) to per-graph triangle
    counts and set hashes on the host: load + dedup, degree ordering, DAG,
    A++ listing.  Batched: tl_graph_load_parts over all graphs, one ordering,
    one listing, per-part count + hash.  Per graph: the same calls on each
    graph in turn.  Both must give identical per-graph results."""
    import torch

    import paper_2203_04774_gb300 as tl
    from paper_2203_04774_gb300 import synth
    from paper_2203_04774_gb300.synth import device as sdev

    fam = synth.chung_lu_family(BATCH["graphs"], BATCH["n_range"], BATCH["avg_degree_range"],
                                BATCH["exponent_range"], BATCH["seed"])
    k = BATCH["graphs"]
    ns, pairs = fam["n"], fam["pairs"]
    po = np.zeros(k + 1, np.int64)
    np.cumsum(pairs, out=po[1:])
    t0 = time.time()
    e_all = torch.empty((int(po[-1]), 2), dtype=torch.int32, device="cuda")
    for i in range(k):
        e_all[po[i]:po[i + 1]] = sdev.chung_lu_device(int(ns[i]), float(fam["deg"][i]),
                                                      float(fam["gamma"][i]),
                                                      int(fam["seeds"][i]))
    torch.cuda.synchronize()
    log(f"[bench] {k} graphs ready in {time.time() - t0:.1f}s: pairs={int(po[-1])}")
    stream = torch.cuda.Stream()
    cstream = torch.cuda.Stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    ch = tl.CountHash(cstream.cuda_stream)
    ch_ptr = tl.tl_count_hash_ptr()
    chp = tl.CountHashParts(ns, cstream.cuda_stream)
    n_all = int(ns.sum())
    rank_all = torch.empty(n_all, dtype=torch.int32, device="cuda")
    vb = np.zeros(k + 1, np.int64)
    np.cumsum(ns, out=vb[1:])

    from paper_2203_04774_gb300 import autotune
    table = autotune.load_table()

    def batched(tuned=True):
        u = tl.tl_graph_load_parts(ns, pairs, e_all, stream.cuda_stream)
        try:
            tl.tl_order_compute(u, tl.TL_ORDER_DEGREE, rank_all)
            tl.tl_order_apply(u, rank_all)
            if tuned:  # the autotuner's split for the union's work profile
                autotune.apply(u, tl.TL_APP, table)
            chp.reset()
            nt = tl.tl_list_triangles(u, tl.TL_APP, CHUNK_BYTES, chp.fn(), chp.user)
            m = tl.tl_graph_size(u)[1]
            st = tl.tl_last_list_stats(u)
        finally:
            tl.tl_graph_free(u)
        c, h = chp.results()
        return nt, m, c, h, st

    def per_graph():
        c = np.zeros(k, np.uint64)
        h = np.zeros(k, np.uint64)
        lat = np.zeros(k)
        m = 0
        for i in range(k):
            t1 = time.perf_counter()
            g = tl.tl_graph_load(int(ns[i]), e_all[po[i]:po[i + 1]], stream.cuda_stream)
            try:
                r = rank_all[vb[i]:vb[i + 1]]
                tl.tl_order_compute(g, tl.TL_ORDER_DEGREE, r)
                tl.tl_order_apply(g, r)
                ch.reset()
                tl.tl_list_triangles(g, tl.TL_APP, tl.TL_MIN_CHUNK_BYTES, ch_ptr, ch.user)
                m += tl.tl_graph_size(g)[1]
            finally:
                tl.tl_graph_free(g)
            c[i], h[i] = ch.state.count, ch.state.hash
            lat[i] = time.perf_counter() - t1
        return int(c.sum()), m, c, h, lat

    def timed(fn, reps, *fa):
        out, ms = None, []
        for _ in range(reps):
            flush.zero_()
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            out = fn(*fa)
            torch.cuda.synchronize()
            ms.append((time.perf_counter() - t1) * 1e3)
        return out, ms

    for _ in range(warmup):
        batched()
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    launches0 = tl.tl_kernel_launches()
    (nt, m, cb, hb, st), b_ms = timed(batched, steps)
    b_launches = (tl.tl_kernel_launches() - launches0) / steps
    batched(False)
    (nt2, m2, cb2, hb2, st2), f_ms = timed(batched, steps, False)
    per_warm = 1
    for _ in range(per_warm):
        per_graph()
    launches0 = tl.tl_kernel_launches()
    (nt1, m1, c1, h1, lat), p_ms = timed(per_graph, max(1, min(steps, 2)))
    p_launches = (tl.tl_kernel_launches() - launches0) / max(1, min(steps, 2))
    clk = clocks.stop()
    assert nt == nt1 and m == m1, (nt, nt1, m, m1)
    assert np.array_equal(cb, c1) and np.array_equal(hb, h1), "per-graph results differ"
    assert np.array_equal(cb, cb2) and np.array_equal(hb, hb2), "the work split changed results"
    # oracle spot check on the three smallest and three other graphs
    import oracle
    spot = []
    others = np.random.default_rng(3).choice(k, 3, replace=False)
    for i in list(np.argsort(ns)[:3]) + list(others):
        e = e_all[po[i]:po[i + 1]].cpu().numpy().view(np.uint32)
        g = oracle.Graph(int(ns[i]), e)
        r = rank_all[vb[i]:vb[i + 1]].cpu().numpy().view(np.uint32)
        g.order_apply(r)
        _, rc, rh, _ = g.list(oracle.APP, store=False)
        spot.append(bool(rc == int(cb[i]) and rh == int(hb[i])))
    assert all(spot), spot
    b_s = statistics.median(b_ms) / 1e3
    f_s = statistics.median(f_ms) / 1e3
    p_s = statistics.median(p_ms) / 1e3
    line = {
        "metric": "graphs/s (batched disjoint-union pass vs one pass per graph)",
        "value": k / b_s, "unit": "graphs/s", "n_gpus": 1, "steps": steps,
        "warmup": warmup, "ms_per_step": b_s * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic (seeded Chung-Lu family, generated on the device)",
        "config": dict(BATCH, m=m, triangles=nt, pairs=int(po[-1]), vertices=n_all,
                       l2="256 MiB buffer written before each step", chunk_bytes=CHUNK_BYTES),
        "batched": {"s_per_step": b_s, "graphs_per_s": k / b_s, "triangles_per_s": nt / b_s,
                    "edges_per_s": m / b_s, "gpu_launches_per_step": b_launches,
                    "latency_s": {"p50": b_s, "p99": b_s,
                                  "note": "every graph completes when the pass ends"},
                    "list_kernel_ms": sum(st["kernel_ms"]), "list_stats": st,
                    "work_split": "autotuned for the union's work profile",
                    "launch_mode": "host-driven: one union build and one listing call, the "
                                   "host launching each kernel and handing full chunks to the "
                                   "consumer (no CUDA-graph replay)"},
        "batched_fixed_split": {"s_per_step": f_s, "graphs_per_s": k / f_s,
                                "list_kernel_ms": sum(st2["kernel_ms"]),
                                "work_split": "library defaults"},
        "autotune_gain": f_s / b_s,
        "per_graph": {"s_per_step": p_s, "graphs_per_s": k / p_s, "triangles_per_s": nt / p_s,
                      "edges_per_s": m / p_s, "gpu_launches_per_step": p_launches,
                      "latency_s": {"p50": float(np.percentile(lat, 50)),
                                    "p99": float(np.percentile(lat, 99)),
                                    "note": "per graph, run back to back"}},
        "speedup_batched_vs_per_graph": p_s / b_s,
        "equal_output": True, "oracle_spot_check_graphs": len(spot),
        "gpu_launches": b_launches * steps,
        "clocks": clk,
    }
    ch.release()
    del e_all, rank_all, flush
    torch.cuda.empty_cache()
    return line


SERVE = {"workload": "serve-chunglu-poisson", "generator": "Chung-Lu family", "pool_graphs": 128,
         "n_range": [1000, 5000000], "n_distribution": "log-uniform",
         "avg_degree_range": [8, 64], "exponent_range": [2.1, 3.0], "seed": 5,
         "orderings": ["degree", "core (level-synchronous peeling)"],
         "algorithms": ["A++", "A+-"],
         "rates_per_s": [100, 1000, 10000], "requests_per_rate": 2000}


SIZE_BUCKETS = [(0, 1e5), (1e5, 1e6), (1e6, 1e7), (1e7, float("inf"))]


def run_serve(args, requests: int) -> dict:
    """Poisson stream of listing requests against the request server.

    The pool graphs and their orderings are generated, loaded and registered
    before timing (device resident).  For each arrival rate, the same request
    sequence is served twice: batched (max_batch 256, 2 workers) and one
    request per pass (max_batch 1, 1 worker).  Latency = scheduled arrival ->
    completion on the server's clock; throughput = requests / (last completion
    - first arrival).  Both modes must give every request the same result."""
    import threading

    import torch

    import paper_2203_04774_gb300 as tl
    from paper_2203_04774_gb300 import synth
    from paper_2203_04774_gb300.synth import device as sdev

    cfg = dict(SERVE)
    cfg["requests_per_rate"] = requests
    fam = synth.chung_lu_family(cfg["pool_graphs"], cfg["n_range"], cfg["avg_degree_range"],
                                cfg["exponent_range"], cfg["seed"])
    t0 = time.time()
    graphs, ranks, ms = [], [], []
    for i in range(cfg["pool_graphs"]):
        n = int(fam["n"][i])
        e = sdev.chung_lu_device(n, float(fam["deg"][i]), float(fam["gamma"][i]),
                                 int(fam["seeds"][i]))
        g = tl.Graph(n, e)
        del e
        graphs.append(g)
        ranks.append([g.order_compute(tl.TL_ORDER_DEGREE), g.order_compute(tl.TL_ORDER_CORE)])
        ms.append(g.m)
    torch.cuda.synchronize()
    log(f"[bench] pool of {len(graphs)} graphs ready in {time.time() - t0:.1f}s: "
        f"edges={sum(ms)}")
    R = cfg["requests_per_rate"]
    budget = 96 << 30

    def requests(rate):
        # counter-based draws under the workload seed: arrivals, graph, ordering, algorithm
        gap = -np.log1p(-synth.counter_uniform(cfg["seed"], 20 + int(rate), R)) / rate
        arr = np.cumsum(gap) - gap[0]
        gi = (synth.counter_uniform(cfg["seed"], 30, R) * len(graphs)).astype(np.int64)
        oi = (synth.counter_uniform(cfg["seed"], 32, R) < 0.5).astype(np.int64)
        al = (synth.counter_uniform(cfg["seed"], 31, R) < 0.5).astype(np.int64)
        return arr, gi, oi, al

    from paper_2203_04774_gb300 import autotune
    table = autotune.load_table()

    def serve(arr, gi, oi, al, max_batch, workers, tuned=False):
        srv = tl.Server(budget, max_batch=max_batch, workers=workers)
        if tuned:  # work splits per batch group, by its degree profile
            srv.set_tuning_table(table)
        ids = []
        for g, rs in zip(graphs, ranks):
            gid = srv.add_graph(g)
            ids.append((gid, [srv.add_ordering(gid, r) for r in rs]))
        rids = [None] * R
        start = tl.Server.now_ns() + 20_000_000

        def submitter():
            for i in range(R):
                target = start + int(arr[i] * 1e9)
                while True:
                    d = target - tl.Server.now_ns()
                    if d <= 0:
                        break
                    if d > 2_000_000:
                        time.sleep((d - 1_000_000) / 1e9)
                rids[i] = srv.submit(ids[gi[i]][0], ids[gi[i]][1][oi[i]], int(al[i]))

        th = threading.Thread(target=submitter)
        th.start()
        th.join()
        res = [srv.wait(r) for r in rids]
        srv.close()
        assert all(r["status"] == tl.TL_OK for r in res)
        done = np.array([r["t_done_ns"] for r in res], np.float64)
        sched = start + arr * 1e9
        lat = (done - sched) / 1e9
        span = (done.max() - sched.min()) / 1e9
        tri = sum(r["triangles"] for r in res)
        out = {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
               "requests_per_s": R / span, "triangles_per_s": tri / span,
               "mean_batch": float(np.mean([r["batch_size"] for r in res])),
               "max_batch_seen": int(max(r["batch_size"] for r in res))}
        # latency by request size (edges of the requested graph)
        req_m = np.asarray(ms, np.float64)[gi]
        by_size = []
        for lo, hi in SIZE_BUCKETS:
            sel = (req_m >= lo) & (req_m < hi)
            if sel.any():
                by_size.append({"edges": [lo, hi if hi < float("inf") else None],
                                "requests": int(sel.sum()),
                                "p50_s": float(np.percentile(lat[sel], 50)),
                                "p99_s": float(np.percentile(lat[sel], 99))})
        out["by_size"] = by_size
        return out, [(r["triangles"], r["hash"]) for r in res]

    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    launches0 = tl.tl_kernel_launches()
    rows = []
    for rate in cfg["rates_per_s"]:
        arr, gi, oi, al = requests(rate)
        b, rb = serve(arr, gi, oi, al, 256, 2, tuned=True)
        f, rf = serve(arr, gi, oi, al, 256, 2, tuned=False)
        p, rp = serve(arr, gi, oi, al, 1, 1)
        assert rb == rp == rf, "a request's result depends on its batch or work split"
        rows.append({"rate_per_s": rate, "batched": b, "batched_fixed_split": f,
                     "per_request": p,
                     "throughput_ratio": b["requests_per_s"] / p["requests_per_s"],
                     "autotune_gain": b["requests_per_s"] / f["requests_per_s"]})
        log(f"[bench] rate {rate}: batched {b} per-request {p}")
    launches = tl.tl_kernel_launches() - launches0
    clk = clocks.stop()
    top = rows[-1]
    line = {
        "metric": "requests/s and p50/p99 latency, batched serving vs one request per pass",
        "value": top["batched"]["requests_per_s"], "unit": "requests/s", "n_gpus": 1,
        "steps": len(rows), "warmup": 0, "ms_per_step": None, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic (seeded Chung-Lu pool generated on the device, Poisson arrivals)",
        "config": dict(cfg, pool_edges=int(sum(ms)), hbm_budget_bytes=budget,
                       batched={"max_batch": 256, "workers": 2,
                                "work_split": "per batch group, nearest tuning-table profile"},
                       batched_fixed_split={"max_batch": 256, "workers": 2,
                                            "work_split": "library defaults"},
                       per_request={"max_batch": 1, "workers": 1}),
        "rates": rows, "equal_output": True, "gpu_launches": launches, "clocks": clk,
    }
    del graphs
    torch.cuda.empty_cache()
    return line



def ordering_sweep(tl, n, e, e_dev, stream):
    """GPU listing time vs the paper's cost for several orderings (Fig. 2 analogue)."""
    from paper_2203_04774_gb300 import synth
    off, adj = synth.simple_csr(n, e)
    makers = {"random": lambda: synth.order_random(n, 2),
              "degree": lambda: synth.order_degree(off),
              "core": lambda: synth.order_core(off, adj),
              "split": lambda: synth.order_split(off),
              "check": lambda: synth.order_check(off, adj),
              "neigh": lambda: synth.order_neigh(off, adj)[0],
              "neigh_c++": lambda: synth.order_neigh(off, adj, objective="C++")[0]}
    orders, host_s = {}, {}
    for name, make in makers.items():  # host orderings (input preparation, not timed above)
        t0 = time.perf_counter()
        orders[name] = make()
        host_s[name] = round(time.perf_counter() - t0, 3)
    import torch
    ch = tl.CountHash(stream.cuda_stream)
    g = tl.tl_graph_load(n, e_dev, stream.cuda_stream)
    rows = []
    try:
        # the device orderings (the ordering step of the full-listing task),
        # CUDA events on the handle's stream, after one warm-up call each
        dev_ms = {}
        rk = torch.empty(n, dtype=torch.int32, device="cuda")
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        for name, kind in (("degree", tl.TL_ORDER_DEGREE), ("split", tl.TL_ORDER_SPLIT),
                           ("core", tl.TL_ORDER_CORE)):
            tl.tl_order_compute(g, kind, rk)
            ev[0].record(stream)
            tl.tl_order_compute(g, kind, rk)
            ev[1].record(stream)
            ev[1].synchronize()
            dev_ms[name] = round(ev[0].elapsed_time(ev[1]), 3)
        for name, r in orders.items():
            tl.tl_order_apply(g, torch.from_numpy(r).cuda())
            for a, an in ((tl.TL_APP, "A++"), (tl.TL_APM, "A+-"), (tl.TL_AMM, "A--")):
                ch.reset()
                tl.tl_list_triangles(g, a, CHUNK_BYTES, tl.tl_count_hash_ptr(), ch.user)
                st = tl.tl_last_list_stats(g)
                rows.append({"ordering": name, "alg": an, "cost": tl.tl_cost(g, a),
                             "list_kernel_ms": sum(st["kernel_ms"]), "triangles": st["triangles"],
                             "host_ordering_s": host_s[name]})
    finally:
        tl.tl_graph_free(g)
        ch.release()
    rows.append({"device_ordering_ms": dev_ms})
    for an in ("A++", "A+-", "A--"):
        xs = [r["cost"] for r in rows if r.get("alg") == an]
        ys = [r["list_kernel_ms"] for r in rows if r.get("alg") == an]
        if len(xs) > 2 and np.std(xs) > 0 and np.std(ys) > 0:
            rows.append({"alg": an, "pearson_r_cost_vs_time": float(np.corrcoef(xs, ys)[0, 1])})
    return rows




def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="tl", choices=["tl", "reference"])
    ap.add_argument("--workload", default="all",
                    choices=["all", "chunglu1e8", "rmat20", "batch4096", "serve", "chunglu8e6"],
                    help="all (default): the 2e9-edge Chung-Lu graph as the headline, with "
                         "rmat20, batch4096 and serve as sub-objects; or one workload alone "
                         "(chunglu8e6: the headline's family at n = 8e6, for profiler captures)")
    ap.add_argument("--sub-steps", type=int, default=5,
                    help="timed steps of the rmat20 and batch4096 sub-objects")
    ap.add_argument("--serve-requests", type=int, default=0,
                    help="requests per arrival rate (default 2000 as a sub-object, 20000 alone)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baselines")
    ap.add_argument("--no-orderings", action="store_true", help="skip the per-ordering sweep")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--chunk-mb", type=int, default=DEFAULT_CHUNK_MB,
                    help="output chunk size in MiB")
    args = ap.parse_args()
    global CHUNK_BYTES
    CHUNK_BYTES = args.chunk_mb << 20
    wl = args.workload
    if args.impl == "reference":
        if wl in ("batch4096", "serve"):
            print(json.dumps({"impl": "reference", "unavailable": f"the {wl} workload has no "
                              "reference arm; its baseline is the unbatched mode in the same "
                              "line"}))
            return
        run_reference(args, wl if wl in ("rmat20", "chunglu8e6") else "chunglu1e8")
        return
    world, rank, local = dist_setup()
    worker = None
    if wl in ("all", "chunglu1e8") and world == 1 and not args.no_cpu:
        worker = OracleWorker("chunglu1e8")  # spawned before the first CUDA call
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    if wl in ("all", "chunglu1e8"):
        line = run_listing(args, "chunglu1e8", args.steps, args.warmup, e2e=not args.no_e2e,
                           orderings=False, cpu=None, dist=dist)
        if wl == "all" and world == 1:
            line["rmat20"] = run_listing(args, "rmat20", args.sub_steps, 3, e2e=not args.no_e2e,
                                         orderings=not args.no_orderings,
                                         cpu=None if args.no_cpu else "inline")
            line["batch4096"] = run_batch(args, args.sub_steps, 1)
            line["serve"] = run_serve(args, args.serve_requests or 2000)
        if worker:
            line["cpu_baseline"] = worker.result()
    elif wl == "rmat20":
        line = run_listing(args, "rmat20", args.steps, args.warmup, e2e=not args.no_e2e,
                           orderings=not args.no_orderings,
                           cpu=None if args.no_cpu or world > 1 else "inline", dist=dist)
    elif wl == "chunglu8e6":
        line = run_listing(args, "chunglu8e6", args.steps, args.warmup, e2e=not args.no_e2e,
                           orderings=False,
                           cpu=None if args.no_cpu or world > 1 else "inline", dist=dist)
    elif wl == "batch4096":
        line = run_batch(args, args.steps, args.warmup)
    else:
        line = run_serve(args, args.serve_requests or 20000)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
