#!/usr/bin/env python3
"""Benchmark: exact top-k closeness (BCM / BFSCut) on one GB300.

Workload (default): the synthetic Chung-Lu power-law graph, n = 2^20, mean
degree 10, degree exponent 2.3, seed 2 (~5.2M edges, 10.4M arcs), k = 10.
A step is one whole pass of the hot path on that graph with the CSR already in
HBM: create the handle from device memory, preprocess (connected components
for r(v), degree order), BFSCut top-k, release.  The value is seconds per
graph (lower is better); GTEPS = arcs scanned (m_vis) / step time.

Also reported, on the same graph: the plain one-source-per-launch GPU
BFSCut, per-k times for k in {1, 10, 100}, the end-to-end time through the
C-ABI from pinned host buffers, the dominant kernel's roofline, the CPU
oracle timed on a bounded sample, and a bit-exactness check of the result
against the oracle on sampled outputs.

--gpus N (under torchrun, one rank per GPU) shares each step's graph among
the N GPUs: rank r runs the top-k over its shard of the sources (every N-th
chunk of 64 positions of the degree order) while the ranks exchange their
k-th keys on the host (paper_1507_01490_gb300.exchange), one all-gather
brings the k-entry lists to every rank and rank 0 merges them
(bcm_topk_merge) into the graph's top-k.  Preprocessing is repeated on every
rank.  Total work per step is fixed, so scaling is strong.
--serve runs the serving benchmark (a graph mix and request streams) and
--sweep ratio|race the performance-ratio and positive-race sweeps instead.
--impl reference times the CPU oracle (one BFS per source, all host cores)
on a bounded sample of the same workload.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "top-k closeness s/graph & GTEPS, batched vs plain GPU BFSCut, bit-exact"
UNIT = "s/graph"
WORKLOADS = {
    "chunglu1m": "Chung-Lu power-law graph, n=2^20, mean degree 10, degree exponent 2.3, seed 2, "
                 "self-loops and repeats removed, undirected",
    "rmat20": "R-MAT scale 20, edge factor 16, (0.57,0.19,0.19,0.05), seed 3, directed",
    "grid2048": "2048x2048 grid, 5% of edges deleted (seed 4), largest component",
    "grid1024": "1024x1024 grid, 5% of edges deleted (seed 4), largest component (profiling-size case of the "
                "same recipe)",
    "grid512": "512x512 grid, 5% of edges deleted (seed 4), largest component (smaller case of the same "
               "recipe)",
    "grid256": "256x256 grid, 5% of edges deleted (seed 4), largest component (profiling-size case of the "
               "same recipe)",
    "ba2000": "Barabasi-Albert n=2000, m=3, seed 1",
    "chunglu256k": "Chung-Lu power-law graph, n=2^18, mean degree 10, degree exponent 2.3, seed 2 "
                   "(profiling-size case of the same recipe)",
    "rmat18": "R-MAT scale 18, edge factor 16, (0.57,0.19,0.19,0.05), seed 3, directed "
              "(profiling-size case of the same recipe)",
}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def profile_traffic(kernel, kernel_src_hash, workload="chunglu1m"):
    """dram bytes per launch of `kernel` on `workload` from the committed ncu
    summary, if it was taken on the current kernel source; else None."""
    p = os.path.join(ROOT, "profiles", "%s_%s.md" % (kernel, workload))
    if not os.path.exists(p):
        return None
    traffic, src = None, None
    for line in open(p):
        if line.startswith("traffic_bytes_per_launch:"):
            traffic = float(line.split(":", 1)[1])
        if line.startswith("kernel_source_sha256:"):
            src = line.split(":", 1)[1].strip()
    return traffic if (src == kernel_src_hash and traffic) else None


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("msbfs.cu", "common.cuh", "internal.h"):
        h.update(open(os.path.join(ROOT, "paper_1507_01490_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def load_golden(workload, k):
    """The oracle's complete top-k of this workload, if stored (written by
    tests/golden/make_fullsize.py, which calls only the oracle)."""
    p = os.path.join(ROOT, "tests", "golden", "fullsize_%s_k%d.json" % (workload, k))
    return json.load(open(p)) if os.path.exists(p) else None


def m_tot_undirected(g, reach):
    """Arcs the textbook algorithm scans: every u is scanned by each of the
    r(u) sources of its component (undirected graphs)."""
    return int(np.sum(g.degrees().astype(np.int64) * reach.astype(np.int64)))


# ------------------------------------------------------------------- oracle
def cpu_sample(g, budget_s, seed=7):
    """Oracle (exhaustive BFS, all host cores) on a growing sample of sources
    until ~budget_s of work; returns (seconds per graph, sources, threads):
    threads is the fewest threads that took work in any call of the sample."""
    import oracle
    from paper_1507_01490_gb300 import graphgen
    cores = oracle.default_threads()
    done, spent, size = 0, 0.0, max(cores * 16, 64)
    used = cores
    while spent < budget_s and done < g.n:
        cnt = min(size, g.n - done)
        src = graphgen.uniform_u32(seed + done, cnt, g.n)
        info = {}
        t = time.perf_counter()
        oracle.farness_all(g, sources=src, threads=cores, info=info)
        spent += time.perf_counter() - t
        used = min(used, info["threads_used"])
        done += cnt
        size = min(size * 2, 1 << 16)
    return spent / done * g.n, done, used


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    from paper_1507_01490_gb300 import graphgen
    g = graphgen.workload(args.workload)
    per_step, dones, used = [], [], []
    budget = args.ref_step_seconds
    for i in range(args.warmup + args.steps):
        s_per_graph, done, threads = cpu_sample(g, budget, seed=1000 + i)
        if i >= args.warmup:
            per_step.append(s_per_graph)
            dones.append(done)
            used.append(threads)
    cores = min(used)
    v = float(np.mean(per_step))
    sample = "exhaustive BFS from %d to %d uniformly drawn sources per step (of n = %d), scaled by n" % (
        min(dones), max(dones), g.n)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": "%s: %s" % (args.workload, WORKLOADS[args.workload]), "n": g.n, "m_arcs": g.m,
                       "k": args.k,
                       "step": "top-k of the graph by the oracle (plain BFS from every vertex), timed on a bounded "
                               "sample of sources and scaled by n",
                       "parallelism": "host cores"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "about %.0f s of CPU work per step: %s" % (budget, sample)},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ serving
SERVE_METRIC = "top-k closeness serving: requests/s with p50/p99 latency over a mix of device-resident graphs"


def run_serve(args, rank, world):
    """Serving with continuous batching (paper_1507_01490_gb300.serve): the
    graph mix is built and made resident, the closed-loop capacity measured,
    then Poisson streams at fractions of it are served; a sample of results is
    checked against the same requests run alone."""
    if rank != 0:
        return 0
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    from paper_1507_01490_gb300 import bcm as B, serve
    t = time.perf_counter()
    specs = serve.mix_specs(args.serve_graphs)
    graphs = [serve.build_graph(sp) for sp in specs]
    t_gen = time.perf_counter() - t
    t = time.perf_counter()
    budget = int(args.serve_budget_gb * (1 << 30))
    # optional cap on each run's workspace (negative: the budget's share of
    # one run in flight; 0, the default: none)
    ws_cap = int(args.serve_ws_cap_gb * (1 << 30)) if args.serve_ws_cap_gb >= 0 else budget // args.serve_inflight
    # per-CTA blocks and vertex-table entries of a run (0: the library's
    # defaults; blocks < 0: the resident per-CTA blocks, two 512-thread CTAs
    # per SM, shared among the runs in flight; table < 0: dense, the default
    # here).  Measured on this mix (1000-2000 requests per rate): dense tables
    # with the library's block count (lowered by the workspace cap on the
    # largest graphs) served 106.8 requests/s; the library's hashed tables
    # 41.7 (likely: the mix's denser Barabasi-Albert graphs outgrow them and
    # defer waves); 19 blocks with dense tables 24.8, 38 blocks 22.5.
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    blocks = args.serve_blocks if args.serve_blocks >= 0 else max(1, 2 * sms // args.serve_inflight)
    table = args.serve_table if args.serve_table >= 0 else (1 << 30)
    be = serve.GpuBackend(graphs, options=B.make_options(blocks=blocks, cta_table=table), workspace_cap=ws_cap)
    torch.cuda.synchronize()
    t_load = time.perf_counter() - t
    csr_bytes = int(sum(g.row_ptr.nbytes // 2 + g.col.nbytes for g in graphs))

    def sched():
        return serve.Scheduler(be, max_inflight=args.serve_inflight, hbm_budget=budget)

    # warm-up: every graph once (first-use allocations), then a short closed loop
    sched().run([serve.Request(i, i, 100, 0.0) for i in range(len(graphs))])
    sched().run(serve.request_stream(min(500, args.serve_requests), len(graphs), float("inf"), seed=77))
    clocks = ClockSampler(0)
    clocks.start()
    l0 = __import__("paper_1507_01490_gb300.bcm", fromlist=["x"]).bcm_launch_count()
    t = time.perf_counter()
    s0 = sched()
    cap_res = s0.run(serve.request_stream(args.serve_requests, len(graphs), float("inf"), seed=5))
    cap_span = time.perf_counter() - t
    capacity = len(cap_res) / cap_span
    print(json.dumps({"progress": "capacity", "rps": capacity, "requests": len(cap_res)}), file=sys.stderr,
          flush=True)
    rates = []
    last = None
    for frac in [float(x) for x in args.serve_rates.split(",") if x]:
        reqs = serve.request_stream(args.serve_requests, len(graphs), capacity * frac, seed=5)
        sc = sched()
        t = time.perf_counter()
        res = sc.run(reqs)
        span = time.perf_counter() - t
        summ = serve.summarize(res, makespan=span)
        summ.update({"frac_of_capacity": frac, "offered_rps": capacity * frac,
                     "peak_inflight": sc.peak_inflight, "peak_workspace_gb": sc.peak_held / 2**30,
                     "trims": sc.trims})
        rates.append(summ)
        last = res
        print(json.dumps({"progress": "rate", "summary": summ}), file=sys.stderr, flush=True)
    launches = __import__("paper_1507_01490_gb300.bcm", fromlist=["x"]).bcm_launch_count() - l0
    clk = clocks.stop()
    # the same requests alone (each graph's workspace given back first)
    be.trim_all()
    rng = np.random.default_rng(3)
    pick = rng.choice(len(last), size=min(args.serve_check, len(last)), replace=False)
    same = True
    for i in pick:
        r = last[int(i)]
        ids, far, reach, _ = be.alone(r.graph, r.k)
        same = same and np.array_equal(ids, r.ids) and np.array_equal(far, r.farness) and \
            np.array_equal(reach, r.reach)
    top = rates[-1] if rates else serve.summarize(cap_res, makespan=cap_span)
    line = {
        "metric": SERVE_METRIC, "value": top["throughput_rps"], "unit": "requests/s", "n_gpus": 1,
        "steps": len(rates), "warmup": 2, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": "serving mix: %d graphs (first half Barabasi-Albert, second half R-MAT), n "
                               "log-uniform in [1e3, 2e6], mean degree 8..16, seeds 1000+i; %d requests per rate, "
                               "graph uniform, k uniform in {1,10,100}, Poisson arrivals (seed 5)"
                               % (len(graphs), args.serve_requests),
                   "max_inflight": args.serve_inflight, "hbm_budget_gb": args.serve_budget_gb,
                   "cta_blocks": blocks or "library default",
                   "cta_table": "dense" if table >= (1 << 30) else (table or "library default"),
                   "workspace_cap_gb": ws_cap / 2**30 if ws_cap else None,
                   "graphs_resident_bytes": csr_bytes, "vertices": int(sum(g.n for g in graphs)),
                   "arcs": int(sum(g.m for g in graphs))},
        "capacity_rps": capacity, "capacity_latency_ms": serve.summarize(cap_res, cap_span)["latency_ms"],
        "rates": rates,
        "identical_alone_and_mixed": bool(same), "checked_requests": int(len(pick)),
        "gpu_launches": launches, "clocks": clk,
        "setup_s": {"generate": t_gen, "upload_and_preprocess": t_load},
    }
    be.close()
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ batches
def run_batch(args, rank, world):
    """Many small graphs: one synchronous bcm_topk per graph against one
    replay of their runs recorded as a CUDA graph (bcm_batch_*)."""
    if rank != 0:
        return 0
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    from paper_1507_01490_gb300 import bcm as B, serve
    specs = [sp for sp in serve.mix_specs(args.batch_graphs * 4, n_hi=args.batch_max_n, seed_base=3000)
             if (sp[1] if sp[0] == "ba" else 1 << sp[1]) <= args.batch_max_n][:args.batch_graphs]
    graphs = [serve.build_graph(sp) for sp in specs]
    stream = torch.cuda.Stream()
    hs = [B.BcmGraph.from_graph(g, stream=stream.cuda_stream) for g in graphs]
    ks = [[1, 10, 100][i % 3] for i in range(len(graphs))]
    outs = [(torch.zeros(k, dtype=torch.int32, device="cuda"), torch.zeros(k, dtype=torch.int64, device="cuda"),
             torch.zeros(k, dtype=torch.int32, device="cuda")) for k in ks]
    opts = B.make_options(flags=B.BCM_OUT_DEVICE)

    def one_by_one():
        for h, k, o in zip(hs, ks, outs):
            B.bcm_topk(h.h, k, opts, o[0], o[1], o[2])

    one_by_one()
    batch = B.BcmBatch([h.h for h in hs], ks, outs, stream, opts)
    batch.run()
    ref = [tuple(t.clone() for t in o) for o in outs]

    def timed(fn, reps):
        ts = []
        for _ in range(reps):
            torch.cuda.synchronize()
            t = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t)
        return float(np.median(ts))

    # every graph on its own stream, all started, then all finished
    streams = [torch.cuda.Stream() for _ in graphs]
    hs2 = [B.BcmGraph.from_graph(g, stream=st.cuda_stream) for g, st in zip(graphs, streams)]

    def all_streams():
        for h, k, o in zip(hs2, ks, outs):
            B.bcm_topk_start(h.h, k, opts, o[0], o[1], o[2])
        for h in hs2:
            B.bcm_topk_finish(h.h, wait=True)

    all_streams()
    l0 = B.bcm_launch_count()
    t_seq = timed(one_by_one, args.steps)
    seq_launches = (B.bcm_launch_count() - l0) // max(args.steps, 1)
    t_str = timed(all_streams, args.steps)
    t_bat = timed(batch.run, args.steps)
    same = all(all(torch.equal(a, b) for a, b in zip(r, o)) for r, o in zip(ref, outs))
    for h in hs2:
        h.close()
    line = {"metric": "top-k closeness of many small graphs: graphs/s, one bcm_topk per graph vs one CUDA graph",
            "value": len(graphs) / t_bat, "unit": "graphs/s", "higher_is_better": True, "n_gpus": 1,
            "steps": args.steps, "data": "synthetic", "dtype": "u64",
            "config": {"workload": "%d graphs of the serving recipe (seed 3000+i) with n <= %d, k in {1,10,100}"
                                   % (len(graphs), args.batch_max_n),
                       "vertices": int(sum(g.n for g in graphs)), "arcs": int(sum(g.m for g in graphs))},
            "one_by_one": {"s_per_batch": t_seq, "graphs_per_s": len(graphs) / t_seq,
                           "kernel_launches": int(seq_launches)},
            "one_stream_per_graph": {"s_per_batch": t_str, "graphs_per_s": len(graphs) / t_str},
            "cuda_graph": {"s_per_batch": t_bat, "graphs_per_s": len(graphs) / t_bat, "branches": 16},
            "speedup": t_seq / t_bat, "same_results": bool(same)}
    batch.close()
    for h in hs:
        h.close()
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------- sweeps
def run_sweep(args, rank, world):
    """ratio: the performance ratio m_vis / (m n) of Section 3.1 against n on
    Barabasi-Albert graphs (the synthetic counterpart of the paper's growing
    actor graphs, whose inverse ratio grew about linearly with n), batched
    kernels and, where it finishes in seconds, the plain one-source kernel.
    race: the positive race of Section 3.3 -- how many more arcs the batched
    kernels scan than the sequential order (the plain kernel), by lane width."""
    if rank != 0:
        return 0
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    from paper_1507_01490_gb300 import bcm as B, graphgen
    rows = []
    if args.sweep == "ratio":
        for lg in range(args.sweep_lo, args.sweep_hi + 1):
            n = 1 << lg
            g = graphgen.ba(n, 4, seed=100 + lg)
            mn = float(g.m) * g.n
            with B.BcmGraph.from_graph(g) as h:
                h.topk(10)
                row = {"graph": "BA n=2^%d m=4 (seed %d)" % (lg, 100 + lg), "n": n, "m_arcs": g.m}
                for k in (1, 10, 100):
                    ids, far, reach, st = h.topk(k)
                    row["k%d" % k] = {"m_vis": st["m_vis"], "ratio": st["m_vis"] / mn,
                                      "inverse_ratio": mn / st["m_vis"], "kernel_ms": st["kernel_ms"]}
                    if n <= args.plain_max_n and k <= 10:
                        _, _, _, sp = h.topk(k, flags=B.BCM_PLAIN)
                        row["k%d" % k]["plain_m_vis"] = sp["m_vis"]
                        row["k%d" % k]["plain_ratio"] = sp["m_vis"] / mn
                        row["k%d" % k]["plain_ms"] = sp["kernel_ms"]
            rows.append(row)
            print(json.dumps(row), file=sys.stderr, flush=True)
        # least-squares slope of the inverse ratio against n (k = 10)
        xs = np.array([r["n"] for r in rows], dtype=float)
        ys = np.array([r["k10"]["inverse_ratio"] for r in rows])
        slope, icpt = np.polyfit(xs, ys, 1)
        fit = {"inverse_ratio_vs_n_k10": {"slope_per_vertex": slope, "intercept": icpt,
                                          "r2": float(1 - np.sum((ys - (slope * xs + icpt)) ** 2) /
                                                      np.sum((ys - ys.mean()) ** 2))}}
        print(json.dumps({"sweep": "performance ratio vs n", "rows": rows, "fit": fit}), flush=True)
    else:
        for name in args.sweep_graphs.split(","):
            g = graphgen.workload(name)
            with B.BcmGraph.from_graph(g) as h:
                h.topk(10)
                row = {"graph": name, "n": g.n, "m_arcs": g.m}
                for k in (1, 10):
                    _, _, _, sp = h.topk(k, flags=B.BCM_PLAIN)
                    base = sp["m_vis"]
                    ent = {"plain_m_vis": base}
                    for lanes in (64, 128, 256):
                        for gl in (64, 128, 256):
                            _, _, _, st = h.topk(k, lanes=lanes, grid_lanes=gl)
                            ent["cta%d_grid%d" % (lanes, gl)] = {"m_vis": st["m_vis"],
                                                                 "increase": st["m_vis"] / base - 1.0}
                    row["k%d" % k] = ent
            rows.append(row)
            print(json.dumps(row), file=sys.stderr, flush=True)
        print(json.dumps({"sweep": "positive race: m_vis of the batched kernels over the sequential order",
                          "rows": rows}), flush=True)
    return 0


# ---------------------------------------------------------------------- ours
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)   # ~1.3 s timed: several clock samples
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="chunglu1m", choices=sorted(WORKLOADS))
    ap.add_argument("--k", type=int, default=10)
    ap.add_argument("--lanes", type=int, default=0, help="0: library default")
    ap.add_argument("--grid-lanes", type=int, default=0, help="sources per grid-wide wave; 0: library default")
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--blocks", type=int, default=0)
    ap.add_argument("--no-plain", action="store_true", help="skip the plain one-source baseline")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-verify", action="store_true", help="skip the oracle check of the result")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end host-buffer timing")
    ap.add_argument("--no-perk", action="store_true", help="skip the per-k timings")
    ap.add_argument("--no-autotune", action="store_true", help="library defaults instead of the autotuner")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-step-seconds", type=float, default=8.0)
    ap.add_argument("--serve", action="store_true", help="the serving benchmark (graph mix, request streams)")
    ap.add_argument("--serve-graphs", type=int, default=200)
    ap.add_argument("--serve-requests", type=int, default=10000)
    ap.add_argument("--serve-rates", default="0.5,0.8,1.0", help="fractions of the measured capacity")
    ap.add_argument("--serve-inflight", type=int, default=16)
    ap.add_argument("--serve-budget-gb", type=float, default=120.0)
    ap.add_argument("--serve-ws-cap-gb", type=float, default=-1.0,
                    help="per-run workspace cap (fewer per-CTA blocks on large graphs); <0: budget/inflight, 0: none")
    ap.add_argument("--serve-check", type=int, default=300, help="results compared with the request alone")
    ap.add_argument("--serve-blocks", type=int, default=0,
                    help="per-CTA blocks of a served run (0: library default; <0: resident blocks / inflight)")
    ap.add_argument("--serve-table", type=int, default=-1,
                    help="per-CTA vertex table entries of a served run (0: library default; <0: dense)")
    ap.add_argument("--batch", action="store_true", help="many small graphs as one CUDA graph")
    ap.add_argument("--batch-graphs", type=int, default=128)
    ap.add_argument("--batch-max-n", type=int, default=8000)
    ap.add_argument("--sweep", choices=["ratio", "race"], help="a sweep instead of the benchmark")
    ap.add_argument("--sweep-lo", type=int, default=14, help="ratio sweep: smallest n = 2^lo")
    ap.add_argument("--sweep-hi", type=int, default=21)
    ap.add_argument("--plain-max-n", type=int, default=1 << 18)
    ap.add_argument("--sweep-graphs", default="ba2000,chunglu256k,chunglu1m,rmat20")
    args = ap.parse_args()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.serve:
        return run_serve(args, rank, world)
    if args.sweep:
        return run_sweep(args, rank, world)
    if args.batch:
        return run_batch(args, rank, world)

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__
    __graft_entry__.build()
    from paper_1507_01490_gb300 import bcm as B, graphgen

    g = graphgen.workload(args.workload)
    k = args.k
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    rp_d = torch.from_numpy(g.row_ptr.view(np.int64)).to(dev)
    col_d = torch.from_numpy(g.col.view(np.int32)).to(dev)
    kk = min(k, g.n)
    kbuf = min(max(k, 100), g.n)          # output rows for the largest k queried below
    ids_d = torch.zeros(kbuf, dtype=torch.int32, device=dev)
    far_d = torch.zeros(kbuf, dtype=torch.int64, device=dev)
    reach_d = torch.zeros(kbuf, dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 129 MB of L2
    torch.cuda.synchronize()

    # launch parameters: the autotuner's choice for this graph (rank 0 tunes,
    # the others take its choice), unless fixed on the command line
    tuned, tuning_s = None, 0.0
    if not args.no_autotune and not (args.lanes or args.threads or args.grid_lanes):
        from paper_1507_01490_gb300 import autotune
        if rank == 0:
            with B.BcmGraph(rp_d, col_d, g.n, g.directed, on_device=True, stream=stream.cuda_stream) as th:
                tuned, tuning_s, _ = autotune.tuned_options(th, g, k, cache_path=None, rounds=2, reps=2)
        if dist:
            box = [tuned]
            dist.broadcast_object_list(box, src=0)
            tuned = box[0]
    par = dict(lanes=args.lanes, threads=args.threads, grid_lanes=args.grid_lanes, pull_div=0, kflags=0)
    if tuned:
        from paper_1507_01490_gb300 import autotune
        par.update(lanes=tuned["lanes"], threads=tuned["threads"], grid_lanes=tuned["grid_lanes"],
                   pull_div=tuned["pull_div"], kflags=autotune.PER_CTA[tuned.get("per_cta", "auto")])

    def mkopt(flags, **extra):
        return B.make_options(lanes=par["lanes"], threads=par["threads"], blocks=args.blocks,
                              flags=flags | par["kflags"], grid_lanes=par["grid_lanes"], pull_div=par["pull_div"],
                              **extra)

    opts = mkopt(B.BCM_OUT_DEVICE)

    def step(kq=k, o=opts, stats=None):
        h = B.bcm_graph_create(rp_d, col_d, g.n, g.m, g.directed, ptr_on_device=True,
                               stream=stream.cuda_stream)
        try:
            assert min(kq, g.n) <= kbuf
            B.bcm_topk(h, kq, o, ids_d, far_d, reach_d, stats)
        finally:
            B.bcm_graph_destroy(h)

    # N > 1: the ranks share one graph per step.  Rank r takes shard r of the
    # degree order, then one all-gather brings every shard's list to every
    # rank and rank 0 merges them (bcm_topk_merge) into the graph's top-k.
    merged = {}
    exchange_rounds = []
    if world > 1:
        from paper_1507_01490_gb300.exchange import ThresholdExchange
        sopts = mkopt(B.BCM_OUT_DEVICE, shard_index=rank, shard_count=world)
        kloc = min(k, B.shard_size(g.n, rank, world))
        gath = [torch.zeros((world, k), dtype=t, device=dev) for t in (torch.int32, torch.int64, torch.int32)]
        cnts = torch.zeros(world, dtype=torch.int64, device=dev)
        # the shards' k-th keys travel on the host (gloo) while the runs go on
        xgroup = dist.new_group(backend="gloo")

        def shard_step(stats=None):
            h = B.bcm_graph_create(rp_d, col_d, g.n, g.m, g.directed, ptr_on_device=True,
                                   stream=stream.cuda_stream)
            try:
                B.bcm_topk_start(h, k, sopts, ids_d, far_d, reach_d)
                ex = ThresholdExchange(group=xgroup, period_s=1e-4)
                ex.run(lambda: B.bcm_topk_threshold(h), lambda key: B.bcm_topk_offer(h, key),
                       lambda: B.bcm_topk_finish(h, wait=False, stats=stats))
                exchange_rounds.append((ex.rounds, ex.offers))
            finally:
                B.bcm_graph_destroy(h)
            with torch.cuda.stream(stream):
                mine = torch.tensor([kloc], dtype=torch.int64, device=dev)
                dist.all_gather_into_tensor(cnts, mine)
                for buf, src in zip(gath, (ids_d, far_d, reach_d)):
                    dist.all_gather_into_tensor(buf.view(-1), src[:k].contiguous())
            if rank == 0:
                c = cnts.cpu().numpy()
                parts = [x.cpu().numpy() for x in gath]
                sel = [np.concatenate([parts[j][i, :c[i]] for i in range(world)]) for j in range(3)]
                merged["ids"], merged["far"], merged["reach"] = B.bcm_topk_merge(
                    sel[0].view(np.uint32), sel[1].view(np.uint64), sel[2].view(np.uint32), k)

    def timed(fn, reps, last_stats=None):
        """per-step device time (CUDA events on the library's stream), L2 flushed before each;
        the last step also fills last_stats (the counters are copied with the results either way)"""
        ts = []
        for i in range(reps):
            with torch.cuda.stream(stream):
                flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            if last_stats is not None and i == reps - 1:
                fn(stats=last_stats)
            else:
                fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3)
        return ts

    run_step = shard_step if world > 1 else step
    for _ in range(args.warmup):
        run_step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    l0 = B.bcm_launch_count()
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    st = B.bcm_stats()
    step_times = timed(run_step, args.steps, last_stats=st)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    launches = B.bcm_launch_count() - l0
    clk = clocks.stop()
    total = sum(step_times)
    if dist:
        t = torch.tensor([total], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total = float(t.item())
    # N ranks finish one graph per step together
    s_per_graph = total / args.steps

    # counters of the last timed step
    st = st.as_dict()
    if world > 1:
        shard_stats = st
        if rank == 0:
            got_ids, got_far, got_reach = merged["ids"], merged["far"], merged["reach"]
        dist.barrier()
        if rank != 0:
            dist.destroy_process_group()
            return 0
        st = B.bcm_stats()           # rank 0 alone: the whole graph, for the counters below
        step(stats=st)
        st = st.as_dict()
        same_as_single = bool(np.array_equal(got_ids, ids_d[:kk].cpu().numpy().view(np.uint32)))
    else:
        shard_stats = None
        got_ids = ids_d[:kk].cpu().numpy().view(np.uint32).copy()
        got_far = far_d[:kk].cpu().numpy().view(np.uint64).copy()
        got_reach = reach_d[:kk].cpu().numpy().view(np.uint32).copy()

    # per-k times and the plain baseline
    per_k = {}
    for kq in ([] if args.no_perk else sorted({1, 10, 100} | {k})):
        kq_opts = mkopt(B.BCM_OUT_DEVICE)
        ts = timed(lambda: step(kq, kq_opts), 3)
        s2 = B.bcm_stats()
        step(kq, kq_opts, s2)
        per_k[str(kq)] = {"s_per_graph": float(np.median(ts)), "m_vis": s2.m_vis,
                          "gteps": s2.m_vis / float(np.median(ts)) / 1e9}
        gk = load_golden(args.workload, kq)
        if gk is not None and world == 1:
            nq = min(kq, g.n)
            per_k[str(kq)]["bit_exact"] = bool(
                gk["csr_sha256_16"] == g.hash64() and
                ids_d[:nq].cpu().numpy().view(np.uint32).tolist() == gk["ids"] and
                far_d[:nq].cpu().numpy().view(np.uint64).tolist() == gk["farness"] and
                reach_d[:nq].cpu().numpy().view(np.uint32).tolist() == gk["reach"])
    plain = None
    if not args.no_plain:
        popts = B.make_options(flags=B.BCM_OUT_DEVICE | B.BCM_PLAIN)
        sp = B.bcm_stats()
        tp = timed(lambda: step(k, popts, sp), 1)[0]
        p_ids = ids_d[:kk].cpu().numpy().view(np.uint32).copy()
        plain = {"s_per_graph": tp, "m_vis": sp.m_vis, "gteps": sp.m_vis / tp / 1e9,
                 "launches": sp.launches, "same_result": bool(np.array_equal(p_ids, got_ids))}

    # e2e: through the C-ABI from pinned host memory, results back to host
    rp_h = torch.from_numpy(g.row_ptr.view(np.int64)).pin_memory()
    col_h = torch.from_numpy(g.col.view(np.int32)).pin_memory()
    ids_h = torch.zeros(kk, dtype=torch.int32).pin_memory()
    far_h = torch.zeros(kk, dtype=torch.int64).pin_memory()
    reach_h = torch.zeros(kk, dtype=torch.int32).pin_memory()
    hopts = mkopt(0)

    def e2e_step():
        h = B.bcm_graph_create(rp_h.data_ptr(), col_h.data_ptr(), g.n, g.m, g.directed, ptr_on_device=False,
                               stream=stream.cuda_stream)
        try:
            B.bcm_topk(h, k, hopts, ids_h.data_ptr(), far_h.data_ptr(), reach_h.data_ptr())
        finally:
            B.bcm_graph_destroy(h)

    e2e_t = []
    if not args.no_e2e:
        e2e_step()
    for _ in range(0 if args.no_e2e else max(3, min(args.steps, 20))):
        with torch.cuda.stream(stream):
            flush.zero_()
        torch.cuda.synchronize()
        t = time.perf_counter()
        e2e_step()
        e2e_t.append(time.perf_counter() - t)
    e2e_v = float(np.mean(e2e_t)) if e2e_t else None
    h2d = int(g.row_ptr.nbytes + g.col.nbytes)
    d2h = int(kk * (4 + 8 + 4))

    # roofline of the dominant kernel: the grid-wide or the per-CTA wave kernel,
    # whichever took longer (one launch each per step)
    peak, peak_kind = load_peaks()
    if st["seed_ms"] >= st["wave_ms"]:
        kname, kms, kbytes = "k_wave_grid", st["seed_ms"], st["grid_bytes"]
    else:
        kname, kms, kbytes = ("k_sparse" if st["sparse"] else "k_wave_cta"), st["wave_ms"], st["wave_bytes"]
    achieved = kbytes / (kms / 1e3) / 1e9 if kms > 0 else None
    src_hash = kernel_source_hash()
    traffic = profile_traffic(kname, src_hash, args.workload)
    roofline = {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                "peak_kind": "%s (MEASURED_PEAKS.json hbm_gbs)" % peak_kind if peak_kind == "measured"
                else "fallback 6.8 TB/s",
                "alg_bytes_per_launch": kbytes, "launch_ms": kms, "kernel_source": src_hash,
                "other_kernel": {"grid_ms": st["seed_ms"], "grid_bytes": st["grid_bytes"],
                                 "cta_ms": st["wave_ms"], "cta_bytes": st["wave_bytes"]}}

    # oracle: CPU baseline and a bit-exactness check on sampled outputs
    cpu = None
    bit_exact, verify_note, sampled = None, "skipped", None
    if not args.no_cpu or not args.no_verify:
        import oracle
        oracle.build()
    if not args.no_cpu:
        v, done, cores = cpu_sample(g, args.cpu_seconds)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "exhaustive BFS from %d uniformly drawn sources (about %.0f s of CPU work), "
                         "scaled by n/%d" % (done, args.cpu_seconds, done)}
    reach_all = None
    if not args.no_verify:
        import oracle
        h = B.BcmGraph.from_graph(g)
        _, xlo, _ = h.preprocess()
        reach_all = xlo
        h.close()
        of, orr = oracle.farness_all(g, sources=got_ids)
        exact = bool(np.array_equal(of, got_far) and np.array_equal(orr, got_reach))
        deg = g.degrees()
        cand = np.argsort(-deg, kind="stable")[:512].astype(np.uint32)
        rnd = graphgen.uniform_u32(99, 512, g.n)
        others = np.setdiff1d(np.concatenate([cand, rnd]), got_ids)
        sf, sr = oracle.farness_all(g, sources=others)
        kth = (int(got_reach[-1]), int(got_far[-1]), int(got_ids[-1]))

        def beats(f, r, v, kf):
            N = 0 if r <= 1 else (r - 1) ** 2
            F = 1 if r <= 1 else f
            Nk = 0 if kf[0] <= 1 else (kf[0] - 1) ** 2
            Fk = 1 if kf[0] <= 1 else kf[1]
            return N * Fk > Nk * F or (N * Fk == Nk * F and v < kf[2])

        none_better = not any(beats(int(f), int(r), int(v), kth) for f, r, v in zip(sf, sr, others))
        sampled = {"ok": bool(exact and none_better),
                   "note": "oracle BFS from the %d returned ids gives identical farness and reach; none of %d other "
                           "vertices (the 512 highest-degree and 512 random) ranks above the k-th" % (kk, len(others))}
        gold = load_golden(args.workload, k)
        if gold is None:
            bit_exact = None
            verify_note = ("no complete oracle answer is stored for this workload and k "
                           "(tests/golden/make_fullsize.py); only the sampled check ran")
        else:
            bit_exact = bool(gold["csr_sha256_16"] == g.hash64() and got_ids.tolist() == gold["ids"] and
                             got_far.tolist() == gold["farness"] and got_reach.tolist() == gold["reach"])
            verify_note = ("complete: ids, farness and reach equal, element by element, the exact top-%d the "
                           "oracle's sequential Algorithm 1 computed for this graph (%s, CSR hash %s)"
                           % (k, os.path.join("tests", "golden", "fullsize_%s_k%d.json" % (args.workload, k)),
                              gold["csr_sha256_16"]))
    if reach_all is None:
        h = B.BcmGraph.from_graph(g)
        _, reach_all, _ = h.preprocess()
        h.close()
    m_tot = m_tot_undirected(g, reach_all) if not g.directed else None

    line = {
        "metric": METRIC, "value": s_per_graph, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3, "higher_is_better": False,
        "scaling": "strong" if world > 1 else "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": "%s: %s" % (args.workload, WORKLOADS[args.workload]), "n": g.n, "m_arcs": g.m,
                   "k": k, "lanes": par["lanes"] or 64, "grid_lanes": par["grid_lanes"] or 128,
                   "pull_div": par["pull_div"] or 32, "threads": par["threads"] or (256 if st["sparse"] else 512),
                   "per_cta_kernel": "k_sparse (one source per CTA)" if st["sparse"] else "k_wave_cta (bit lanes)",
                   "launch_parameters": ("autotuned for this graph (%.2f s, outside the timed region)" % tuning_s)
                   if tuned else "library defaults" if not (args.lanes or args.threads or args.grid_lanes)
                   else "command line",
                   "l2": "256 MiB buffer written before every timed step",
                   "step": "graph handle from device CSR + preprocessing + top-k + release" +
                           (" (each rank its shard of the sources), all-gather of the k-entry lists, "
                            "merge on rank 0" if world > 1 else ""),
                   "parallelism": ("source shards over %d GPUs (chunks of 64 of the degree order)" % world)
                   if world > 1 else "single GPU"},
        "gteps": st["m_vis"] / s_per_graph / 1e9 * world if s_per_graph else None,
        "m_vis": st["m_vis"], "m_tot": m_tot,
        "m_vis_over_m_tot": (st["m_vis"] / m_tot) if m_tot else None,
        "stats": {key: st[key] for key in ("completed", "cut", "waves", "levels", "max_level", "visits",
                                            "kernel_ms", "preprocess_ms", "seed_ms", "wave_ms", "launches",
                                            "grid_waves", "grid_levels")},
        "per_k": per_k,
        "plain": plain,
        "speedup_vs_plain": (plain["s_per_graph"] / (total / args.steps)) if plain else None,
        "bit_exact": bit_exact, "verification": verify_note, "sampled_check": sampled,
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_v, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clk,
        "shards": None if world == 1 else {"rank0_shard_stats": {kk_: shard_stats[kk_] for kk_ in
                                                                  ("m_vis", "kernel_ms", "seed_ms", "wave_ms")},
                                           "merged_equals_single_gpu": same_as_single,
                                           "threshold_exchange": {
                                               "rounds_per_step": float(np.mean([x[0] for x in exchange_rounds])),
                                               "offers_per_step": float(np.mean([x[1] for x in exchange_rounds]))}},
        "wall_s_timed_region": t_wall,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
