"""Benchmark: maximal cliques/s of ParMCE on R-MAT scale 18 (edge factor 16).

Workload: the R-MAT graph (2^18 vertices, 16 * 2^18 samples, (a, b, c, d) =
(0.57, 0.19, 0.19, 0.05)) with the degeneracy rank, restricted to the
subproblems whose TTT search tree (Algorithm 1 on G_v, Algorithm 5) has at
most 2^24 nodes.  The full graph has far more maximal cliques than any
implementation can enumerate in a benchmark (scale 16 already exceeds 1.2e10);
the cap removes 17 of the 173,824 non-trivial subproblems and keeps about
1.5e9 cliques.  The capped set is fixed by the algorithm (tree size under the
stated rank and pivot rule), found in an untimed sizing pass and checked
against the oracle's list (tests/golden/rmat_18_capped.json).  The 17 left
out are far beyond a benchmark: 120 s of search on them reached 9.4e11 tree
nodes and 4.0e11 cliques without finishing (vertex 0 alone 8.7e11 nodes).

One step = the whole static path on input already resident in device memory:
CSR ingest of the raw edge samples, core-number ranking, Γ+ lists,
subproblem scheduling and the persistent search kernel over the fixed set,
ending with the summary (count, histogram, set hash) read back.

After the timed region the same line also reports the rest of the metric:
the rank comparison on the Chung-Lu 1.7M graph with planted cliques (rank
and enumeration time per rank, learned vs degree, degeneracy and triangles,
with makespan and imbalance: key "c3_ranks") and the incremental serving
loop on the Chung-Lu 500k graph with its 10^6-edge stream (edges/s, p50/p99
batch latency, per-batch latency against change size, and the same stream
deleted again batch by batch: key "c5_serving").

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
  python bench.py --workload batched   # 4,096 disjoint G(n, p), batched plan
  python bench.py --workload serve     # IMCE serving loop, Chung-Lu 500k + 1M stream edges
  python bench.py --workload ranks     # Chung-Lu 1.7M + planted cliques: rank and enumeration
                                       # time per rank (degree, degeneracy, triangles, learned)
  python bench.py --workload scaling   # search time against SMs covered; split on / off ablation

Under torchrun every rank runs the same workload as an independent replica
(the per-vertex subproblems need no exchange), the slowest
rank's time is used and value = cliques of all ranks / that time.
`--impl reference` times the CPU oracle (the paper's algorithms as plain C on
the host cores) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MCE wall time & cliques/s (bit-exact), learned vs degeneracy rank; IMCE p99"
UNIT = "cliques/s"
POPC_PER_CLK_PER_SM = 16       # 32-bit population counts per clock per SM (bounds AND+POPC word ops)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[3:7]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def replica_max(values, device):
    """Element-wise maximum of per-rank values over the process group (the
    slowest replica's times)."""
    import torch
    import torch.distributed as tdist
    t = torch.tensor(values, dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]


def whole_job_rate(units_per_replica, world, ms):
    """Units all replicas processed per second of the slowest replica."""
    return world * units_per_replica / (ms / 1000.0)


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


TREE_CAP = 1 << 24          # nodes per subproblem search tree in the benchmark set
# launch shape for this workload, from a sweep on GB300 (2, 3 or 4 resident
# blocks of 8 warps per SM x hand-over every 2048..32768 nodes x 1024..3040
# words of lane-search arena per warp): 2 x 12288 x 2048
BLOCKS_PER_SM = 2
SPLIT_NODES = 12288
LANE_SEARCH_WORDS = 2048
LANE_HOLD_WAITING = 0

# Counters of one k_bk launch of this workload from ncu, valid only for the
# kernel sources they were taken with (profiles/k_bk_rmat18.md): DRAM bytes
# (read + write) and warp instructions of one-pass captures of the whole
# timed launch.
K_BK_COUNTERS = {"dram_bytes": 984_233_216 + 899_319_296, "dram_tree_nodes": 4_057_750_785,
                 "warp_inst": 95_832_110_570, "inst_tree_nodes": 4_057_750_785,
                 "sha256": {"bk.cu": "32f53fb462e3b1fa3e9eac500a151b753cb0bbe334b7459c72b48e01db8c831d",
                            "bk.cuh": "46878bf93e68a8fac1a9fd948adb51137c5b9eebc0eb2775d789126daf185cab"}}


def _same_sources(digests) -> bool:
    import hashlib
    csrc = os.path.join(ROOT, "paper_2001_11433_gb300", "csrc")
    for name, digest in digests.items():
        with open(os.path.join(csrc, name), "rb") as f:
            if hashlib.sha256(f.read()).hexdigest() != digest:
                return False       # the kernel changed since the counters were taken
    return True


def k_bk_traffic(tree_nodes: int):
    if not _same_sources(K_BK_COUNTERS["sha256"]):
        return None
    return K_BK_COUNTERS["dram_bytes"] * tree_nodes / K_BK_COUNTERS["dram_tree_nodes"]


def issue_roofline(tree_nodes: int, kernel_s: float, sms: int, sm_mhz: float):
    """Issue-rate roofline of the search kernel: warp instructions per tree
    node (from the one-pass ncu capture of the whole launch) times the tree
    nodes per second, against 4 schedulers x SMs x clock (one warp
    instruction per scheduler per clock)."""
    if not _same_sources(K_BK_COUNTERS["sha256"]) or kernel_s <= 0:
        return None
    per_node = K_BK_COUNTERS["warp_inst"] / K_BK_COUNTERS["inst_tree_nodes"]
    achieved = per_node * tree_nodes / kernel_s
    peak = 4 * sms * sm_mhz * 1e6
    return {"bound": "issue", "achieved": achieved, "peak": peak, "unit": "warp instructions/s",
            "frac": achieved / peak, "warp_inst_per_tree_node": per_node,
            "peak_source": f"4 schedulers x {sms} SMs x {sm_mhz:.0f} MHz"}
CPU_NODE_BUDGET = 2_000_000   # tree nodes of the subproblem sample the CPU baseline times


def workload():
    import graphgen
    return graphgen.rmat_18()


def capped_vertices():
    """Subproblems of the R-MAT 18 workload whose search tree (degeneracy rank)
    has more than TREE_CAP nodes, as the oracle found them
    (tests/golden/rmat_18_capped.json, written by tests/golden/make_golden.py);
    None if that file is absent."""
    p = os.path.join(ROOT, "tests", "golden", "rmat_18_capped.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    assert d["tree_cap"] == TREE_CAP
    return np.array(d["capped_vertices"], dtype=np.int32)


def sample_prefix(subset, nodes, budget, seed):
    """A seeded permutation of the benchmark set, cut before the first
    subproblem that would take the sample past `budget` tree nodes.  No
    subproblem is skipped for its size: the sample is a plain prefix."""
    perm = np.random.default_rng(seed).permutation(subset)
    cum = np.cumsum(nodes[perm].astype(np.float64))
    k = int(np.searchsorted(cum, budget, side="right"))
    return np.sort(perm[:max(k, 1)]).astype(np.int32)


def cpu_baseline_same_set(w, sample, repeats=3):
    """Time the oracle (Algorithm 5 + Algorithm 1, degeneracy rank) on a
    sample of the benchmark set: one host thread and all host threads, median
    of `repeats` runs each (graph and rank built untimed).  Returns a dict."""
    import oracle as O
    g = O.Graph(w.n, w.u, w.v)
    rk = O.rank(g, "degen")
    out = {}
    for label, th in (("single_thread", 1), ("all_threads", os.cpu_count() or 1)):
        ts, r = [], None
        for _ in range(repeats):
            t0 = time.perf_counter()
            r = O.parmce(g, rk, subset=sample, threads=th, node_cap=TREE_CAP)
            ts.append(time.perf_counter() - t0)
        el = float(np.median(ts))
        out[label] = {"threads": th, "seconds": el, "cliques": r.count, "tree_nodes": r.nodes,
                      "cliques_per_s": r.count / el if el > 0 else 0.0, "hash": f"{r.hash:#018x}",
                      "runs_s": ts}
    return out


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle as O
    w = workload()
    threads = os.cpu_count() or 1
    g = O.Graph(w.n, w.u, w.v)
    rk = O.rank(g, "degen")
    capped = capped_vertices()
    pool = np.setdiff1d(np.arange(w.n, dtype=np.int32), capped if capped is not None else [])
    perm = np.random.default_rng(100).permutation(pool).astype(np.int32)
    target = max(2.0, 60.0 / max(1, args.warmup + args.steps))
    vals, pos, descs = [], 0, []
    for i in range(args.warmup + args.steps):
        cl, el, done, chunk = 0, 0.0, 0, 256
        while el < target and pos < len(perm):
            sub = perm[pos:pos + chunk]
            t0 = time.perf_counter()
            r = O.parmce(g, rk, subset=sub, threads=threads, node_cap=TREE_CAP)
            el += time.perf_counter() - t0
            cl += r.count
            pos += len(sub)
            done += len(sub)
            chunk *= 2
        if i >= args.warmup:
            vals.append(cl / el if el > 0 else 0.0)
            descs.append(done)
    value = float(np.median(vals)) if vals else 0.0
    desc = (f"oracle ParMCE (Algorithm 5 + Algorithm 1, degeneracy rank, {threads} threads, node cap {TREE_CAP}) "
            f"on consecutive chunks of one seeded permutation of the benchmark set (every vertex except the "
            f"{0 if capped is None else len(capped)} whose tree passes the cap); {int(np.median(descs)) if descs else 0} "
            f"subproblems per timed step (median), value = median over steps of cliques / seconds")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "dtype": "int32",
        "data": "synthetic", "scaling": "weak", "vs_baseline": None,
        "config": {"workload": f"{w.name}, degeneracy rank, subproblems with <= 2^24 tree nodes", "rank": "degen",
                   "sample": "bounded per step"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- our arm

def run_ours(args):
    import torch
    rank, world, local = dist_env()
    dist = world > 1
    if dist:
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import paper_2001_11433_gb300 as mce
    mce.load(build_if_missing=False)
    w = workload()
    m = len(w.u)
    dev_u = torch.from_numpy(w.u).cuda()
    dev_v = torch.from_numpy(w.v).cuda()
    pin_u = torch.from_numpy(w.u).pin_memory()
    pin_v = torch.from_numpy(w.v).pin_memory()
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")   # 512 MB > 129 MB L2

    # untimed sizing pass: the fixed set of subproblems with at most TREE_CAP tree nodes
    g0 = mce.Graph(w.n, dev_u, dev_v)
    pv = tuple(torch.zeros(w.n, dtype=torch.int64, device="cuda") for _ in range(3))
    r0 = mce.enumerate_cliques(g0, rank="degen", per_vertex=pv, subproblem_budget=TREE_CAP)
    nodes = pv[2].cpu().numpy().view(np.uint64)
    g0.close()
    subset_host = np.nonzero(nodes <= TREE_CAP)[0].astype(np.int32)
    excluded = int(w.n - len(subset_host))
    if args.sample < 1.0:
        # a seeded fraction of the set, for profiler captures of one short launch
        pick = np.random.default_rng(11).choice(len(subset_host), int(len(subset_host) * args.sample), replace=False)
        subset_host = np.sort(subset_host[pick])
    dev_subset = torch.from_numpy(subset_host).cuda()
    pin_subset = torch.from_numpy(subset_host).pin_memory()
    del pv, r0

    def step_device():
        g = mce.Graph(w.n, dev_u, dev_v)
        r = mce.enumerate_cliques(g, rank="degen", subset=dev_subset, blocks_per_sm=args.blocks_per_sm,
                                  split_nodes=args.split_nodes, warp_small_search=args.warp_small_search,
                                  lane_search_words=args.lane_search_words,
                                  lane_hold_waiting=args.lane_hold_waiting)
        g.close()
        return r

    def barrier():
        if dist:
            import torch.distributed as tdist
            tdist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        r = step_device()
    barrier()
    launches0 = mce.kernel_launches()
    sampler = ClockSampler(local)
    sampler.start()
    times, search_ms, word_ops, res = [], [], [], None
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        res = step_device()
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
        search_ms.append(res.ms_search)
        word_ops.append(res.word_ops)
    barrier()
    launches = mce.kernel_launches() - launches0
    # end to end through the public API with host buffers (pinned), result read back
    e2e_times = []
    for _ in range(max(1, min(2, args.steps))):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g = mce.Graph(w.n, pin_u.numpy(), pin_v.numpy())
        r2 = mce.enumerate_cliques(g, rank="degen", subset=pin_subset.numpy(), blocks_per_sm=args.blocks_per_sm,
                                   split_nodes=args.split_nodes, warp_small_search=args.warp_small_search,
                                  lane_search_words=args.lane_search_words,
                                  lane_hold_waiting=args.lane_hold_waiting)
        g.close()
        e2e_times.append((time.perf_counter() - t0) * 1000.0)
    clocks = sampler.stop()
    ms = float(np.mean(times))
    e2e_ms = float(np.mean(e2e_times))
    if dist:
        ms, e2e_ms = replica_max([ms, e2e_ms], "cuda")
    if rank != 0:
        return
    assert r2.count == res.count and r2.hash == res.hash
    count = res.count
    value = whole_job_rate(count, world, ms)
    peaks, peak_src = load_peaks()
    props = torch.cuda.get_device_properties(local)
    sm_mhz = clocks.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    peak_ops = POPC_PER_CLK_PER_SM * props.multi_processor_count * sm_mhz * 1e6
    kern_s = float(np.mean(search_ms)) / 1000.0
    achieved = float(np.mean(word_ops)) / kern_s if kern_s > 0 else 0.0
    # the capped set must be the one the oracle found (tests/golden/rmat_18_capped.json)
    capped = capped_vertices()
    capped_match = None
    if capped is not None and args.sample >= 1.0:
        capped_match = bool(np.array_equal(np.nonzero(nodes > TREE_CAP)[0], capped))
        assert capped_match, "capped subproblems differ from the oracle's"
    cpu = {"value": None, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle", "sample": "skipped"}
    if not args.no_cpu_baseline:
        sample = sample_prefix(subset_host, nodes, CPU_NODE_BUDGET, seed=7)
        base = cpu_baseline_same_set(w, sample)
        # the GPU on the very same subproblems (enumeration time: Γ+ lists, prepass, search)
        gs = mce.Graph(w.n, dev_u, dev_v)
        gpu_runs = [mce.enumerate_cliques(gs, rank="degen", subset=torch.from_numpy(sample).cuda(),
                                          blocks_per_sm=args.blocks_per_sm, split_nodes=args.split_nodes,
                                          warp_small_search=args.warp_small_search,
                                          lane_search_words=args.lane_search_words,
                                  lane_hold_waiting=args.lane_hold_waiting) for _ in range(3)]
        gs.close()
        assert all(x.count == base["all_threads"]["cliques"] for x in gpu_runs)
        assert all(f"{x.hash:#018x}" == base["single_thread"]["hash"] for x in gpu_runs)
        gpu_ms = float(np.median([x.ms_enum for x in gpu_runs]))
        cpu = {"value": base["all_threads"]["cliques_per_s"], "unit": UNIT, "cores": base["all_threads"]["threads"],
               "kind": "oracle",
               "sample": (f"{len(sample)} subproblems: a seeded permutation of the benchmark set cut before the first "
                          f"subproblem that would pass {CPU_NODE_BUDGET} tree nodes (no size filter); "
                          f"{base['all_threads']['cliques']} cliques, {base['all_threads']['tree_nodes']} tree nodes; "
                          "oracle ParMCE with the degeneracy rank, median of 3 runs, graph and rank built untimed"),
               "single_thread": base["single_thread"], "all_threads": base["all_threads"],
               "gpu_same_sample": {"enumerate_ms": gpu_ms, "cliques_per_s": gpu_runs[0].count / (gpu_ms / 1e3),
                                   "note": "mce_enumerate on the same subproblems, ms_enum (rank excluded like the "
                                           "oracle's), median of 3"}}
    secondary = {}
    if not args.no_secondary:
        secondary["c3_ranks"] = measure_ranks(mce, steps=3, warmup=1)
        secondary["c5_serving"] = measure_serve(mce)
        secondary["c5_serving"]["deletions"] = measure_deletions(mce)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": f"{w.name}, degeneracy rank, subproblems with <= 2^24 tree nodes",
                   "n": w.n, "edge_samples": m, "rank": "degen", "tree_cap": TREE_CAP,
                   "subproblems_excluded": excluded, "sample_fraction": args.sample, "cliques": count, "hash": f"{res.hash:#018x}",
                   "max_clique": len(res.hist) - 1, "tree_nodes": res.tree_nodes,
                   "tree_nodes_per_s": world * res.tree_nodes / (ms / 1000.0),
                   "l2": "512 MB buffer written between timed steps", "parallelism": f"replicas x{world}",
                   "launch": {"blocks_per_sm": args.blocks_per_sm, "warps_per_block": 8, "split_nodes": args.split_nodes,
                              "small_search": "warp" if args.warp_small_search else "lane-parallel",
                              "lane_search_words": args.lane_search_words,
                              "lane_hold_waiting": args.lane_hold_waiting}},
        "phases_ms": {"rank": res.ms_rank, "enumerate": res.ms_enum, "search_kernel": float(np.mean(search_ms))},
        "roofline": {"bound": "alu", "kernel": "k_bk (persistent search)", "achieved": achieved, "peak": peak_ops,
                     "unit": "word-ops/s", "frac": achieved / peak_ops if peak_ops else None,
                     "traffic": k_bk_traffic(res.tree_nodes), "traffic_unit": "DRAM bytes per launch",
                     "peak_source": f"{POPC_PER_CLK_PER_SM} POPC/clk/SM x {props.multi_processor_count} SMs x "
                                    f"{sm_mhz:.0f} MHz (median SM clock sampled during the run)",
                     "work": "per tree node (|cand|+|fini|)*ceil(|cand|/32) pivot AND+POPC words + "
                             "2*ceil((|cand|+|fini|)/32) per child + |K| per clique, counted by the kernel"},
        "e2e": {"value": whole_job_rate(count, world, e2e_ms), "unit": UNIT,
                "h2d_bytes_per_step": 8 * m + 4 * len(subset_host),
                "d2h_bytes_per_step": 8 * (16 + 1024) + 8 * 8},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "issue_roofline": issue_roofline(res.tree_nodes, kern_s, props.multi_processor_count, sm_mhz),
        "cpu_baseline": cpu,
        "capped_set_matches_oracle": capped_match,
        "balance": balance_stats(res),
        "peaks_source": peak_src,
        **secondary,
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- secondary workloads

def run_batched(args):
    """4,096 independent G(n, p) (n log-uniform in [32, 2048], p ~ U[0.1, 0.6])
    in one reusable plan: one persistent search launch per run, captured in a
    CUDA graph and replayed.  Dense graphs have astronomically many maximal
    cliques, so every graph gets the same search-tree node budget; graphs that
    finish within it are 'completed' and their cliques are what is counted."""
    import torch
    import graphgen
    import paper_2001_11433_gb300 as mce
    mce.load(build_if_missing=False)
    w = graphgen.batched_er_4096()
    gptr = w.extra["graph_ptr"]
    budget = args.graph_budget
    g = mce.Graph(w.n, torch.from_numpy(w.u).cuda(), torch.from_numpy(w.v).cuda())
    plan = mce.BatchedPlan(g, gptr, node_budget=budget)
    t0 = time.perf_counter()
    bps, split, ws = plan.tune(tune_budget=max(budget // 16, 1 << 12), repeats=1)
    tune_s = time.perf_counter() - t0
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        plan.run()
        plan.read()
    launches0 = mce.kernel_launches()
    sampler = ClockSampler(0)
    sampler.start()
    times, first = [], None
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        plan.run()
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
        out = plan.read()
        if first is None:
            first = out
        # graphs over budget stop at a timing-dependent point; completed ones are exact
        ok = first[2] == 0
        assert np.array_equal(out[2], first[2])
        assert np.array_equal(out[0][ok], first[0][ok]) and np.array_equal(out[1][ok], first[1][ok])
    launches = mce.kernel_launches() - launches0
    clocks = sampler.stop()
    counts, hashes, status, tot = first
    # after the timed region: the tuner again, at the full per-graph budget,
    # to check the shape it picked from the cheaper lowered-budget runs
    t1 = time.perf_counter()
    bps_full, split_full, ws_full = plan.tune(tune_budget=0, repeats=1)
    tune_full_s = time.perf_counter() - t1
    ok = status == 0
    ms = float(np.mean(times))
    done_cl = int(counts[ok].sum())
    # end to end: host arrays in, per-graph results out, through mce_enumerate_batched
    pin_u = torch.from_numpy(w.u).pin_memory()
    pin_v = torch.from_numpy(w.v).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g2 = mce.Graph(w.n, pin_u.numpy(), pin_v.numpy())
    c2, h2, s2, _ = mce.enumerate_batched(g2, gptr, node_budget=budget)
    e2e_ms = (time.perf_counter() - t0) * 1000.0
    g2.close()
    assert np.array_equal(s2, status) and np.array_equal(c2[ok], counts[ok])
    line = {
        "metric": "batched MCE: maximal cliques/s of the graphs completed within the per-graph budget",
        "value": done_cl / (ms / 1000.0), "unit": "cliques/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int32", "data": "synthetic",
        "config": {"workload": w.name, "graphs": len(gptr) - 1, "n": w.n, "edges": len(w.u),
                   "node_budget_per_graph": budget, "completed": int(ok.sum()),
                   "cliques_completed": done_cl, "cliques_all": int(tot.count), "tree_nodes": int(tot.tree_nodes),
                   "tree_nodes_per_s": tot.tree_nodes / (ms / 1000.0),
                   "tuned": {"blocks_per_sm": bps, "split_nodes": split, "warp_small_search": ws, "tune_s": tune_s,
                             "tune_budget": max(budget // 16, 1 << 12),
                             "best_at_full_budget": {"blocks_per_sm": bps_full, "split_nodes": split_full,
                                                     "warp_small_search": ws_full, "tune_s": tune_full_s},
                             "pick_matches_full_budget": (bps, split, ws) == (bps_full, split_full, ws_full)},
                   "l2": "512 MB buffer written between timed steps"},
        "e2e": {"value": done_cl / (e2e_ms / 1000.0), "unit": "cliques/s", "h2d_bytes_per_step": 8 * len(w.u)
                + 4 * len(gptr), "d2h_bytes_per_step": 20 * (len(gptr) - 1)},
        "gpu_launches": int(launches), "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def measure_serve(mce, slots=4, load=0.7):
    """IMCE serving: base Chung-Lu graph (n = 500,000, about 2M edges,
    exponent 2.3) and a stream of 10^6 new edges in batches of log-uniform size
    10^3..10^5.  Pass 1 submits every batch at time 0 (saturation: service
    throughput); pass 2 replays the stream on a fresh state with Poisson
    arrivals at `load` times that throughput (latency p50/p99).  Both passes
    must give the same per-batch results."""
    import torch
    import graphgen
    w = graphgen.chung_lu_stream()
    su, sv = w.extra["stream_u"], w.extra["stream_v"]
    sizes, gaps = w.extra["batch_sizes"], w.extra["gaps"]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    g = mce.Graph(w.n, torch.from_numpy(w.u).cuda(), torch.from_numpy(w.v).cuda())

    def one_pass(arrivals):
        srv = mce.Server(slots=slots)
        t0 = time.perf_counter()
        t = srv.add_tenant(g)
        open_s = time.perf_counter() - t0
        srv.reset_clock()
        launches0 = mce.kernel_launches()
        ids = [srv.submit(t, su[offs[i]:offs[i + 1]], sv[offs[i]:offs[i + 1]], arrival_ms=arrivals[i])
               for i in range(len(sizes))]
        infos = [srv.wait(i) for i in ids]
        st = srv.stats()
        launches = mce.kernel_launches() - launches0
        srv.close()
        assert all(i.status == 0 for i in infos)
        return st, infos, open_s, launches

    sat, sat_infos, open_s, _ = one_pass([0.0] * len(sizes))
    rate = sat["edges"] / (sat["span_ms"] / 1000.0)                 # edges/s at saturation
    mean_gap_ms = float(np.mean(sizes)) / (load * rate) * 1000.0
    arrivals = np.concatenate([[0.0], np.cumsum(gaps[:-1])]) * mean_gap_ms
    st, infos, _, launches = one_pass(list(arrivals))
    g.close()
    assert [(i.delta.new_hash, i.delta.sub_hash) for i in infos] == \
        [(i.delta.new_hash, i.delta.sub_hash) for i in sat_infos]
    return {
        "workload": w.name, "n": w.n, "base_edge_samples": len(w.u), "stream_edges": int(len(su)),
        "batches": int(len(sizes)), "slots": slots, "offered_load": load, "mean_gap_ms": mean_gap_ms,
        "imce_open_s": open_s, "edges_per_s": st["edges_per_s"], "span_ms": st["span_ms"],
        "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "max_ms": st["max_ms"],
        "wait_p50_ms": st["wait_p50_ms"], "wait_p99_ms": st["wait_p99_ms"],
        "saturation_edges_per_s": rate, "saturation_p50_ms": sat["p50_ms"], "saturation_p99_ms": sat["p99_ms"],
        "new_cliques": int(st["new_cliques"]), "subsumed_cliques": int(st["subsumed_cliques"]),
        "alive_after": int(infos[-1].delta.alive), "applied_edges": int(st["applied"]),
        "device_ms_total": float(sum(i.delta.ms for i in infos)), "gpu_launches": int(launches),
        "batch_latency": [{"edges": int(sizes[i]), "new": int(x.delta.new_count), "subsumed": int(x.delta.sub_count),
                           "device_ms": float(x.delta.ms)} for i, x in enumerate(sat_infos)],
        "latency_vs_change": latency_vs_change([int(sizes[i]) for i in range(len(sizes))],
                                               [int(x.delta.new_count + x.delta.sub_count) for x in sat_infos],
                                               [float(x.delta.ms) for x in sat_infos]),
    }


def measure_deletions(mce):
    """Edge deletions (imce_remove_edges, by the reduction G = (G - H) + H):
    the serving stream's 45 batches are added to the Chung-Lu 500k base graph
    (untimed), then deleted again in reverse order; each deletion batch is
    timed by the library (CUDA events around the call).  The clique set must
    return to the base graph's (same number of alive cliques, and every
    batch's removed cliques are the cliques its addition created)."""
    import torch
    import graphgen
    w = graphgen.chung_lu_stream()
    su, sv = w.extra["stream_u"], w.extra["stream_v"]
    sizes = w.extra["batch_sizes"]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    g = mce.Graph(w.n, torch.from_numpy(w.u).cuda(), torch.from_numpy(w.v).cuda())
    st = mce.Imce(g)
    alive0 = st.add_edges(np.zeros(0, np.int32), np.zeros(0, np.int32)).alive
    du = [torch.from_numpy(np.ascontiguousarray(su[offs[i]:offs[i + 1]])).cuda() for i in range(len(sizes))]
    dv = [torch.from_numpy(np.ascontiguousarray(sv[offs[i]:offs[i + 1]])).cuda() for i in range(len(sizes))]
    added = [st.add_edges(du[i], dv[i]) for i in range(len(sizes))]
    launches0 = mce.kernel_launches()
    dels = {}
    for i in reversed(range(len(sizes))):
        dels[i] = st.remove_edges(du[i], dv[i])
    launches = mce.kernel_launches() - launches0
    alive_end = dels[0].alive
    st.close()
    g.close()
    for i in range(len(sizes)):
        assert (dels[i].sub_count, dels[i].sub_hash) == (added[i].new_count, added[i].new_hash), i
        assert (dels[i].new_count, dels[i].new_hash) == (added[i].sub_count, added[i].sub_hash), i
    assert alive_end == alive0
    ms = np.array([dels[i].ms for i in range(len(sizes))], float)
    edges = int(sum(dels[i].applied for i in range(len(sizes))))
    return {"batches": int(len(sizes)), "edges": edges, "device_ms_total": float(ms.sum()),
            "edges_per_s": edges / (ms.sum() / 1000.0), "batch_ms_p50": float(np.percentile(ms, 50)),
            "batch_ms_p99": float(np.percentile(ms, 99)),
            "removed_cliques": int(sum(dels[i].sub_count for i in range(len(sizes)))),
            "created_cliques": int(sum(dels[i].new_count for i in range(len(sizes)))),
            "alive_restored": bool(alive_end == alive0), "gpu_launches": int(launches),
            "latency_vs_change": latency_vs_change([int(sizes[i]) for i in range(len(sizes))],
                                                   [int(dels[i].new_count + dels[i].sub_count)
                                                    for i in range(len(sizes))], list(ms))}


def latency_vs_change(edges, changes, ms):
    """Device time of a batch against its size and its change |Λnew| + |Λdel|
    (the analogue of the paper's latency-against-change-size figure): least-
    squares line ms = a + b * x for each, with the correlation."""
    out = {}
    for name, x in (("per_edge", np.asarray(edges, float)), ("per_changed_clique", np.asarray(changes, float))):
        y = np.asarray(ms, float)
        if len(x) < 2 or np.ptp(x) == 0:
            out[name] = None
            continue
        b, a = np.polyfit(x, y, 1)
        out[name] = {"intercept_ms": float(a), "ms_per_1000": float(b * 1000.0),
                     "correlation": float(np.corrcoef(x, y)[0, 1])}
    return out


def run_serve(args):
    import paper_2001_11433_gb300 as mce
    mce.load(build_if_missing=False)
    sampler = ClockSampler(0)
    sampler.start()
    m = measure_serve(mce, args.slots, args.load)
    m["deletions"] = measure_deletions(mce)
    clocks = sampler.stop()
    line = {
        "metric": "IMCE serving: edges/s and p99 batch latency (arrival to completion)",
        "value": m["edges_per_s"], "unit": "edges/s", "n_gpus": 1, "steps": m["batches"], "warmup": 0,
        "ms_per_step": m["span_ms"] / m["batches"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {k: m[k] for k in ("workload", "n", "base_edge_samples", "stream_edges", "batches", "slots",
                                     "offered_load", "mean_gap_ms", "imce_open_s", "saturation_edges_per_s",
                                     "saturation_p50_ms", "saturation_p99_ms")},
        "latency_ms": {"p50": m["p50_ms"], "p99": m["p99_ms"], "max": m["max_ms"],
                       "wait_p50": m["wait_p50_ms"], "wait_p99": m["wait_p99_ms"]},
        "cliques": {"new": m["new_cliques"], "subsumed": m["subsumed_cliques"], "alive_after": m["alive_after"],
                    "applied_edges": m["applied_edges"]},
        "device_ms_total": m["device_ms_total"],
        "deletions": m["deletions"],
        "e2e": {"value": m["edges_per_s"], "unit": "edges/s", "h2d_bytes_per_step": int(8 * m["stream_edges"] /
                                                                                       m["batches"]),
                "d2h_bytes_per_step": 2 * 8 * (1024 + 8)},
        "gpu_launches": m["gpu_launches"], "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def independent_sets(row, col, rounds=4, seed=5):
    """`rounds` disjoint independent sets of a CSR graph (each vertex with a
    neighbour at most once): a vertex joins when its random priority is below
    all its neighbours' (vertices already taken never join again)."""
    n = len(row) - 1
    deg = np.diff(row)
    has = deg > 0
    rng = np.random.default_rng(seed)
    done = np.zeros(n, bool)
    out = []
    for _ in range(rounds):
        pri = rng.random(n)
        pri[done] = 2.0                      # already taken: never chosen, never blocks
        nb_min = np.full(n, 3.0)
        nb_min[has] = np.minimum.reduceat(pri[col], row[:-1][has])
        S = np.nonzero((pri < nb_min) & has & ~done)[0].astype(np.int32)
        out.append(S)
        done[S] = True
    return out


def lowest_first_rank(n, S):
    """A total rank (permutation of [0, n)) with the vertices of S lowest, in
    id order, then every other vertex in id order."""
    rank = np.empty(n, np.int32)
    rest = np.setdiff1d(np.arange(n, dtype=np.int32), S, assume_unique=True)
    rank[S] = np.arange(len(S), dtype=np.int32)
    rank[rest] = np.arange(len(S), n, dtype=np.int32)
    return rank


def neighbourhood_cost_labels(mce, g, rounds=4, seed=5):
    """Training labels for the learned rank key: log(1 + TTT tree nodes) of
    each sampled vertex's whole neighbourhood (cand = Γ(v), fini = ∅: the cost
    of v's subproblem if v were ranked lowest).  Section 4.2 ranks a vertex
    higher the costlier its neighbourhood, so that its own subproblem (the
    higher-ranked neighbours only) stays small.  For each independent set S,
    a user rank puts S below every other vertex and only the subproblems of S
    run: each then has its whole neighbourhood as candidates."""
    import torch
    n = g.n
    row, col = g.csr()
    vs, ls = [], []
    for S in independent_sets(row, col, rounds, seed):
        rank = lowest_first_rank(n, S)
        pv = tuple(torch.zeros(n, dtype=torch.int64, device="cuda") for _ in range(3))
        mce.enumerate_cliques(g, rank="user", user_rank=torch.from_numpy(rank).cuda(),
                              subset=torch.from_numpy(S).cuda(), per_vertex=pv)
        nodes = pv[2].cpu().numpy()[S].astype(np.float64)
        vs.append(S)
        ls.append(np.log1p(nodes).astype(np.float32))
    return np.concatenate(vs), np.concatenate(ls)


def train_learned_model(mce):
    """Two MLPs 8-64-64-1 on the one-pass features (degrees only), trained
    (FP32, on the GPU, the library's own kernels) on a smaller Chung-Lu graph
    of the C3 family (n = 200,000, another seed):
      rank model  - log(1 + search-tree nodes) of a vertex's whole
                    neighbourhood (neighbourhood_cost_labels); its prediction
                    is the rank key (Section 4.2: costlier ranks higher);
      split model - log(1 + search-tree nodes) of each subproblem under the
                    learned rank, recorded by the search itself; it orders the
                    subproblems and marks the heavy ones for early splitting.
    Returns (rank model, split model, info)."""
    import torch
    import graphgen
    tu, tv, _ = graphgen.chung_lu(200_000, 2.2, 35_000.0 * (200_000 / 1_700_000) ** 0.5, 200_000 * 6.47,
                                  graphgen.substream_seed(graphgen.BASE_SEED + 103, 0))
    tg = mce.Graph(200_000, torch.from_numpy(tu).cuda(), torch.from_numpy(tv).cuda())
    t0 = time.perf_counter()
    lab_v, lab = neighbourhood_cost_labels(mce, tg, rounds=4, seed=5)
    feat = mce.features(tg, kind="light")
    model = mce.Model(64, seed=3, features="light")
    loss = model.train(feat[torch.from_numpy(lab_v).cuda().long()].contiguous(), torch.from_numpy(lab).cuda(),
                       epochs=60, batch=2048, lr=3e-3, seed=4)
    pv = tuple(torch.zeros(200_000, dtype=torch.int64, device="cuda") for _ in range(3))
    mce.enumerate_cliques(tg, rank="learned", model=model, per_vertex=pv)
    sub_lab = torch.log1p(pv[2].double()).float()
    split_model = mce.Model(64, seed=5, features="light")
    loss2 = split_model.train(feat.contiguous(), sub_lab.contiguous(), epochs=30, batch=4096, lr=3e-3, seed=6)
    train_s = time.perf_counter() - t0
    tg.close()
    return model, split_model, {"graph": "chung-lu n=200000, other seed", "features": "one pass (degrees only)",
                                "rank_labels": int(len(lab)),
                                "rank_label": "log1p(tree nodes of the whole neighbourhood)", "rank_final_mse": loss,
                                "split_label": "log1p(tree nodes of the subproblem under the learned rank)",
                                "split_final_mse": loss2, "seconds": train_s}


def balance_stats(r):
    """Makespan and per-warp busy-time imbalance of one search launch, from
    the kernel's own counters (stats: build ns, search ns, idle ns, builds,
    pieces, largest busy ns of one warp, warps, endgame ns)."""
    st = r.stats
    warps = max(st[6], 1)
    mean_busy = (st[0] + st[1]) / warps
    return {"search_ms": r.ms_search, "max_warp_busy_ms": st[5] / 1e6, "mean_warp_busy_ms": mean_busy / 1e6,
            "imbalance": st[5] / mean_busy if mean_busy else None, "idle_frac": st[2] / max(st[0] + st[1] + st[2], 1),
            "endgame_ms": st[7] / 1e6, "pieces": st[4], "builds": st[3],
            "build_frac": st[0] / max(st[0] + st[1], 1)}


def measure_ranks(mce, steps=3, warmup=1, kinds=("degree", "degen", "triangle", "learned", "learned_split")):
    """Chung-Lu n = 1.7M (exponent 2.2, w_max 35,000, about 11M edges) plus
    200 planted cliques of size U[20, 60].  Per rank: rank time (RT) and
    enumeration time (ET), CUDA events inside the library, median of the timed
    runs, with the search's makespan and imbalance; every rank must give the
    same clique set (count, hash, histogram)."""
    import torch
    import graphgen
    w = graphgen.chung_lu_planted()
    g = mce.Graph(w.n, torch.from_numpy(w.u).cuda(), torch.from_numpy(w.v).cuda())
    model, split_model, train = (train_learned_model(mce) if any(k.startswith("learned") for k in kinds)
                                 else (None, None, None))
    out, ref = {}, None
    for kind in kinds:
        # the learned configuration: the rank model's key (Section 4.2); the
        # split model's heavy-subtree marking is measured beside it
        kw = {"rank": kind}
        if kind == "learned":
            kw = {"rank": "learned", "model": model}
        elif kind == "learned_split":
            kw = {"rank": "learned", "model": model, "split_model": split_model, "heavy_nodes": 4096,
                  "heavy_split_nodes": 256}
        runs = []
        for it in range(warmup + steps):
            r = mce.enumerate_cliques(g, **kw)
            if it >= warmup:
                runs.append(r)
        key = (runs[0].count, runs[0].hash, tuple(runs[0].hist))
        ref = ref or key
        assert key == ref, f"{kind}: clique set differs"
        rt = float(np.median([x.ms_rank for x in runs]))
        et = float(np.median([x.ms_enum for x in runs]))
        mid = sorted(runs, key=lambda x: x.ms_enum)[len(runs) // 2]
        out[kind] = {"rt_ms": rt, "et_ms": et, "total_ms": rt + et, "cliques_per_s": runs[0].count / ((rt + et) / 1e3),
                     "tree_nodes": runs[0].tree_nodes, "splits": mid.tasks_split, **balance_stats(mid)}
    g.close()
    best = min(out, key=lambda k: out[k]["total_ms"])
    return {"workload": w.name, "n": w.n, "edge_samples": len(w.u), "cliques": ref[0], "hash": f"{ref[1]:#018x}",
            "max_clique": len(ref[2]) - 1, "learned_train": train, "fastest_rank": best, "ranks": out,
            "steps": steps, "warmup": warmup}


def run_ranks(args):
    import paper_2001_11433_gb300 as mce
    mce.load(build_if_missing=False)
    m = measure_ranks(mce, args.steps, args.warmup)
    out = m["ranks"]
    line = {
        "metric": "MCE wall time (RT + ET) and cliques/s per rank, learned vs degeneracy (bit-exact across ranks)",
        "value": out["degen"]["cliques_per_s"], "unit": "cliques/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": out["degen"]["total_ms"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32 (features FP32, inference BF16)", "data": "synthetic",
        "config": {k: m[k] for k in ("workload", "n", "edge_samples", "cliques", "hash", "max_clique", "learned_train",
                                     "fastest_rank")},
        "ranks": out,
    }
    print(json.dumps(line), flush=True)


def run_scaling(args):
    """Search time of the R-MAT 18 benchmark set against the number of SMs
    the persistent grid covers (the analogue of the paper's thread-scaling
    figures), and the split ablation (hand-over of subtrees on / off, the
    PECO-style comparison of Section 4.2) on R-MAT 18 and on the Chung-Lu
    1.7M graph (degree rank)."""
    import torch
    import graphgen
    import paper_2001_11433_gb300 as mce
    mce.load(build_if_missing=False)
    props = torch.cuda.get_device_properties(0)
    w = workload()
    capped = capped_vertices()
    keep = np.setdiff1d(np.arange(w.n, dtype=np.int32), capped if capped is not None else [])
    g = mce.Graph(w.n, torch.from_numpy(w.u).cuda(), torch.from_numpy(w.v).cuda())
    sub = torch.from_numpy(keep).cuda()

    def timed(gr, reps=2, **kw):
        rs = [mce.enumerate_cliques(gr, **kw) for _ in range(reps + 1)][1:]
        r = min(rs, key=lambda x: x.ms_search)
        return {"search_ms": r.ms_search, "enumerate_ms": r.ms_enum, "cliques": r.count, "hash": f"{r.hash:#018x}",
                "tree_nodes": r.tree_nodes, "splits": r.tasks_split, **balance_stats(r)}

    sms = props.multi_processor_count
    scaling = {}
    for k in (sms // 8, sms // 4, sms // 2, sms):
        scaling[str(k)] = timed(g, rank="degen", subset=sub, blocks_per_sm=BLOCKS_PER_SM, split_nodes=SPLIT_NODES,
                                lane_search_words=LANE_SEARCH_WORDS, sm_limit=k)
        print(json.dumps({"sms": k, **scaling[str(k)]}), flush=True)
    ablation = {"rmat18_split_on": scaling[str(sms)],
                "rmat18_split_off": timed(g, reps=1, rank="degen", subset=sub, blocks_per_sm=BLOCKS_PER_SM,
                                             lane_search_words=LANE_SEARCH_WORDS, split=False)}
    c3 = graphgen.chung_lu_planted()
    g3 = mce.Graph(c3.n, torch.from_numpy(c3.u).cuda(), torch.from_numpy(c3.v).cuda())
    ablation["chunglu_split_on"] = timed(g3, rank="degree")
    ablation["chunglu_split_off"] = timed(g3, rank="degree", split=False)
    line = {"metric": "search time against SMs covered, and the split ablation", "unit": "ms",
            "higher_is_better": False, "n_gpus": 1, "data": "synthetic",
            "config": {"workload": f"{w.name} benchmark set (degeneracy rank) and {c3.name} (degree rank)"},
            "sm_scaling": scaling, "split_ablation": ablation}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-secondary", action="store_true",
                    help="rmat18: skip the Chung-Lu rank comparison and the serving loop after the timed region")
    ap.add_argument("--sample", type=float, default=1.0, help="rmat18: timed fraction of the subproblem set")
    ap.add_argument("--workload", choices=["rmat18", "batched", "serve", "ranks", "scaling"], default="rmat18")
    ap.add_argument("--blocks-per-sm", type=int, default=BLOCKS_PER_SM, help="rmat18: resident search blocks per SM")
    ap.add_argument("--split-nodes", type=int, default=SPLIT_NODES, help="rmat18: proactive hand-over interval (nodes)")
    ap.add_argument("--lane-search-words", type=int, default=LANE_SEARCH_WORDS,
                    help="rmat18: per-warp shared words of the lane-parallel small search (0 = automatic)")
    ap.add_argument("--lane-hold-waiting", type=int, default=LANE_HOLD_WAITING,
                    help="rmat18: waiting warps from which small subtrees stay with the whole warp")
    ap.add_argument("--warp-small-search", action="store_true",
                    help="rmat18: search small subtrees with the whole warp (the lane-parallel search is the default)")
    ap.add_argument("--graph-budget", type=int, default=1 << 20, help="batched: tree nodes per graph")
    ap.add_argument("--slots", type=int, default=4, help="serve: concurrent batches")
    ap.add_argument("--load", type=float, default=0.7, help="serve: offered load / saturation throughput")
    args = ap.parse_args()
    if args.workload == "batched":
        run_batched(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "ranks":
        run_ranks(args)
    elif args.workload == "scaling":
        run_scaling(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
