#!/usr/bin/env python
"""Benchmark of the triad-census hot path on B300 (one JSON line on stdout).

A step is one pass of the whole hot path over the workload's arc list, which
is already resident in HBM: the device graph build (dedup, tagged adjacency)
and the census (vertex ranks, suffix and dyadic terms, forward lists, the
triangle lookups, fold and 003 closure).  `census_ms` is the census alone.
`value` is an effective rate: sum over canonical dyads of |N(u)|+|N(v)|
(= sum_v d_v^2, what a full union merge of every dyad would read) per second
of step time; the census reads far less than that, so `roofline` reports the
dominant kernel against its own algorithmic bytes.  The default run (c3)
adds sub-records for the heavy-skew workload (`c5`) and the batched one
(`c4`: graphs/s of a CUDA-graph plan replay, each graph checked against the
oracle's stored census).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload c3]
    python bench.py --impl reference ...   # the CPU oracle on host cores

With N > 1 (torchrun) every rank censuses its own replica of the workload
(weak scaling, no collective on the data path); only the timing uses a
barrier and a max over ranks.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "census time; merged adjacency entries/s vs HBM roofline; graphs/s batched"
UNIT = "effective merged adjacency entries/s (full-union equivalent)"
WORKLOAD_DESC = {
    "c1": "G(n,p) n=1024 p=8/1023 reciprocity 0.25 seed 1",
    "c2": "R-MAT scale 20 edge factor 8 (.57,.19,.19,.05) 10% reciprocated, ids permuted, seed 2",
    "c3": "R-MAT scale 22 edge factor 4 (.57,.19,.19,.05), arcs oriented high->low id, ids permuted, seed 3",
    "c3s": "R-MAT scale 21 edge factor 4, arcs oriented high->low id, ids permuted, seed 3 (profiling case)",
    "c4": "4096 graphs, n log-uniform in [64, 65536], even G(n,p) mean out-degree U(4,32), odd R-MAT edge factor 8, reciprocity U(0,0.5), seed 4",
    "c5": "Chung-Lu n=2^22 gamma 2.1 mean total degree 16, largest realised degree ~1e5, reciprocity 0.15, seed 5",
}
# graph-build launches on the bucket path with no crowded hub segment (c3, c5):
# k_bkt_hist, 3 scan kernels, k_bkt_scatter, k_bkt_rows, k_rows, k_long_split_w,
# k_long_split, k_seg_sort, k_big_sort, k_long_count, 3 scan kernels,
# k_compact, k_long_write, k_rowstats, k_fill_tail
OWN_BUILD_KERNELS = 19
FLUSH_BYTES = 512 << 20  # > 126 MB L2


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # let nvidia-smi start and take its first sample before the timed
            # steps, so its start-up does not land inside one of them
            t0 = time.perf_counter()
            while not self.lines and self.proc.poll() is None and time.perf_counter() - t0 < 3.0:
                time.sleep(0.01)
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        backend = "gloo" if args.impl == "reference" else "nccl"
        dist.init_process_group(backend=backend)
        pg = dist
    return world, rank, local, pg


def max_over_ranks(x, pg):
    if pg is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64)
    if pg.get_backend() == "nccl":
        t = t.cuda()
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def barrier(pg):
    if pg is not None:
        pg.barrier()


# ------------------------------------------------------------ CPU oracle arm

def vertex_costs(arcs):
    """Merged entries (d_u + d_v summed over the canonical dyads <u,v>, u < v)
    charged to each vertex as the dyads' lower endpoint: sample sizing only."""
    n = arcs.n
    s = arcs.src.astype(np.int64)
    d = arcs.dst.astype(np.int64)
    keep = s != d
    u = np.minimum(s[keep], d[keep])
    v = np.maximum(s[keep], d[keep])
    key = np.unique(u * n + v)
    u = key // n
    v = key - u * n
    deg = np.bincount(u, minlength=n) + np.bincount(v, minlength=n)
    return np.bincount(u, weights=(deg[u] + deg[v]).astype(np.float64), minlength=n)


def cost_ranges(cost, target, cap, rng):
    """Consecutive vertex ranges of about `target` merged entries each (a
    heavier vertex forms a range of its own), in random order; ranges above
    `cap` are left out.  Returns [(a, b, entries)], and the number left out."""
    cc = np.cumsum(cost)
    cuts = np.unique(np.searchsorted(cc, np.arange(target, cc[-1], target), side="right"))
    bounds = np.concatenate([[0], cuts[(cuts > 0) & (cuts < cost.size)], [cost.size]])
    csum = np.concatenate([[0.0], cc])
    out, skipped = [], 0
    for a, b in zip(bounds[:-1], bounds[1:]):
        c = csum[b] - csum[a]
        if c > cap:
            skipped += 1
        elif c > 0:
            out.append((int(a), int(b), float(c)))
    order = rng.permutation(len(out))
    return [out[k] for k in order], skipped


def oracle_sample_rate(arcs, seconds, threads=None, cost=None, seed=0, og=None):
    """Run the oracle census on random disjoint vertex ranges (the dyads whose
    lower endpoint lies in a range) on `threads` host threads, the ranges
    chosen by their merged entries so that the run takes about `seconds` of
    wall time.  A range whose entries one thread could not finish within that
    time (a hub as lower endpoint) is left out."""
    import oracle
    threads = threads or os.cpu_count() or 1
    rng = np.random.default_rng(seed)
    cost = vertex_costs(arcs) if cost is None else cost
    own = og is None  # an oracle graph built here is freed here
    if own:
        og = oracle.Graph(arcs.n, arcs.src, arcs.dst)
    # calibrate the single-thread rate on ~0.25 s of small ranges
    cal, _ = cost_ranges(cost, 2e5, 2e7, rng)
    e_cal, t = 0, time.perf_counter()
    for a, b, _ in cal:
        e_cal += og.census_range(a, b)[1]
        if time.perf_counter() - t > 0.25:
            break
    rate1 = max(e_cal, 1) / max(time.perf_counter() - t, 1e-4)
    budget = seconds * threads * rate1
    ranges, skipped = cost_ranges(cost, budget / (threads * 16), seconds * rate1, rng)
    take, acc = [], 0.0
    for r in ranges:
        if acc >= budget:
            break
        take.append(r)
        acc += r[2]
    lock = threading.Lock()
    done = {"entries": 0, "vertices": 0}

    def work():
        while True:
            with lock:
                if not take:
                    return
                a, b, _ = take.pop()
            _, e = og.census_range(a, b)
            with lock:
                done["entries"] += e
                done["vertices"] += b - a

    t = time.perf_counter()
    pool = [threading.Thread(target=work) for _ in range(threads)]
    for th in pool:
        th.start()
    for th in pool:
        th.join()
    wall = time.perf_counter() - t
    if own:
        og.close()
    return done["entries"] / max(wall, 1e-9), threads, done["vertices"], done["entries"], wall, skipped


def run_reference_batched(args, world):
    """The oracle on a bounded sample of the batched workload's graphs, graphs
    processed in parallel on the host threads (one graph per thread)."""
    import oracle
    import synth
    b = synth.c4()
    G = len(b)
    threads = os.cpu_count() or 1
    order = np.random.default_rng(4).permutation(G)
    per_step_s = max(2.0, min(8.0, 150.0 / max(1, args.steps + args.warmup)))
    rates, walls, done_total = [], [], 0
    k = 0
    for i in range(args.warmup + args.steps):
        graphs = 0
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < per_step_s:  # whole graphs, all host threads each
            a = b.graph(int(order[k % G]))
            k += 1
            og = oracle.Graph(a.n, a.src, a.dst)
            og.census(threads)
            og.close()
            graphs += 1
        wall = time.perf_counter() - t0
        if i >= args.warmup:
            rates.append(graphs / wall)
            walls.append(wall)
            done_total += graphs
    value = float(np.mean(rates))
    sample = (f"oracle census of {done_total} of the {G} c4 graphs (a fixed random order, each graph on "
              f"all {threads} host threads, ~{per_step_s:.0f} s per step)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "graphs/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(walls)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": f"c4: {WORKLOAD_DESC['c4']}", "graphs": G,
                   "parallelism": f"host threads x{threads}"},
        "cpu_baseline": {"value": value, "unit": "graphs/s", "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "graphs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_reference(args, world, rank, pg):
    import synth
    if rank != 0:
        return
    if args.workload == "c4":
        return run_reference_batched(args, world)
    arcs = synth.WORKLOADS[args.workload]()
    import oracle
    og = oracle.Graph(arcs.n, arcs.src, arcs.dst)
    stats = og.stats()
    threads = os.cpu_count() or 1
    per_step_s = max(2.0, min(8.0, 150.0 / max(1, args.steps + args.warmup)))
    rates, walls = [], []
    cost = vertex_costs(arcs)
    for i in range(args.warmup + args.steps):
        rate, thr, verts, ents, wall, skipped = oracle_sample_rate(arcs, per_step_s, threads, cost, seed=i, og=og)
        if i >= args.warmup:
            rates.append(rate)
            walls.append(wall)
    value = float(np.mean(rates))
    sample = (f"oracle census of the canonical dyads whose lower endpoint lies in random disjoint vertex "
              f"ranges sized by their merged entries (~{per_step_s:.0f} s per step on {threads} host "
              f"threads; ranges one thread could not finish in that time, {skipped} of them, left "
              f"out) of workload {args.workload}; rate = merged entries processed / wall time")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(walls)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": f"{args.workload}: {WORKLOAD_DESC.get(args.workload, '')}",
                   "n": arcs.n, "arcs": stats["arcs"], "merged_entries": stats["merged_entries"],
                   "parallelism": f"host threads x{threads}"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------ native arm

def dominant_kernel(tc, profs, stats):
    """The census kernel with the largest share of the step, its algorithmic
    bytes per launch and its event-timed duration.  Forward path: the tag-map
    lookups (k_tri_big) read, per lookup, one 4-byte lookup-list entry; per
    dyad record 16 B; per staged owner-list entry 4 B; per triangle the 4-byte
    rank-permutation entry of its third vertex.  Merge path: k_owner (4 B per
    lookup plus 4 B per indexed owner entry)."""
    pl = profs[-1]
    mean = lambda k: float(np.mean([p[k] for p in profs]))
    if pl["fwd_entries"] > 0:
        kern = {"k_tri_big": "ms_tri_map", "k_tri_small": "ms_tri_search", "forward lists": "ms_forward",
                "task pass": "ms_tasks", "k_fold": "ms_fold"}
        ms = {k: mean(f) for k, f in kern.items()}
        big = {"kernel": "k_tri_big", "ms": ms["k_tri_big"],
               "bytes": 4 * pl["map_lookups"] + 16 * pl["map_dyads"] + 4 * pl["map_list_entries"]
               + 4 * pl["map_triangles"],
               "units": {"lookups": pl["map_lookups"], "dyad_records": pl["map_dyads"],
                         "staged_list_entries": pl["map_list_entries"], "triangles": pl["map_triangles"]},
               "bytes_per_unit": "4 B per lookup-list entry + 16 B per dyad record + 4 B per staged "
                                 "owner-list entry + 4 B per triangle (third vertex's id)"}
        small = {"kernel": "k_tri_small", "ms": ms["k_tri_small"],
                 "bytes": 4 * pl["search_lookups"] + 16 * pl["search_dyads"] + 4 * pl["search_triangles"]}
        top = big if big["ms"] >= small["ms"] else small
    else:
        kern = {"task pass": "ms_tasks", "k_owner_prep": "ms_owner_prep", "k_owner": "ms_owner",
                "merge kernels": "ms_merge", "k_fold": "ms_fold"}
        ms = {k: mean(f) for k, f in kern.items()}
        top = {"kernel": "k_owner", "ms": ms["k_owner"], "bytes": 4 * (pl["owner_probes"] + pl["owner_staged"]),
               "units": {"lookups": pl["owner_probes"], "indexed_owner_entries": pl["owner_staged"]},
               "bytes_per_unit": "4 B per lookup + 4 B per indexed owner entry"}
    return top, ms


def source_key():
    """sha256 prefix of the census kernels' code (census.cu, forward.cuh) with
    comments and blank space removed: the key under which profiles/issue.txt
    and profiles/traffic.txt store counters, so that a record is used only on
    the code it was taken on, and comment edits do not void it."""
    import hashlib
    import re
    csrc = os.path.join(ROOT, "paper_1603_02655_b300", "csrc")
    h = hashlib.sha256()
    for f in ("census.cu", "forward.cuh"):
        text = open(os.path.join(csrc, f)).read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


def issue_record(kernel):
    """Warp instructions per lookup of `kernel` from the committed ncu summary
    (profiles/issue.txt), if it was taken on the current kernel code."""
    sha = source_key()
    try:
        for line in open(os.path.join(ROOT, "profiles", "issue.txt")):
            parts = line.split()
            if len(parts) >= 3 and parts[0] == kernel and parts[2] == sha:
                return float(parts[1]), sha
    except OSError:
        pass
    return None, sha


def recorded_traffic_fwd(kernel, sha):
    """DRAM bytes per lookup of `kernel` from profiles/traffic.txt for this
    source (None if the capture predates it)."""
    try:
        for line in open(os.path.join(ROOT, "profiles", "traffic.txt")):
            parts = line.split()
            if len(parts) >= 3 and parts[0] == kernel and parts[2] == sha:
                return float(parts[1])
    except OSError:
        pass
    return None


def time_census(tc, torch, g, opts, out, stream, flush, steps):
    """CUDA-event times (ms) of `steps` census calls, L2 flushed before each."""
    ts = []
    for k in range(steps):
        flush.fill_(k)
        a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        tc.tc_census(g, opts, out=out, stream=stream)
        c.record(stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(c))
    return ts


def c5_record(tc, torch, stream, flush, steps, peak):
    """The heavy-skew Chung-Lu workload: census time (device-resident graph,
    default options), the dominant kernel's own-byte fraction, and the census
    checked against the oracle's stored census."""
    import synth
    a = synth.c5()
    src = torch.from_numpy(a.src).cuda()
    dst = torch.from_numpy(a.dst).cuda()
    g = tc.tc_graph_build(a.n, src, dst)
    del src, dst
    out = torch.zeros(17, dtype=torch.int64, device="cuda")
    st = tc.tc_graph_stats(g)
    run = tc.tc_opts_default()
    prof = tc.tc_opts_default(profile=1)
    for _ in range(3):
        tc.tc_census(g, run, out=out, stream=stream)
    ts = time_census(tc, torch, g, run, out, stream, flush, steps)
    census = tc.census_from_device_words(out.cpu().tolist())
    profs = []
    for k in range(3):
        flush.fill_(k)
        tc.tc_census(g, prof, out=out, stream=stream)
        profs.append(tc.tc_census_profile())
    merge = tc.tc_opts_default(tri_path=tc.TC_TRI_MERGE)
    merge_ms = float(np.median(time_census(tc, torch, g, merge, out, stream, flush, 3)))
    tc.tc_graph_free(g)
    top, ms = dominant_kernel(tc, profs, st)
    gpath = os.path.join(ROOT, "tests", "golden", "census_c5.json")
    gold = json.load(open(gpath)) if os.path.exists(gpath) else None
    match = None
    if gold and gold["stats"]["arcs"] == st["arcs"]:
        match = gold["census"] == census
    cms = float(np.median(ts))
    return {"workload": f"c5: {WORKLOAD_DESC['c5']}", "n": a.n, "arcs": st["arcs"], "dyads": st["dyads"],
            "max_degree": st["max_degree"], "merged_entries": st["merged_entries"],
            "census_ms": cms, "census_ms_merge_path": merge_ms,
            "effective_entries_per_s": st["merged_entries"] / (cms / 1e3),
            "kernel_ms": ms,
            "roofline": {"kernel": top["kernel"], "bytes_per_launch": top["bytes"], "ms_per_launch": top["ms"],
                         "achieved": top["bytes"] / (top["ms"] / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": top["bytes"] / (top["ms"] / 1e3) / 1e9 / peak},
            "oracle_census_match": match}


def path_routing(tc, torch, gs, stream, words):
    """Plan-replay time of the batch with every graph on the forward path,
    on the merge path, routed by the degree-skew rule (the default), and
    routed by the learned path model trained on batch-scale costs of a
    separate batch of 160 graphs (same generator, seed 40)."""
    from paper_1603_02655_b300 import costmodel
    import synth
    G = len(gs)

    def replay(over):
        out = torch.zeros(17 * G, dtype=torch.int64, device="cuda")
        plan = tc.tc_plan_create(gs, out, tc.tc_opts_default(**over), stream=stream)
        for _ in range(2):
            tc.tc_plan_run(plan, stream)
        torch.cuda.synchronize()
        ts = []
        for k in range(5):
            a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            tc.tc_plan_run(plan, stream)
            c.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(c))
        tc.tc_plan_free(plan)
        assert out.cpu().tolist() == words, "a route changed the counts"
        return float(np.median(ts))

    rec = {"forward_ms": replay(dict(tri_path=tc.TC_TRI_FORWARD)),
           "merge_ms": replay(dict(tri_path=tc.TC_TRI_MERGE)),
           "skew_rule_ms": replay(dict(tri_path=tc.TC_TRI_AUTO)),
           "skew_rule_merge_graphs": sum(tc.tc_path_route(gs))}
    t0 = time.perf_counter()
    train = synth.batch(160, 64, 65536, 4.0, 32.0, 8, 0.5, seed=40)
    params, rep = costmodel.train_path_model([train.graph(i) for i in range(len(train))], copies=32)
    rec["train_s"] = time.perf_counter() - t0
    rec["train_report"] = rep
    tc.tc_path_model_load(params)
    try:
        rec["learned_ms"] = replay(dict(tri_path=tc.TC_TRI_AUTO))
        rec["learned_merge_graphs"] = sum(tc.tc_path_route(gs))
    finally:
        tc.tc_path_model_load(None)
    rec["learned_vs_skew_rule"] = rec["skew_rule_ms"] / rec["learned_ms"]
    return rec


def c4_record(tc, torch, stream, flush, steps, route=True):
    """The batched workload: 4096 graphs censused by one CUDA-graph plan
    replay (graphs/s), against one tc_census call per graph, and every
    graph's census checked against the oracle's stored per-graph census."""
    import synth
    t0 = time.perf_counter()
    b = synth.c4()
    gen_s = time.perf_counter() - t0
    G = len(b)
    src = torch.from_numpy(b.src).cuda()
    dst = torch.from_numpy(b.dst).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    gs = tc.tc_graph_build_batched(b.ns, b.goff, src, dst)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    del src, dst
    merged = sum(tc.tc_graph_stats(g)["merged_entries"] for g in gs)
    out = torch.zeros(17 * G, dtype=torch.int64, device="cuda")
    opts = tc.tc_opts_default()
    plan = tc.tc_plan_create(gs, out, opts, stream=stream)
    for _ in range(3):
        tc.tc_plan_run(plan, stream)
    torch.cuda.synchronize()
    ts = []
    for k in range(steps):
        flush.fill_(k)
        a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        tc.tc_plan_run(plan, stream)
        c.record(stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(c))
    tc.tc_plan_free(plan)
    words = out.cpu().tolist()
    census = [tc.census_from_device_words(words[17 * i:17 * i + 17]) for i in range(G)]
    # one census call (one launch sequence) per graph
    per_out = torch.zeros(17 * G, dtype=torch.int64, device="cuda")
    flush.fill_(0)
    torch.cuda.synchronize()
    a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for i, g in enumerate(gs):
        tc.tc_census(g, opts, out=per_out[17 * i:17 * i + 17], stream=stream)
    c.record(stream)
    torch.cuda.synchronize()
    per_ms = a.elapsed_time(c)
    same = per_out.cpu().tolist() == words
    routing = path_routing(tc, torch, gs, stream, words) if route else None
    for g in gs:
        tc.tc_graph_free(g)
    gpath = os.path.join(ROOT, "tests", "golden", "census_c4.json")
    match = None
    if os.path.exists(gpath):
        gold = json.load(open(gpath))
        if "census" in gold:
            match = gold["census"] == census
    ms = float(np.median(ts))
    return {"workload": f"c4: {WORKLOAD_DESC['c4']}", "graphs": G, "arcs": int(b.src.size),
            "vertices": int(b.ns.sum()), "merged_entries": merged,
            "ms_per_replay": ms, "graphs_per_s": G / (ms / 1e3),
            "per_graph_calls": {"ms": per_ms, "graphs_per_s": G / (per_ms / 1e3),
                                "same_counts": same},
            "speedup_vs_per_graph": per_ms / ms,
            "step": "census of all 4096 graphs of one batched build (CUDA-graph plan replay of separate kernel launches; the one-persistent-launch form, persistent = 1, is slower and not used; build excluded)",
            "path_routing": routing,
            "build_s": build_s, "generate_s": gen_s, "oracle_census_match_every_graph": match}


def run_native(args, world, rank, local, pg):
    import torch
    import synth
    import paper_1603_02655_b300 as tc
    from paper_1603_02655_b300 import build as tcbuild

    torch.cuda.set_device(local)
    tcbuild.build()
    tc.load()
    arcs = synth.WORKLOADS[args.workload]()
    src_d = torch.from_numpy(arcs.src).cuda()
    dst_d = torch.from_numpy(arcs.dst).cuda()
    src_h = torch.from_numpy(arcs.src).pin_memory()
    dst_h = torch.from_numpy(arcs.dst).pin_memory()
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    out = torch.zeros(17, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    over = dict(kv.split("=") for kv in args.opts.split(",") if kv) if args.opts else {}
    prof_opts = tc.tc_opts_default(profile=1, **{k: int(v) for k, v in over.items()})

    learned = None
    if args.mlp:
        learned, prof_opts = train_and_compare(tc, [tc.tc_graph_build(arcs.n, src_d, dst_d)], prof_opts,
                                               stream, free=True)
    tune = None
    if args.autotune:
        g = tc.tc_graph_build(arcs.n, src_d, dst_d)
        t0 = time.perf_counter()
        default_ms = tc.tc_autotune([g], prof_opts, max_trials=1, stream=stream)[1]
        best, tuned_ms, trials = tc.tc_autotune([g], prof_opts, max_trials=args.autotune, stream=stream)
        tune = {"default_ms": default_ms, "tuned_ms": tuned_ms, "trials": trials,
                "seconds": time.perf_counter() - t0}
        best.profile = 1
        prof_opts = best
        tc.tc_graph_free(g)
    # the timed steps run uninstrumented; the per-kernel breakdown comes from
    # separate profiled steps afterwards (per-kernel events and a counter read)
    run_opts = tc.tc_opts_default(**{k: getattr(prof_opts, k) for k in tc.TUNED_FIELDS})
    for _ in range(args.warmup):  # warm-up steps
        g = tc.tc_graph_build(arcs.n, src_d, dst_d, stream=stream)
        tc.tc_census(g, run_opts, out=out, stream=stream)
        tc.tc_graph_free(g)
    torch.cuda.synchronize()
    g = tc.tc_graph_build(arcs.n, src_d, dst_d)
    stats = tc.tc_graph_stats(g)
    tc.tc_graph_free(g)

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier(pg)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.fill_(k)   # L2 flush between steps (outside the step's events)
            a, b, c = ev[k]
            a.record(stream)
            g = tc.tc_graph_build(arcs.n, src_d, dst_d, stream=stream)
            b.record(stream)
            tc.tc_census(g, run_opts, out=out, stream=stream)
            c.record(stream)
            tc.tc_graph_free(g)
        torch.cuda.synchronize()
    barrier(pg)
    census = tc.census_from_device_words(out.cpu().tolist())
    step_ms = [a.elapsed_time(c) for a, b, c in ev]
    build_ms = [a.elapsed_time(b) for a, b, c in ev]
    census_ms = [b.elapsed_time(c) for a, b, c in ev]
    total_ms = max_over_ranks(sum(step_ms), pg)
    ms_per_step = total_ms / args.steps
    value = world * stats["merged_entries"] * args.steps / (total_ms / 1e3)

    profs = []
    for k in range(max(3, min(args.steps, 5))):
        flush.fill_(k)
        g = tc.tc_graph_build(arcs.n, src_d, dst_d, stream=stream)
        tc.tc_census(g, prof_opts, out=out, stream=stream)
        profs.append(tc.tc_census_profile())
        tc.tc_graph_free(g)
    torch.cuda.synchronize()
    pl = profs[-1]
    top, kernel_ms = dominant_kernel(tc, profs, stats)
    peak, peak_kind = peaks()
    achieved = top["bytes"] / (top["ms"] / 1e3) / 1e9
    ipl, sha = issue_record(top["kernel"])
    clocks = clk.summary()
    lookups = (top.get("units") or {}).get("lookups")
    dram_per_lookup = recorded_traffic_fwd(top["kernel"], sha)
    roofline = {"bound": "hbm", "kernel": top["kernel"], "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_kind": peak_kind,
                "traffic": (dram_per_lookup * lookups) if (dram_per_lookup and lookups) else None,
                "algorithmic_bytes_per_launch": top["bytes"], "units_per_launch": top.get("units"),
                "bytes_per_unit": top.get("bytes_per_unit"), "ms_per_launch": top["ms"]}
    if ipl and lookups:
        # issue roofline: warp instructions the launch executes (ncu count per
        # lookup on this source x lookups) over what 4 schedulers per SM
        # issue at the sampled clock in the launch's time
        import torch as _t
        sms = _t.cuda.get_device_properties(local).multi_processor_count
        mhz = clocks.get("sm_mhz") or 1.0
        inst = ipl * lookups
        roofline["issue"] = {"warp_instructions": inst, "per_lookup": ipl, "sms": sms, "sm_mhz": mhz,
                             "frac": inst / (sms * 4 * mhz * 1e6 * top["ms"] / 1e3)}

    # end to end through the public API from pinned host memory (run options)
    e2e_steps = max(3, min(args.steps, 10))
    host_out = None
    e2e_ms = []
    for k in range(e2e_steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g = tc.tc_graph_build(arcs.n, src_h.numpy(), dst_h.numpy())
        host_out = tc.tc_census(g, run_opts)
        t1 = time.perf_counter()
        tc.tc_graph_free(g)
        if k > 0:
            e2e_ms.append((t1 - t0) * 1e3)
    assert host_out == census, "end-to-end census differs from the device-resident run"
    e2e_total = max_over_ranks(sum(e2e_ms), pg)
    e2e = {"value": world * stats["merged_entries"] * e2e_steps / (e2e_total / 1e3), "unit": UNIT,
           "h2d_bytes_per_step": int(arcs.src.nbytes + arcs.dst.nbytes),
           "d2h_bytes_per_step": 17 * 8, "ms_per_step": e2e_total / e2e_steps}

    gold_ok = None
    gpath = os.path.join(ROOT, "tests", "golden", f"census_{args.workload}.json")
    if os.path.exists(gpath):
        gold = json.load(open(gpath))
        if gold.get("stats", {}).get("arcs") == stats["arcs"]:
            gold_ok = gold["census"] == census

    subs = {}
    if rank == 0 and world == 1 and args.workload == "c3" and not args.no_sub:
        subs["c5"] = c5_record(tc, torch, stream, flush, 10, peak)
        subs["c4"] = c4_record(tc, torch, stream, flush, 10)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, thr, verts, ents, wall, skipped = oracle_sample_rate(arcs, args.cpu_seconds)
        cpu = {"value": rate, "unit": UNIT, "cores": thr, "kind": "oracle",
               "sample": f"oracle census of the canonical dyads with lower endpoint in {verts} of "
                         f"{arcs.n} vertices, random ranges sized by merged entries ({ents:.3e} "
                         f"merged entries, {wall:.1f} s on {thr} host threads; {skipped} ranges "
                         f"too heavy for one thread in that time left out, so the rate is that of "
                         f"the cheaper dyads)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "census_ms": float(np.median(census_ms)), "build_ms": float(np.median(build_ms)),
            "config": {"workload": f"{args.workload}: {WORKLOAD_DESC.get(args.workload, '')}",
                       "n": arcs.n, "arcs": stats["arcs"], "dyads": stats["dyads"],
                       "merged_entries": stats["merged_entries"],
                       "max_degree": stats["max_degree"],
                       "step": "graph build + census, arc list resident in HBM",
                       "value": "effective rate: sum_v d_v^2 (the merged entries a full union merge of every "
                                "canonical dyad would read) per step time; no kernel reads at this rate",
                       "l2": "512 MB buffer written between timed steps (L2 flush)",
                       "parallelism": "single GPU" if world == 1 else f"replicas x{world}",
                       "census_opts": {k: getattr(prof_opts, k) for k in tc.TUNED_FIELDS}},
            "breakdown": {"census_ms_steps": [round(float(x), 3) for x in census_ms],
                          "kernel_ms": kernel_ms,
                          "forward": {k: pl[k] for k in ("fwd_entries", "map_items", "map_dyads", "map_lookups",
                                                         "map_triangles", "search_dyads", "search_lookups",
                                                         "search_triangles", "map_list_entries")},
                          "census_entries_per_s": stats["merged_entries"] / (np.median(census_ms) / 1e3)},
            "oracle_census_match": gold_ok,
            "roofline": roofline,
            "autotune": tune,
            "learned_binning": learned,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clocks,
            "gpu_launches": args.steps * (OWN_BUILD_KERNELS + pl["launches"]),
            "census": [str(x) for x in census],
        }
        line.update(subs)
        print(json.dumps(line), flush=True)


def run_batched(args, world, rank, local, pg):
    """Workload c4 alone: the batched plan replay timed over --steps, with
    the per-graph comparison and the oracle check of every graph."""
    import torch
    import paper_1603_02655_b300 as tc
    from paper_1603_02655_b300 import build as tcbuild

    torch.cuda.set_device(local)
    tcbuild.build()
    tc.load()
    stream = torch.cuda.current_stream()
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    barrier(pg)
    with ClockSampler(local) as clk:
        rec = c4_record(tc, torch, stream, flush, args.steps)
    barrier(pg)
    ms = max_over_ranks(rec["ms_per_replay"], pg)
    if rank == 0:
        line = {"metric": METRIC, "value": world * rec["graphs"] / (ms / 1e3), "unit": "graphs/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
                "data": "synthetic",
                "config": {"workload": rec["workload"], "graphs": rec["graphs"], "step": rec["step"],
                           "l2": "512 MB buffer written between timed steps (L2 flush)"},
                "c4": rec, "clocks": clk.summary()}
        print(json.dumps(line), flush=True)


def train_and_compare(tc, gs, opts, stream, free):
    """Binning on the merge path (the only path with bins): train the
    task-cost model on timings recorded on these graphs, install it, and time
    the census (best of 5 after 2 warm-ups) with degree-sum binning, with
    exact-|S| binning (its |S| pass timed apart: the census time without it
    is the ceiling of a one-number cost rule) and with learned binning, each
    with owner lookups for hub dyads (own_min as given) and with merges only
    (own_min = 0).  Returns (report, opts with learned binning)."""
    import torch
    from paper_1603_02655_b300 import costmodel
    t0 = time.perf_counter()
    params, rep = costmodel.train_cost_model(gs, mask=63, steps=3000, stream=stream)
    train_s = time.perf_counter() - t0
    costmodel.install(params)

    def best_ms(o):
        out = torch.zeros(17 * len(gs), dtype=torch.int64, device="cuda")
        ts = []
        for k in range(7):
            a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            tc.tc_census_batched(gs, o, out=out, stream=stream)
            c.record(stream)
            torch.cuda.synchronize()
            if k >= 2:
                ts.append(a.elapsed_time(c))
        return float(np.min(ts)), out.cpu().tolist()

    def with_mode(mode, own_min):
        o = tc.tc_opts_default(**{k: getattr(opts, k) for k in tc.TUNED_FIELDS})
        o.bin_mode, o.tri_path, o.own_min = mode, tc.TC_TRI_MERGE, own_min
        return o

    report = {"path": "merge (tri_path = TC_TRI_MERGE): the bins exist only there",
              "rmse_log2_cycles_mlp": rep["rmse_mlp"], "rmse_log2_cycles_degree_sum": rep["rmse_degree_sum"],
              "rmse_log2_cycles_exact_size": rep.get("rmse_exact_size"),
              "samples": rep["samples"], "train_s": train_s}
    ref = None
    for label, own_min in (("owner_lookups", opts.own_min if opts.own_min > 0 else 128), ("merges_only", 0)):
        rec = {"own_min": own_min}
        for name, mode in (("degree_sum", tc.TC_BIN_HEURISTIC), ("exact_size", tc.TC_BIN_EXACT),
                           ("learned", tc.TC_BIN_MLP)):
            o = with_mode(mode, own_min)
            ms, out = best_ms(o)
            if ref is None:
                ref = out
            assert out == ref, f"{name} binning changed the counts"
            o.profile = 1
            tc.tc_census_batched(gs, o, stream=stream)
            p = tc.tc_census_profile()
            rec[name] = {"census_ms": ms, "bin_tasks": p["bin_tasks"]}
            if mode == tc.TC_BIN_EXACT:
                rec[name]["exact_pass_ms"] = p["ms_exact_cost"]
                rec[name]["census_ms_without_pass"] = ms - p["ms_exact_cost"]
        rec["speedup_learned"] = rec["degree_sum"]["census_ms"] / rec["learned"]["census_ms"]
        rec["speedup_exact_ceiling"] = rec["degree_sum"]["census_ms"] / rec["exact_size"]["census_ms_without_pass"]
        report[label] = rec
    learn = with_mode(tc.TC_BIN_MLP, opts.own_min)
    learn.tri_path = opts.tri_path
    learn.profile = opts.profile
    if free:
        for g in gs:
            tc.tc_graph_free(g)
    return report, learn


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="c3", choices=sorted(WORKLOAD_DESC))
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sub", action="store_true", help="skip the c5 and c4 sub-records of the default run")
    ap.add_argument("--opts", default="", help="census options, e.g. thr_warp=512,stream_max=1024")
    ap.add_argument("--mlp", action="store_true",
                    help="train the learned cost model on the workload and bin with it")
    ap.add_argument("--autotune", type=int, default=0, metavar="TRIALS",
                    help="autotune the census options first (at most TRIALS timed options)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world, rank, local, pg = dist_setup(args)
    try:
        if args.impl == "reference":
            run_reference(args, world, rank, pg)
        elif args.workload == "c4":
            run_batched(args, world, rank, local, pg)
        else:
            run_native(args, world, rank, local, pg)
    finally:
        if pg is not None:
            pg.destroy_process_group()


if __name__ == "__main__":
    main()
