#!/usr/bin/env python
"""Benchmark of the triad-census hot path on B300 (one JSON line on stdout).

A step is one pass of the whole hot path over the workload's arc list, which
is already resident in HBM: device graph build (dedup, tagged adjacency) and
the census (task build + binning, union merges, classification, fold and
003 closure).  `value` is merged adjacency entries per second of step time
(entries = sum over canonical dyads of |N(u)|+|N(v)|, the data the merges must
read); `census_ms` in the breakdown is the census alone.

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
UNIT = "merged adjacency entries/s"
WORKLOAD_DESC = {
    "c1": "G(n,p) n=1024 p=8/1023 reciprocity 0.25 seed 1",
    "c2": "R-MAT scale 20 edge factor 8 (.57,.19,.19,.05) 10% reciprocated, ids permuted, seed 2",
    "c3": "R-MAT scale 22 edge factor 4 (.57,.19,.19,.05), arcs oriented high->low id, ids permuted, seed 3",
    "c3s": "R-MAT scale 21 edge factor 4, arcs oriented high->low id, ids permuted, seed 3 (profiling case)",
    "c4": "4096 graphs, n log-uniform in [64, 65536], even G(n,p) mean out-degree U(4,32), odd R-MAT edge factor 8, reciprocity U(0,0.5), seed 4",
    "c5": "Chung-Lu n=2^22 gamma 2.1 mean total degree 16 max 1e5 reciprocity 0.15, seed 5",
}
OWN_BUILD_KERNELS = 8   # k_dyad_keys k_heads k_dyads k_row_counts k_place_lo k_place_up k_fill_sent k_rowstats (plus CUB sort/scan)
FLUSH_BYTES = 512 << 20  # > 126 MB L2


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def recorded_traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it
    was taken on the current kernel source (else None)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    src = os.path.join(ROOT, "paper_1603_02655_b300", "csrc", "census.cu")
    try:
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        for line in open(path):
            parts = line.split()
            if len(parts) >= 3 and parts[0] == kernel and parts[2] == sha:
                return int(parts[1])
    except OSError:
        pass
    return None


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
                 "--format=csv,noheader,nounits", "-lms", "200"],
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

    def step_device():
        g = tc.tc_graph_build(arcs.n, src_d, dst_d, stream=stream)
        tc.tc_census(g, prof_opts, out=out, stream=stream)
        return g

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
    # warm-up
    for _ in range(args.warmup):
        g = step_device()
        tc.tc_graph_free(g)
    torch.cuda.synchronize()
    g = tc.tc_graph_build(arcs.n, src_d, dst_d)
    stats = tc.tc_graph_stats(g)
    tc.tc_census(g, prof_opts, out=out)
    torch.cuda.synchronize()
    census = tc.census_from_device_words(out.cpu().tolist())
    tc.tc_graph_free(g)

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    # the timed steps run uninstrumented; the per-kernel breakdown comes from
    # separate profiled steps afterwards (per-kernel events and a counter read)
    run_opts = tc.tc_opts_default(**{k: getattr(prof_opts, k) for k in tc.TUNED_FIELDS})
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
    profs = []
    for k in range(max(3, min(args.steps, 5))):
        flush.fill_(k)
        g = tc.tc_graph_build(arcs.n, src_d, dst_d, stream=stream)
        tc.tc_census(g, prof_opts, out=out, stream=stream)
        profs.append(tc.tc_census_profile())
        tc.tc_graph_free(g)
    torch.cuda.synchronize()
    step_ms = [a.elapsed_time(c) for a, b, c in ev]
    build_ms = [a.elapsed_time(b) for a, b, c in ev]
    census_ms = [b.elapsed_time(c) for a, b, c in ev]
    total_ms = max_over_ranks(sum(step_ms), pg)
    ms_per_step = total_ms / args.steps
    value = world * stats["merged_entries"] * args.steps / (total_ms / 1e3)

    # dominant kernel and its roofline (algorithmic bytes = 4 B per merged entry)
    # merged entries per merge kernel: the bins it runs, hub tasks (streamed
    # by k_hub, counted in bin 2) moved out of the kernel that would cut them
    pl = profs[-1]
    hub = pl["hub_entries"]
    # k_owner reads, per owner dyad, the other endpoint's list (one lookup per
    # entry) and, per work item, the owner's list: those are its bytes
    own_bytes_entries = pl["owner_probes"] + pl["owner_staged"]
    if prof_opts.persistent:
        kern = {"k_tasks": "ms_tasks", "k_split": "ms_split", "k_owner": "ms_owner", "k_hub": "ms_stream",
                "k_fold": "ms_fold"}
        avg = {k: float(np.mean([p[f] for p in profs])) for k, f in kern.items()}
        avg["k_merge"] = float(np.mean([p["ms_merge"] - p["ms_stream"] for p in profs]))
        merge_entries = {"k_merge": sum(pl["bin_entries"]) - hub, "k_hub": hub, "k_owner": own_bytes_entries}
    else:
        kern = {"k_tasks": "ms_tasks", "k_split": "ms_split", "k_owner": "ms_owner", "k_warp[tiles]": "ms_tiles",
                "k_stream+k_hub": "ms_stream", "k_warp": "ms_warp", "k_thread": "ms_thread", "k_fold": "ms_fold"}
        avg = {k: float(np.mean([p[f] for p in profs])) for k, f in kern.items()}
        be = pl["bin_entries"]
        merge_entries = {"k_warp[tiles]": be[2] - hub, "k_stream+k_hub": be[3] + hub, "k_warp": be[1],
                         "k_thread": be[0], "k_owner": own_bytes_entries}
    top = max(merge_entries, key=lambda k: avg[k])
    entries_top = merge_entries[top]
    peak, peak_kind = peaks()
    achieved = 4.0 * entries_top / (avg[top] / 1e3) / 1e9
    traffic = recorded_traffic(top)
    roofline = {"bound": "hbm", "kernel": top, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                "algorithmic_bytes_per_launch": 4 * entries_top,
                "bytes_per_unit": ("4 B per lookup plus 4 B per owner-list entry indexed" if top == "k_owner"
                                   else "4 B per merged adjacency entry"),
                "ms_per_launch": avg[top],
                # the full-union merge work over the whole census (the paper's
                # cost), as if every dyad were merged: an effective rate
                "effective_frac": 4.0 * stats["merged_entries"] / (np.mean(census_ms) / 1e3) / 1e9 / peak}
    merge_ms = sum(avg[k] for k in merge_entries)

    # end to end through the public API from pinned host memory
    e2e_steps = max(3, min(args.steps, 5))
    host_out = None
    e2e_ms = []
    for k in range(e2e_steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g = tc.tc_graph_build(arcs.n, src_h.numpy(), dst_h.numpy())
        host_out = tc.tc_census(g, prof_opts)
        t1 = time.perf_counter()
        tc.tc_graph_free(g)
        if k > 0:
            e2e_ms.append((t1 - t0) * 1e3)
    assert host_out == census, "end-to-end census differs from the device-resident run"
    e2e_total = max_over_ranks(sum(e2e_ms), pg)
    e2e = {"value": world * stats["merged_entries"] * e2e_steps / (e2e_total / 1e3), "unit": UNIT,
           "h2d_bytes_per_step": int(arcs.src.nbytes + arcs.dst.nbytes),
           "d2h_bytes_per_step": 17 * 8, "ms_per_step": e2e_total / e2e_steps}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, thr, verts, ents, wall, skipped = oracle_sample_rate(arcs, args.cpu_seconds)
        cpu = {"value": rate, "unit": UNIT, "cores": thr, "kind": "oracle",
               "sample": f"oracle census of the canonical dyads with lower endpoint in {verts} of "
                         f"{arcs.n} vertices, random ranges sized by merged entries ({ents:.3e} "
                         f"merged entries, {wall:.1f} s on {thr} host threads; {skipped} ranges "
                         f"too heavy for one thread in that time left out)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {WORKLOAD_DESC.get(args.workload, '')}",
                       "n": arcs.n, "arcs": stats["arcs"], "dyads": stats["dyads"],
                       "merged_entries": stats["merged_entries"],
                       "max_degree": stats["max_degree"],
                       "step": "graph build + census, arc list resident in HBM",
                       "l2": "512 MB buffer written between timed steps (L2 flush)",
                       "parallelism": "single GPU" if world == 1 else f"replicas x{world}",
                       "census_opts": {k: getattr(prof_opts, k) for k in tc.TUNED_FIELDS}},
            "breakdown": {"census_ms": float(np.mean(census_ms)), "build_ms": float(np.mean(build_ms)),
                          "census_ms_steps": [round(float(x), 3) for x in census_ms],
                          "merge_ms": merge_ms, "kernel_ms": avg,
                          "bin_tasks": profs[-1]["bin_tasks"], "bin_entries": profs[-1]["bin_entries"],
                          "hub_tasks": profs[-1]["hub_tasks"], "hub_entries": hub,
                          "owner": {k: pl[k] for k in ("owner_items", "owner_tasks", "owner_entries",
                                                       "owner_probes", "owner_staged")},
                          "chunks": profs[-1]["chunks"],
                          "census_entries_per_s": stats["merged_entries"] / (np.mean(census_ms) / 1e3)},
            "roofline": roofline,
            "autotune": tune,
            "learned_binning": learned,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clk.summary(),
            "gpu_launches": args.steps * (OWN_BUILD_KERNELS + profs[-1]["launches"]),
            "census": [str(x) for x in census],
        }
        print(json.dumps(line), flush=True)


def run_batched(args, world, rank, local, pg):
    """Workload c4: every graph censused in one batch (a CUDA-graph plan over
    one batched build), against one census call per graph."""
    import torch
    import synth
    import paper_1603_02655_b300 as tc
    from paper_1603_02655_b300 import build as tcbuild

    torch.cuda.set_device(local)
    tcbuild.build()
    tc.load()
    t0 = time.perf_counter()
    b = synth.c4()
    gen_s = time.perf_counter() - t0
    G = len(b)
    over = dict(kv.split("=") for kv in args.opts.split(",") if kv) if args.opts else {}
    opts = tc.tc_opts_default(**{k: int(v) for k, v in over.items()})
    src_d = torch.from_numpy(b.src).cuda()
    dst_d = torch.from_numpy(b.dst).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    gs = tc.tc_graph_build_batched(b.ns, b.goff, src_d, dst_d)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    del src_d, dst_d
    stats = [tc.tc_graph_stats(g) for g in gs]
    merged = sum(st["merged_entries"] for st in stats)
    out = torch.zeros(17 * G, dtype=torch.int64, device="cuda")
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    learned = None
    if args.mlp:
        learned, opts = train_and_compare(tc, gs, opts, stream, free=False)
    tune = None
    if args.autotune:
        t0 = time.perf_counter()
        default_ms = tc.tc_autotune(gs, opts, max_trials=1, stream=stream)[1]
        opts, tuned_ms, trials = tc.tc_autotune(gs, opts, max_trials=args.autotune, stream=stream)
        tune = {"default_ms": default_ms, "tuned_ms": tuned_ms, "trials": trials,
                "seconds": time.perf_counter() - t0}
    plan = tc.tc_plan_create(gs, out, opts, stream=stream)
    for _ in range(args.warmup):
        tc.tc_plan_run(plan, stream)
    torch.cuda.synchronize()
    words = out.cpu().tolist()
    census = [tc.census_from_device_words(words[17 * i:17 * i + 17]) for i in range(G)]
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    barrier(pg)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.fill_(k)
            ev[k][0].record(stream)
            tc.tc_plan_run(plan, stream)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
    barrier(pg)
    total_ms = max_over_ranks(sum(a.elapsed_time(c) for a, c in ev), pg)
    ms = total_ms / args.steps
    tc.tc_plan_free(plan)
    # one census call (one launch sequence) per graph, plain degree-sum binning
    heur = tc.tc_opts_default(persistent=0)
    per_out = torch.zeros(17 * G, dtype=torch.int64, device="cuda")
    per_ms = []
    for rep_ in range(2):
        flush.fill_(rep_)
        torch.cuda.synchronize()
        a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for i, g in enumerate(gs):
            tc.tc_census(g, heur, out=per_out[17 * i:17 * i + 17], stream=stream)
        c.record(stream)
        torch.cuda.synchronize()
        per_ms.append(a.elapsed_time(c))
    per_words = per_out.cpu().tolist()
    assert per_words == words, "per-graph census differs from the batched census"
    # checksum against the stored oracle values when present
    gold_ok = None
    gpath = os.path.join(ROOT, "tests", "golden", "census_c4.json")
    if os.path.exists(gpath):
        gold = json.load(open(gpath))
        tot = [sum(c[t] for c in census) for t in range(16)]
        wsum = [sum((i + 1) * c[t] for i, c in enumerate(census)) for t in range(16)]
        gold_ok = tot == gold["total"] and wsum == gold["weighted"]
    for g in gs:
        tc.tc_graph_free(g)
    if rank == 0:
        line = {
            "metric": METRIC, "value": world * G / (ms / 1e3), "unit": "graphs/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": f"c4: {WORKLOAD_DESC['c4']}", "graphs": G, "arcs": int(b.src.size),
                       "vertices": int(b.ns.sum()), "merged_entries": merged,
                       "step": "batched census of all graphs (CUDA-graph plan replay), graphs built",
                       "l2": "512 MB buffer written between timed steps (L2 flush)",
                       "census_opts": {k: getattr(opts, k) for k in
                                       ("bin_mode", "thr_thread", "thr_warp", "chunk", "stream_max",
                                        "persistent")}},
            "merged_entries_per_s": merged / (ms / 1e3),
            "per_graph_launches": {"ms": float(np.min(per_ms)), "graphs_per_s": G / (np.min(per_ms) / 1e3),
                                   "opts": "degree-sum binning, one tc_census per graph"},
            "speedup_vs_per_graph": float(np.min(per_ms)) / ms,
            "build_s": build_s, "generate_s": gen_s, "golden_checksums_match": gold_ok,
            "autotune": tune,
            "learned_binning": learned,
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)


def train_and_compare(tc, gs, opts, stream, free):
    """Train the task-cost model on timings recorded on these graphs, install
    it, and time the census with degree-sum binning and with learned binning
    (best of 5 after 2 warm-ups each).  Returns (report, opts with learned
    binning)."""
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

    heur = tc.tc_opts_default(**{k: getattr(opts, k) for k in tc.TUNED_FIELDS})
    heur.bin_mode = tc.TC_BIN_HEURISTIC
    learn = tc.tc_opts_default(**{k: getattr(opts, k) for k in tc.TUNED_FIELDS})
    learn.bin_mode = tc.TC_BIN_MLP
    h_ms, h_out = best_ms(heur)
    l_ms, l_out = best_ms(learn)
    bins_used = {}
    for name, o in (("degree_sum", heur), ("learned", learn)):
        o.profile = 1
        tc.tc_census_batched(gs, o, stream=stream)
        bins_used[name] = tc.tc_census_profile()["bin_tasks"]
        o.profile = 0
    assert h_out == l_out, "learned binning changed the counts"
    learn.profile = opts.profile
    report = {"census_ms_degree_sum": h_ms, "census_ms_learned": l_ms, "speedup": h_ms / l_ms,
              "rmse_log2_cycles_mlp": rep["rmse_mlp"], "rmse_log2_cycles_degree_sum": rep["rmse_degree_sum"],
              "rmse_log2_cycles_exact_size": rep.get("rmse_exact_size"),
              "samples": rep["samples"], "train_s": train_s,
              "bin_tasks": bins_used}
    if free:
        for g in gs:
            tc.tc_graph_free(g)
    return report, learn


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="c3", choices=sorted(WORKLOAD_DESC))
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
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
