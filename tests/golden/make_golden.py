"""Write the stored expected censuses under tests/golden/ .

Every value here comes from the CPU oracle (``oracle/``) run on the seeded
workloads of ``synth/``; nothing comes from the CUDA library.  Usage:

    python tests/golden/make_golden.py c1 c2 c3 c4 c5 [--threads T]

The large workloads take from minutes (c2) to hours (c5) of host time.
For the batched workload c4 the file holds the census of every graph
(``census``: one list of 16 counts per graph, in graph order) and, per type,
the sum over graphs and the weighted sum  sum_g (g+1) * count_g[t]  as extra
checks, plus the statistics of a sample of graphs.
"""
import argparse
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

C4_SAMPLE = list(range(0, 4096, 64)) + [1, 3, 5, 4093, 4095]


def one(arcs, threads):
    g = oracle.Graph(arcs.n, arcs.src, arcs.dst)
    st = g.stats()
    t0 = time.time()
    c = g.census(threads)
    dt = time.time() - t0
    g.close()
    return c, st, dt


def write(name, payload):
    path = os.path.join(HERE, f"census_{name}.json")
    every = payload.pop("census") if name == "c4" else None
    with open(path, "w") as f:
        if every is None:
            json.dump(payload, f, indent=1)
        else:  # one line per graph keeps the 4096 censuses readable and small
            text = json.dumps(payload, indent=1)
            rows = ",\n".join("  " + json.dumps(c) for c in every)
            f.write(text[:-2] + ',\n "census": [\n' + rows + "\n ]\n}\n")
    print("wrote", path, flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("workloads", nargs="+")
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    args = ap.parse_args()
    for name in args.workloads:
        gen = synth.WORKLOADS[name]
        if name != "c4":
            arcs = gen()
            c, st, dt = one(arcs, args.threads)
            write(name, {"workload": name, "types": list(oracle.TYPE_NAMES), "census": c,
                         "stats": st, "m_input": arcs.m,
                         "oracle_seconds": round(dt, 1), "oracle_threads": args.threads})
        else:
            b = gen()
            G = len(b)
            total = [0] * 16
            weighted = [0] * 16
            sample = {}
            every = []
            merged = 0
            t0 = time.time()
            for g in range(G):
                a = b.graph(g)
                c, st, _ = one(a, args.threads if a.n > 4096 else 1)
                merged += st["merged_entries"]
                for t in range(16):
                    total[t] += c[t]
                    weighted[t] += (g + 1) * c[t]
                every.append(c)
                if g in C4_SAMPLE:
                    sample[str(g)] = {"census": c, "stats": st}
                if g % 256 == 0:
                    print(f"c4 graph {g}/{G} {time.time() - t0:.0f}s", flush=True)
            write(name, {"workload": name, "graphs": G, "types": list(oracle.TYPE_NAMES),
                         "census": every, "total": total, "weighted": weighted, "sample": sample,
                         "merged_entries": merged, "m_input": int(b.src.size),
                         "oracle_seconds": round(time.time() - t0, 1),
                         "oracle_threads": args.threads})


if __name__ == "__main__":
    main()
