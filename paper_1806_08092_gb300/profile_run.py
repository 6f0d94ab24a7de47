"""Runs GPOP algorithms once each on the seeded RMAT graph that bench.py measures (edge factor 16, weights
in [1, 255], partition size 16384, Eq. (mode)'s BW_PC/BW_SC = 8/1 for BFS and SSSP) and prints each run's
statistics as one JSON line.  Kernel counters taken over this process (for example DRAM bytes of every
k_scatter_sc launch) can then be divided by the run's own counts: active SC vertices and edges, destinations
gathered, iterations.

    python paper_1806_08092_gb300/profile_run.py --scale 24 --algos bfs,sssp
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--scale", type=int, default=24)
    ap.add_argument("--partition", type=int, default=16384)
    ap.add_argument("--algos", default="bfs,sssp")
    ap.add_argument("--root-index", type=int, default=0, help="which of the generator's 16 roots")
    ap.add_argument("--bw-ratio", type=int, default=8)
    a = ap.parse_args()

    import graphgen as gg
    import paper_1806_08092_gb300 as gp

    g = gg.rmat(a.scale).with_weights(hi=255)
    root = int(gg.roots(g, 16)[a.root_index])
    G = gp.Graph.from_csr(g.row_ptr, g.col, g.weights, partition_size=a.partition)
    print(json.dumps({"layout": G.info()}), flush=True)
    keys = ("iterations", "device_ms", "edges_scattered", "vertices_scattered", "sc_vertices_scattered",
            "sc_edges_scattered", "gathered_vertices", "model_bytes", "pc_partition_steps", "sc_partition_steps")
    for algo in a.algos.split(","):
        if algo in ("pagerank", "pr"):  # to an L1 change below 1e-9, as bench.py runs it
            r = G.run("pagerank", max_iters=300, tol=1e-9)
        else:
            r = G.run(algo, source=root, bw_ratio=(a.bw_ratio, 1))
        out = {"algo": algo, "scale": a.scale, "root": root}
        out.update({k: r.stats[k] for k in keys if k in r.stats})
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
