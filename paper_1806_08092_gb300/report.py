"""Measurements of the synthetic configurations on one GPU, one JSON line per result.

    python -m paper_1806_08092_gb300.report [--configs c1,c2,c3,c4,c4_graphs,nibble,ablation,isg,degree]

c1        PageRank, 10 iterations, d = 0.85, RMAT-16 (P = 1024): time and GTEPS = 10 E / t.  The graph
          and its bins fit in L2, so no HBM fraction is meaningful for it.
c2        RMAT-22: BFS and SSSP (weights in [1, 255]) from 16 roots, TEPS = traversed edges / t (the
          out-degrees of the reached vertices, Graph500 style), harmonic mean over the roots; CC on the
          symmetrised graph, E_sym / t.  The partition size is swept over {2K, 4K, 8K, 16K} and every
          setting is reported, the fastest marked.
c3        PageRank to an L1 residual below 1e-9 on RMAT-24 and on a uniform random directed graph of the
          same size and average degree, with FP32 and with BF16 bin messages: GTEPS = E x iterations / t
          and per-kernel times (the errors against the FP64 oracle come from the GPU tests).
c4        RMAT-22 BFS from 64 sources: gpop_run_msbfs (two 32-source passes) against 64 single-source
          gpop_run calls, TEPS = sum over sources of traversed edges / t, and the batching speedup; PPR
          from 256 seeds (alpha = 0.15, L1 change < 1e-9 or 100 iterations), one gpop_run per seed; and
          the same 256 seeds through gpop_run_ppr_batch (32 seeds per message, P = 1024), with the
          largest relative difference of three of its rows from the single-seed runs of the same seeds
          (the error against the FP64 oracle is checked by the GPU tests).
c4_graphs 128 independent RMAT graphs (scales 10-18, edge factors 8-32): BFS on their disjoint union
          (gpop_graph_build_union + gpop_run_bfs_union) against one gpop_run per graph.
nibble    parallel Nibble (Alg. 4) on RMAT-24 from 16 seeds with Sec. 5's threshold eps = 1e-9, at most
          100 iterations: time, iterations, vertices with PR > 0 and edges scattered per seed.
degree    time against average degree (Sec. 5, execution time vs degree): RMAT-26 (64 M vertices) from
          edge factor 1 to 32 (the paper goes to 128; 32 keeps the largest layout near 70 GB), PageRank
          10 iterations, BFS, SSSP and Nibble (eps = 1e-9, at most 100 iterations) from one root, and CC
          on the symmetrised graph up to edge factor 16; with the PC / SC partition-steps of each run.
ablation  RMAT-24 BFS and SSSP and symmetrised RMAT-24 CC with every partition forced to SC, forced to
          PC, and with Eq. (mode): time, iterations and the number of PC / SC partition-steps.
isg       interleaved scatter-gather (Sec. 3.3) with 0 (bulk-synchronous), 2, 4 and 8 waves: SSSP on
          RMAT-24 from 4 roots and CC on symmetrised RMAT-24, Eq. (mode) at BW_PC/BW_SC = 8/1.

Times are CUDA-event device times of gpop_run (inputs resident on the GPU), median of three runs after
a warm-up run unless stated.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np
import torch

from . import Graph

KERNELS = ["k_plan", "k_scatter_pc", "k_scatter_sc", "k_gather", "k_gather_pc", "k_merge_pc"]


def _gen():
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import graphgen
    return graphgen


def _emit(d):
    print(json.dumps(d), flush=True)


def _median_run(G, algo, reps=3, **kw):
    G.run(algo, **kw)  # warm-up
    runs = [G.run(algo, profile=True, **kw) for _ in range(reps)]
    runs.sort(key=lambda r: r.stats["device_ms"])
    return runs[len(runs) // 2]


def _traversed(g, values):
    """Out-degree sum of the vertices a BFS reached (Graph500 traversed edges)."""
    deg = torch.from_numpy(np.diff(g.row_ptr).astype(np.int64)).cuda()
    return int(deg[values.to(torch.int64) != 0xFFFFFFFF].sum().item())


def _kernels(stats):
    return {k: round(v, 3) for k, v in zip(KERNELS, stats["kernel_ms"])}


def c1():
    gg = _gen()
    g = gg.rmat(16)
    G = Graph.from_csr(g.row_ptr, g.col, None, partition_size=1024)
    r = _median_run(G, "pagerank", max_iters=10, tol=0.0)
    ms = r.stats["device_ms"]
    _emit({"config": "c1", "graph": "rmat16", "vertices": g.num_vertices, "edges": g.num_edges,
           "partition_size": 1024, "algo": "pagerank", "iterations": r.stats["iterations"], "ms": ms,
           "gteps": g.num_edges * r.stats["iterations"] / (ms / 1e3) / 1e9, "kernels_ms": _kernels(r.stats),
           "note": "graph and bins are L2-resident"})
    G.close()


def c2(sizes=(2048, 4096, 8192, 16384), nroots=16):
    gg = _gen()
    g = gg.rmat(22).with_weights()
    gs = gg.symmetrized(gg.rmat(22))
    roots = [int(x) for x in gg.roots(g, nroots)]
    results = []
    for P in sizes:
        G = Graph.from_csr(g.row_ptr, g.col, g.weights, partition_size=P)
        out = {"config": "c2", "graph": "rmat22", "vertices": g.num_vertices, "edges": g.num_edges,
               "partition_size": P}
        total = 0.0
        for algo in ("bfs", "sssp"):
            teps, ms_all = [], 0.0
            for r in roots:
                res = _median_run(G, algo, reps=1, source=r)
                te = _traversed(g, G.run("bfs", source=r).values) if algo == "sssp" else _traversed(g, res.values)
                teps.append(te / (res.stats["device_ms"] / 1e3))
                ms_all += res.stats["device_ms"]
            out[algo] = {"gteps_harmonic_mean": len(teps) / sum(1.0 / t for t in teps) / 1e9,
                         "ms_mean": ms_all / len(roots), "roots": len(roots)}
            total += ms_all
        G.close()
        Gs = Graph.from_csr(gs.row_ptr, gs.col, None, partition_size=P)
        rc = _median_run(Gs, "cc")
        out["cc"] = {"edges_sym": gs.num_edges, "ms": rc.stats["device_ms"], "iterations": rc.stats["iterations"],
                     "gteps": gs.num_edges / (rc.stats["device_ms"] / 1e3) / 1e9}
        total += rc.stats["device_ms"]
        Gs.close()
        out["total_ms"] = total
        results.append(out)
    best = min(results, key=lambda o: o["total_ms"])
    for o in results:
        o["fastest"] = o is best
        _emit(o)


def c3():
    gg = _gen()
    n = 1 << 24
    for name, g in (("rmat24", gg.rmat(24)), ("uniform24", gg.uniform(n, 16 * n))):
        G = Graph.from_csr(g.row_ptr, g.col, None, partition_size=16384)
        info = G.info()
        for bf16 in (False, True):
            r = _median_run(G, "pagerank", max_iters=300, tol=1e-9, msg_bf16=bf16)
            ms, it = r.stats["device_ms"], r.stats["iterations"]
            _emit({"config": "c3", "graph": name, "vertices": g.num_vertices, "edges": g.num_edges,
                   "partition_size": 16384, "r": info["num_png"] / g.num_edges, "algo": "pagerank",
                   "messages": "bf16" if bf16 else "fp32", "iterations": it, "residual": r.stats["residual"],
                   "converged": r.stats["converged"], "ms": ms, "gteps": g.num_edges * it / (ms / 1e3) / 1e9,
                   "kernels_ms": _kernels(r.stats)})
        G.close()
        del g


def c4(nsrc=64):
    gg = _gen()
    g = gg.rmat(22)
    src = [int(x) for x in gg.roots(g, nsrc)]
    G = Graph.from_csr(g.row_ptr, g.col, None, partition_size=16384)
    deg = torch.from_numpy(np.diff(g.row_ptr).astype(np.int64)).cuda()
    G.run_msbfs(src)  # warm-up
    runs = sorted((G.run_msbfs(src, profile=True) for _ in range(3)), key=lambda r: r.stats["device_ms"])
    r = runs[1]
    lv = r.values
    te = sum(int(deg[lv[j] != 0xFFFFFFFF].sum().item()) for j in range(nsrc))
    ms_b = r.stats["device_ms"]
    single = 0.0
    for s in src:
        single += _median_run(G, "bfs", reps=1, source=s).stats["device_ms"]
    _emit({"config": "c4", "graph": "rmat22", "vertices": g.num_vertices, "edges": g.num_edges,
           "partition_size": 16384, "algo": "msbfs", "sources": nsrc, "passes": (nsrc + 31) // 32,
           "iterations": r.stats["iterations"], "ms": ms_b, "traversed_edges": te,
           "gteps": te / (ms_b / 1e3) / 1e9, "single_source_ms_total": single,
           "single_source_gteps": te / (single / 1e3) / 1e9, "batching_speedup": single / ms_b,
           "pc_partition_steps": r.stats["pc_partition_steps"], "sc_partition_steps": r.stats["sc_partition_steps"],
           "kernels_ms": _kernels(r.stats)})
    seeds = [int(x) for x in gg.roots(g, 256)]
    G.run("ppr", source=seeds[0], max_iters=100, tol=1e-9)  # warm-up
    ms = its = edges = conv = 0
    rows = (0, 100, 255)
    single_rows = {}
    for j, s in enumerate(seeds):
        r = G.run("ppr", source=s, max_iters=100, tol=1e-9)
        ms += r.stats["device_ms"]
        its += r.stats["iterations"]
        edges += r.stats["edges_scattered"]
        conv += int(r.stats["converged"])
        if j in rows:
            single_rows[j] = r.values.cpu().numpy().astype(np.float64)
    _emit({"config": "c4", "graph": "rmat22", "algo": "ppr", "seeds": len(seeds), "alpha": 0.15, "tol_l1": 1e-9,
           "ms_total": ms, "ms_per_seed": ms / len(seeds), "iterations_mean": its / len(seeds), "converged": conv,
           "gteps_scattered": edges / (ms / 1e3) / 1e9})
    G.close()
    # the same 256 seeds batched (gpop_run_ppr_batch: 32 seeds per message, partition size 1024), against
    # the single-seed runs above: time, and the largest relative difference of three rows where the
    # single-seed value is at least 1e-9 (both runs stop at an L1 change below 1e-9)
    Gb = Graph.from_csr(g.row_ptr, g.col, None, partition_size=1024)
    Gb.run_ppr_batch(seeds[:32], max_iters=5)  # warm-up
    rb = Gb.run_ppr_batch(seeds, max_iters=300, tol=1e-9)
    vals = rb.values.cpu().numpy()
    it_pass = rb.stats["iterations"] // ((len(seeds) + 31) // 32)
    diffs = []
    for j in rows:
        ref, x = single_rows[j], vals[j].astype(np.float64)
        big = ref >= 1e-9
        diffs.append(float(np.max(np.abs(x[big] - ref[big]) / ref[big])))
    _emit({"config": "c4", "graph": "rmat22", "algo": "ppr_batch", "seeds": len(seeds), "seeds_per_pass": 32,
           "partition_size": 1024, "alpha": 0.15, "tol_l1": 1e-9, "ms_total": rb.stats["device_ms"],
           "single_seed_ms_total": ms, "speedup_vs_single_seed_runs": ms / rb.stats["device_ms"],
           "iterations_per_pass": it_pass, "converged": rb.stats["converged"],
           "max_rel_diff_vs_single_seed_rows_0_100_255": diffs, "mass_per_row_max": float(vals.sum(axis=1).max())})
    Gb.close()


def c4_graphs(count=128, seed=128, partition_size=16384, reps=3):
    """C4's 128 independent RMAT graphs (scales 10-18, edge factors 8-32, from a fixed seed) running BFS:
    as one disjoint union (gpop_graph_build_union + gpop_run_bfs_union, up to 32 graphs per traversal)
    against one gpop_run per graph on its own layout; median of reps, device times."""
    gg = _gen()
    rng = np.random.default_rng(seed)
    gs = [gg.rmat(int(rng.integers(10, 19)), int(rng.choice([8, 16, 32]))) for _ in range(count)]
    src = [int(gg.roots(g, 1)[0]) for g in gs]
    G = Graph.from_many([(g.row_ptr, g.col) for g in gs], partition_size=partition_size)
    G.run_bfs_union(src)
    union = sorted(G.run_bfs_union(src).stats["device_ms"] for _ in range(reps))[reps // 2]
    lv = G.run_bfs_union(src).values.cpu().numpy()
    off = G.union_offsets()
    G.close()
    single = 0.0
    for g, s in zip(gs, src):
        Gi = Graph.from_csr(g.row_ptr, g.col, partition_size=min(partition_size, 1 << max(5, int(np.log2(g.num_vertices)) - 2)))
        Gi.run("bfs", source=s)
        single += sorted(Gi.run("bfs", source=s).stats["device_ms"] for _ in range(reps))[reps // 2]
        Gi.close()
    te = 0
    for i, g in enumerate(gs):
        deg = np.diff(g.row_ptr)
        te += int(deg[lv[off[i]:off[i + 1]] != 0xFFFFFFFF].sum())
    _emit({"config": "c4", "algo": "bfs_union", "graphs": count, "vertices": int(off[-1]),
           "edges": int(sum(g.num_edges for g in gs)), "partition_size": partition_size, "union_ms": union,
           "separate_runs_ms": single, "speedup": single / union, "traversed_edges": te,
           "union_gteps": te / (union / 1e3) / 1e9})


def nibble(nseeds=16, eps=1e-9, max_iters=100):
    gg = _gen()
    g = gg.rmat(24)
    G = Graph.from_csr(g.row_ptr, g.col, None, partition_size=16384)
    for s in gg.roots(g, nseeds):
        s = int(s)
        r = _median_run(G, "nibble", reps=3, source=s, epsilon=eps, max_iters=max_iters)
        _emit({"config": "nibble", "graph": "rmat24", "vertices": g.num_vertices, "edges": g.num_edges,
               "partition_size": 16384, "seed": s, "epsilon": eps, "max_iters": max_iters,
               "iterations": r.stats["iterations"], "converged": r.stats["converged"],
               "ms": r.stats["device_ms"], "support": int((r.values > 0).sum().item()),
               "edges_scattered": r.stats["edges_scattered"], "pc_partition_steps": r.stats["pc_partition_steps"],
               "sc_partition_steps": r.stats["sc_partition_steps"], "kernels_ms": _kernels(r.stats)})
    G.close()


def degree(scale=26, efs=(1, 2, 4, 8, 16, 32), cc_max_ef=16):
    from . import GpopError
    gg = _gen()
    for ef in efs:
        g = gg.rmat(scale, ef).with_weights()
        root = int(gg.roots(g, 1)[0])
        out = {"config": "degree", "graph": f"rmat{scale}", "edge_factor": ef, "vertices": g.num_vertices,
               "edges": g.num_edges, "partition_size": 16384}
        try:
            G = Graph.from_csr(g.row_ptr, g.col, g.weights, partition_size=16384)
        except GpopError as e:  # the layout does not fit: recorded, and the sweep goes on
            out["skipped"] = str(e)
            _emit(out)
            del g
            continue
        info = G.info()
        out["r"] = info["num_png"] / max(g.num_edges, 1)
        for algo, kw in (("pagerank", dict(max_iters=10)), ("bfs", dict(source=root)), ("sssp", dict(source=root)),
                         ("nibble", dict(source=root, epsilon=1e-9, max_iters=100))):
            r = _median_run(G, algo, **kw)
            out[algo] = {"ms": r.stats["device_ms"], "iterations": r.stats["iterations"],
                         "pc_partition_steps": r.stats["pc_partition_steps"],
                         "sc_partition_steps": r.stats["sc_partition_steps"]}
        G.close()
        if ef <= cc_max_ef:
            gs = gg.symmetrized(g)
            try:
                Gs = Graph.from_csr(gs.row_ptr, gs.col, None, partition_size=16384)
                r = _median_run(Gs, "cc")
                out["cc"] = {"ms": r.stats["device_ms"], "iterations": r.stats["iterations"],
                             "edges_sym": gs.num_edges, "pc_partition_steps": r.stats["pc_partition_steps"],
                             "sc_partition_steps": r.stats["sc_partition_steps"]}
                Gs.close()
            except GpopError as e:
                out["cc"] = {"edges_sym": gs.num_edges, "skipped": str(e)}
            del gs
        _emit(out)
        del g


def ablation():
    gg = _gen()
    g = gg.rmat(24).with_weights()
    root = int(gg.roots(g, 1)[0])
    G = Graph.from_csr(g.row_ptr, g.col, g.weights, partition_size=16384)
    for algo in ("bfs", "sssp"):
        for mode in ("force_sc", "force_pc", "analytic"):
            r = _median_run(G, algo, source=root, mode=mode)
            _emit({"config": "ablation", "graph": "rmat24", "algo": algo, "mode": mode, "root": root,
                   "ms": r.stats["device_ms"], "iterations": r.stats["iterations"],
                   "pc_partition_steps": r.stats["pc_partition_steps"],
                   "sc_partition_steps": r.stats["sc_partition_steps"], "model_bytes": r.stats["model_bytes"],
                   "kernels_ms": _kernels(r.stats)})
    G.close()
    del g
    gs = gg.symmetrized(gg.rmat(24))
    Gs = Graph.from_csr(gs.row_ptr, gs.col, None, partition_size=16384)
    for mode in ("force_sc", "force_pc", "analytic"):
        r = _median_run(Gs, "cc", mode=mode)
        _emit({"config": "ablation", "graph": "rmat24_sym", "algo": "cc", "mode": mode, "edges": gs.num_edges,
               "ms": r.stats["device_ms"], "iterations": r.stats["iterations"],
               "pc_partition_steps": r.stats["pc_partition_steps"],
               "sc_partition_steps": r.stats["sc_partition_steps"], "kernels_ms": _kernels(r.stats)})
    Gs.close()


def isg(waves=(0, 2, 4, 8), ratio=8):
    """Interleaved scatter-gather (Sec. 3.3) against bulk-synchronous iterations, the paper's GPOP_DI / GPOP_DC
    comparison: SSSP on RMAT-24 (4 roots) and CC on symmetrised RMAT-24, Eq. (mode) at the measured ratio;
    device time, iterations (one wave each) and sweeps."""
    gg = _gen()
    g = gg.rmat(24).with_weights()
    roots = [int(r) for r in gg.roots(g, 4)]
    G = Graph.from_csr(g.row_ptr, g.col, g.weights, partition_size=16384)
    for w in waves:
        ms = its = 0.0
        for root in roots:
            r = _median_run(G, "sssp", source=root, isg_waves=w, bw_ratio=(ratio, 1))
            ms += r.stats["device_ms"]
            its += r.stats["iterations"]
        _emit({"config": "isg", "graph": "rmat24", "algo": "sssp", "isg_waves": w, "roots": len(roots),
               "ms_mean": ms / len(roots), "iterations_mean": its / len(roots),
               "sweeps_mean": its / len(roots) / max(w, 1)})
    G.close()
    del g
    gs = gg.symmetrized(gg.rmat(24))
    Gs = Graph.from_csr(gs.row_ptr, gs.col, None, partition_size=16384)
    for w in waves:
        r = _median_run(Gs, "cc", isg_waves=w, bw_ratio=(ratio, 1))
        _emit({"config": "isg", "graph": "rmat24_sym", "algo": "cc", "isg_waves": w, "ms": r.stats["device_ms"],
               "iterations": r.stats["iterations"], "sweeps": r.stats["iterations"] / max(w, 1)})
    Gs.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--configs", default="c1,c2,c3,c4,c4_graphs,nibble,ablation,isg,degree")
    a = ap.parse_args()
    fns = {"c1": c1, "c2": c2, "c3": c3, "c4": c4, "c4_graphs": c4_graphs, "nibble": nibble, "ablation": ablation,
           "isg": isg, "degree": degree}
    for c in a.configs.split(","):
        fns[c]()


if __name__ == "__main__":
    main()
