"""Train and evaluate the learned SC/PC selector.

1. collect: run BFS and SSSP with GPOP_MODE_LOG_BOTH on training graphs; every scattered partition of
   every iteration yields one record (8 features, t_PC, t_SC in SM-microseconds, chosen mode, ...).
2. train: fit y = log(t_PC / t_SC) with the library's GPU training kernels (gpop_selector_train).
3. evaluate: end-to-end time of BFS and SSSP with Eq. (mode) (analytic) and with the trained MLP
   (learned) on a held-out graph, same GPU, median over repetitions; plus the mispredicted-bytes regret
   of each policy judged by Eq. (mode)'s own byte model on held-out records.

    python -m paper_1806_08092_gb300.selector_train --out paper_1806_08092_gb300/selector_rmat.f32   # train + eval
    python -m paper_1806_08092_gb300.selector_train --params paper_1806_08092_gb300/selector_rmat.f32 --eval-scale 25
    python -m paper_1806_08092_gb300.selector_train --nibble --out selector.f32   # + Nibble records and evaluation

`selector_rmat.f32` in this package was written by the first command; bench.py reads it.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

from . import Graph, SELECTOR_WEIGHTS as GPOP_WEIGHTS, selector_set, selector_train


def _gen():
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import graphgen
    return graphgen


def training_graphs(scales=(20, 21, 22, 23, 24), uniform_scales=(21, 22)):
    gg = _gen()
    for s in scales:
        yield f"rmat{s}", gg.rmat(s).with_weights()
    for s in uniform_scales:
        n = 1 << s
        yield f"uniform{s}", gg.uniform(n, 16 * n).with_weights()


def collect(graphs, partition_size=16384, roots_per_graph=4, algos=("bfs", "sssp"), capacity=2_000_000,
            nibble_iters=40):
    """LOG_BOTH records of every run.  Nibble runs use eps = 1 / E of the graph, the threshold at which
    its frontier stays large and made of low-degree vertices (the walk thins out to about 1 / volume),
    and stop after nibble_iters iterations."""
    gg = _gen()
    recs = []
    for name, g in graphs:
        G = Graph.from_csr(g.row_ptr, g.col, g.weights, partition_size=partition_size)
        for root in gg.roots(g, roots_per_graph):
            for algo in algos:
                kw = dict(epsilon=1.0 / max(g.num_edges, 1), max_iters=nibble_iters) if algo == "nibble" else {}
                r = G.run(algo, source=int(root), mode="log_both", log_capacity=capacity, **kw)
                if r.log is not None and len(r.log):
                    recs.append(r.log.copy())
        G.close()
    return np.concatenate(recs) if recs else np.zeros((0, 13), np.float32)


def targets(records):
    return np.log(np.maximum(records[:, 8], 1e-3) / np.maximum(records[:, 9], 1e-3)).astype(np.float32)


# features that scale with the graph (log1p E^p, log1p n_png, log1p k): the network extrapolates in them
# (it is piecewise linear), so they get no range limit; the others keep 10 % of their range as margin
SCALE_FEATURES = (2, 5, 6)


def widen_ranges(params):
    nw = GPOP_WEIGHTS
    p = np.array(params, dtype=np.float32).copy()
    fmin, fmax = p[nw + 16:nw + 24], p[nw + 24:nw + 32]
    span = fmax - fmin
    fmin -= 0.1 * span
    fmax += 0.1 * span
    for k in SCALE_FEATURES:
        fmin[k], fmax[k] = -1e30, 1e30  # no limit (parameters must be finite)
    p[nw + 16:nw + 24], p[nw + 24:nw + 32] = fmin, fmax
    return p


def train(records, epochs=3000, lr=3e-3, seed=7):
    params, loss = selector_train(records[:, :8], targets(records), epochs=epochs, lr=lr, seed=seed)
    return widen_ranges(params), loss


def regret_report(params, records):
    """Extra time (SM-us) over the per-record best mode, for Eq. (mode) and for the trained MLP."""
    t_pc, t_sc = records[:, 8].astype(np.float64), records[:, 9].astype(np.float64)
    best = np.minimum(t_pc, t_sc)
    model_pc = records[:, 7] <= 0  # feature 7: log of Eq. (mode)'s cost ratio; <= 0 means PC
    nw = (32 * 8 + 32 + 32 * 32 + 32 + 32 + 1)
    mean, sd = params[nw:nw + 8], params[nw + 8:nw + 16]
    z = (records[:, :8] - mean) / sd
    W1 = params[:256].reshape(32, 8); b1 = params[256:288]; W2 = params[288:1312].reshape(32, 32)
    b2 = params[1312:1344]; W3 = params[1344:1376]; b3 = params[1376]
    h1 = np.maximum(z @ W1.T + b1, 0); h2 = np.maximum(h1 @ W2.T + b2, 0)
    learned_pc = (h2 @ W3 + b3) <= 0
    return {"records": int(len(records)),
            "regret_model_us": float(np.sum(np.where(model_pc, t_pc, t_sc) - best)),
            "regret_learned_us": float(np.sum(np.where(learned_pc, t_pc, t_sc) - best)),
            "agree_with_best_model": float(np.mean(model_pc == (t_pc <= t_sc))),
            "agree_with_best_learned": float(np.mean(learned_pc == (t_pc <= t_sc)))}


def evaluate(g, params, partition_size=16384, roots=4, reps=5, algos=("bfs", "sssp"), run_kw=None,
             calibrated_ratio=(8, 1)):
    """Median device time per (root, algorithm) with Eq. (mode) at the paper's BW_PC/BW_SC = 2 (the model
    the selector replaces), with the trained selector, and with Eq. (mode) at the ratio measured on this GPU
    (autotune.pick_bw_ratio); whether the selector's per-partition modes differ from Eq. (mode)'s."""
    gg = _gen()
    G = Graph.from_csr(g.row_ptr, g.col, g.weights, partition_size=partition_size)
    out = {"analytic_ms": 0.0, "learned_ms": 0.0, "calibrated_ms": 0.0, "fallbacks": 0, "same_modes": True}
    selector_set(params)
    try:
        for root in gg.roots(g, roots):
            for algo in algos:
                t = {"analytic": [], "learned": [], "calibrated": []}
                modes = {}
                for _ in range(reps):
                    for mode in ("analytic", "learned", "calibrated"):
                        kw = dict(run_kw or {})
                        if mode == "calibrated":
                            kw["bw_ratio"] = calibrated_ratio
                        r = G.run(algo, source=int(root), mode="analytic" if mode == "calibrated" else mode,
                                  trace=True, **kw)
                        t[mode].append(r.stats["device_ms"])
                        modes[mode] = r.modes
                for m in t:
                    out[m + "_ms"] += float(np.median(t[m]))
                out["same_modes"] &= bool(np.array_equal(modes["analytic"], modes["learned"]))
    finally:
        selector_set(None)
        G.close()
    out["speedup"] = out["analytic_ms"] / out["learned_ms"] if out["learned_ms"] > 0 else None
    out["calibrated_speedup"] = out["analytic_ms"] / out["calibrated_ms"] if out["calibrated_ms"] > 0 else None
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=None)
    ap.add_argument("--params", default=None)
    ap.add_argument("--eval-scale", type=int, default=25)
    ap.add_argument("--partition", type=int, default=16384)
    ap.add_argument("--epochs", type=int, default=3000)
    ap.add_argument("--nibble", action="store_true",
                    help="also train on Nibble runs (eps = 1 / E) and evaluate Nibble on RMAT-26, edge factor 16")
    ap.add_argument("--nibble-eval-scale", type=int, default=26)
    ap.add_argument("--nibble-eval-ef", type=int, default=16)
    a = ap.parse_args()
    report = {}
    if a.params:
        params = np.fromfile(a.params, dtype=np.float32)
    else:
        t0 = time.time()
        algos = ("bfs", "sssp", "nibble") if a.nibble else ("bfs", "sssp")
        recs = collect(training_graphs(), partition_size=a.partition, algos=algos)
        rng = np.random.default_rng(0)
        idx = rng.permutation(len(recs))
        cut = int(0.8 * len(recs))
        params, loss = train(recs[idx[:cut]], epochs=a.epochs)
        report["train"] = {"records": int(cut), "mse": loss, "seconds": time.time() - t0}
        report["held_out"] = regret_report(params, recs[idx[cut:]])
        if a.out:
            params.astype(np.float32).tofile(a.out)
    gg = _gen()
    g = gg.rmat(a.eval_scale).with_weights()
    report["eval"] = evaluate(g, params, partition_size=a.partition)
    report["eval"]["graph"] = f"rmat{a.eval_scale}"
    del g
    if a.nibble:
        g = gg.rmat(a.nibble_eval_scale, a.nibble_eval_ef)
        report["eval_nibble"] = evaluate(g, params, partition_size=a.partition, roots=2, reps=3, algos=("nibble",),
                                         run_kw=dict(epsilon=1e-9, max_iters=100))
        report["eval_nibble"]["graph"] = f"rmat{a.nibble_eval_scale}_ef{a.nibble_eval_ef}"
    print(json.dumps(report))


if __name__ == "__main__":
    main()
