"""Partition-size autotuner: builds the layout at each candidate partition size P and keeps the one whose
runs take the least device time.

The paper fixes P by cache capacity (Sec. 5: 256 KB of vertex data); here P also sets the number of
bins, the PC gather's block sizes and the shared-memory column accumulator, so the best P depends on
the graph and the applications run on it.  Every candidate is measured through the library itself
(gpop_graph_build + gpop_run, CUDA-event device times); nothing is modelled.

    from paper_1806_08092_gb300.autotune import pick_partition_size
    best, table = pick_partition_size(row_ptr, col, weights, runs=[("bfs", {"source": r}), ("sssp", {"source": r})])
"""
from __future__ import annotations

from . import Graph, GpopError

DEFAULT_CANDIDATES = (2048, 4096, 8192, 16384)


def pick_partition_size(row_ptr, col, weights=None, runs=(("pagerank", {"max_iters": 10}),),
                        candidates=DEFAULT_CANDIDATES, reps: int = 3):
    """Returns (best P, [(P, total median device ms or None, build seconds or None, reason)...]).

    runs: (algorithm, keyword arguments of Graph.run) pairs timed together; each is run once to warm up,
    then `reps` times, and its median device time is summed over the runs.  A candidate the library
    rejects when building it (an out-of-range P, a layout that does not fit in device memory) or when
    running on it (run buffers that do not fit) is listed with None and the library's message, and skipped.  Raises ValueError when no candidate works."""
    import time
    table = []
    best = None
    for P in candidates:
        try:
            t0 = time.time()
            G = Graph.from_csr(row_ptr, col, weights, partition_size=int(P))
            build_s = time.time() - t0
        except GpopError as e:
            table.append((int(P), None, None, str(e)))
            continue
        try:
            total = 0.0
            for algo, kw in runs:
                G.run(algo, **kw)
                ts = sorted(G.run(algo, **kw).stats["device_ms"] for _ in range(reps))
                total += ts[len(ts) // 2]
        except GpopError as e:  # e.g. run buffers that do not fit, or a gather shape the layout rejects
            table.append((int(P), None, build_s, str(e)))
            continue
        finally:
            G.close()
        table.append((int(P), total, build_s, ""))
        if best is None or total < best[1]:
            best = (int(P), total)
    if best is None:
        raise ValueError("no candidate partition size could be built: " + "; ".join(r[3] for r in table))
    return best[0], table
