"""Autotuners: the partition size P (builds the layout at each candidate and keeps the one whose runs take
the least device time) and the bandwidth ratio BW_PC / BW_SC of Eq. (mode) (runs on one layout at each
candidate ratio).

The paper fixes P by cache capacity (Sec. 5: 256 KB of vertex data); here P also sets the number of
bins, the PC gather's block sizes and the shared-memory column accumulator, so the best P depends on
the graph and the applications run on it.  Every candidate is measured through the library itself
(gpop_graph_build + gpop_run, CUDA-event device times); nothing is modelled.

    from paper_1806_08092_gb300.autotune import pick_partition_size, pick_bw_ratio
    best, table = pick_partition_size(row_ptr, col, weights, runs=[("bfs", {"source": r}), ("sssp", {"source": r})])
    ratio, table = pick_bw_ratio(G, runs=[("bfs", {"source": r}), ("sssp", {"source": r})])

Eq. (mode) sends a partition to PC mode when its PC traffic divided by BW_PC is at most its SC traffic
divided by BW_SC.  The paper sets BW_PC / BW_SC = 2 from its CPUs' sequential and random bandwidths; on
another machine the ratio of the two access patterns' sustained bandwidths is different, so it is
measured here: the ratio whose runs take the least device time is kept.
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


DEFAULT_RATIOS = (1, 2, 4, 8, 16, 32)


def pick_bw_ratio(G, runs, candidates=DEFAULT_RATIOS, reps: int = 3):
    """Returns (best BW_PC / BW_SC as (num, 1), [(ratio, total median device ms or None, reason)...]).

    G: a built Graph.  runs: (algorithm, keyword arguments of Graph.run) pairs timed together at each
    candidate ratio (passed as bw_ratio=(ratio, 1)); each is run once to warm up, then `reps` times, and its
    median device time is summed over the runs.  A ratio the library rejects is listed with None."""
    table = []
    best = None
    for r in candidates:
        try:
            total = 0.0
            for algo, kw in runs:
                G.run(algo, bw_ratio=(int(r), 1), **kw)
                ts = sorted(G.run(algo, bw_ratio=(int(r), 1), **kw).stats["device_ms"] for _ in range(reps))
                total += ts[len(ts) // 2]
        except GpopError as e:
            table.append((int(r), None, str(e)))
            continue
        table.append((int(r), total, ""))
        if best is None or total < best[1]:
            best = (int(r), total)
    if best is None:
        raise ValueError("no candidate ratio could be run: " + "; ".join(x[2] for x in table))
    return (best[0], 1), table
