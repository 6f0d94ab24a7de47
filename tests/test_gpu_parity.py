"""CUDA path vs the CPU oracle through the C ABI, element by element.

Integer results (BFS levels and parents, SSSP distances, CC labels) must be
bit-exact; FP32 PageRank / PPR must be within L-inf relative error 1e-5 of the
FP64 oracle (PPR: relative on the oracle's support, absolute 1e-12 elsewhere).
Per-iteration modes and frontier sizes must equal the serial GPOP engine's
(Tier 2) exactly: both evaluate Eq. (mode) in exact integers.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PR_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def lib():
    import paper_1806_08092_gb300 as gp
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gp.build()
    return gp


def G(g, P):
    import paper_1806_08092_gb300 as gp
    return gp.Graph.from_csr(g.row_ptr, g.col, g.weights, partition_size=P)


def pr_err(x, ref):
    return float(np.max(np.abs(x.astype(np.float64) - ref) / ref))


def u64_to_u32(a):
    out = a.copy()
    out[a == O.U64_INF] = O.U32_INF
    return out.astype(np.uint32)


SMALL = [
    ("ring", gg.ring(100)), ("path", gg.path(70)), ("star", gg.star(200)), ("complete", gg.complete(40)),
    ("rings", gg.disjoint_rings([33, 1, 64, 7])), ("uniform_ragged", gg.uniform(3001, 20000)),
    ("sparse_sinks", gg.uniform(2500, 3000)), ("rmat10", gg.rmat(10)), ("rmat13", gg.rmat(13)),
    ("multi", gg.multigraph(40, list(range(40)) * 3 + [5] * 5, [(3 * i) % 40 for i in range(120)] + [5, 5, 6, 6, 7])),
]
POLICIES = ["analytic", "force_sc", "force_pc"]


@pytest.mark.parametrize("name,g", SMALL, ids=[s[0] for s in SMALL])
@pytest.mark.parametrize("P", [32, 256, 4096])
def test_pagerank_small(name, g, P):
    ref, _, _ = O.pagerank(g, 0.85, max_iters=15)
    Gd = G(g, P)
    for pol in POLICIES:
        r = Gd.run("pagerank", max_iters=15, mode=pol)
        assert r.stats["iterations"] == 15
        assert pr_err(r.values.cpu().numpy(), ref) <= PR_TOL, pol


@pytest.mark.parametrize("name,g", SMALL, ids=[s[0] for s in SMALL])
@pytest.mark.parametrize("P", [32, 1024])
def test_bfs_sssp_small(name, g, P):
    gw = g.with_weights()
    Gd = G(gw, P)
    for root in gg.roots(g, 3):
        root = int(root)
        level, parent = O.bfs(g, root)
        dist = u64_to_u32(O.sssp(gw, root))
        for pol in POLICIES:
            r = Gd.run("bfs", source=root, mode=pol)
            assert np.array_equal(r.values.cpu().numpy(), level), pol
            assert np.array_equal(r.parent.cpu().numpy(), parent), pol
            r = Gd.run("sssp", source=root, mode=pol)
            assert np.array_equal(r.values.cpu().numpy(), dist), pol


@pytest.mark.parametrize("name,g", SMALL, ids=[s[0] for s in SMALL])
def test_cc_small(name, g):
    gs = gg.symmetrized(g)
    label = O.cc(gs)
    for P in (32, 512):
        Gd = G(gs, P)
        for pol in POLICIES:
            r = Gd.run("cc", mode=pol)
            assert np.array_equal(r.values.cpu().numpy(), label), (P, pol)


@pytest.mark.parametrize("name,g", SMALL[4:], ids=[s[0] for s in SMALL[4:]])
def test_ppr_small(name, g):
    Gd = G(g, 64)
    for s in gg.roots(g, 2):
        s = int(s)
        ref, _, _ = O.ppr(g, s, 0.15, max_iters=30)
        for pol in POLICIES:
            r = Gd.run("ppr", source=s, damping=0.85, max_iters=30, mode=pol)
            x = r.values.cpu().numpy().astype(np.float64)
            sup = ref > 0
            assert np.all(np.abs(x[sup] - ref[sup]) / ref[sup] <= PR_TOL), pol
            assert np.all(np.abs(x[~sup]) <= 1e-12), pol


@pytest.mark.parametrize("scale,P", [(12, 64), (14, 512), (16, 1024)])
def test_modes_and_frontiers_match_tier2(scale, P):
    g = gg.rmat(scale).with_weights()
    Gd = G(g, P)
    root = int(gg.roots(g, 1)[0])
    for algo in ("bfs", "sssp"):
        t2 = O.gpop(g, P, algo, root)
        r = Gd.run(algo, source=root, trace=True)
        assert r.stats["iterations"] == t2.iterations
        assert np.array_equal(r.modes, t2.modes)
        assert np.array_equal(r.frontier[:, 0], t2.frontier_vertices)
        assert np.array_equal(r.frontier[:, 1], t2.frontier_edges)
        assert r.stats["model_bytes"] == pytest.approx(float(t2.model_bytes.sum()), rel=1e-12)
    gs = gg.symmetrized(gg.rmat(scale))
    t2 = O.gpop(gs, P, "cc")
    r = G(gs, P).run("cc", trace=True)
    assert r.stats["iterations"] == t2.iterations
    assert np.array_equal(r.modes, t2.modes)


def _dense_column_graph():
    # every one of 16384 sources sends 16 edges into partition 0 (P = 1024): one message block of 262144
    # entries (16384 messages), split over several PC gather tasks
    n, P, fan = 16384, 1024, 16
    u = np.repeat(np.arange(n, dtype=np.int64), fan)
    j = np.tile(np.arange(fan, dtype=np.int64), n)
    v = (u * 37 + j * 61) % P
    return gg.multigraph(n, u.tolist(), v.tolist()).with_weights(), P


@pytest.mark.parametrize("case", ["rmat18_p8192", "rmat18_p16384", "dense_column"])
def test_large_partitions_multi_task_columns(case):
    # columns split over several PC gather tasks (partial vectors), blocks of several entry chunks,
    # blocks whose entries are split over tasks, and at P = 16384 the largest accumulator
    if case == "dense_column":
        g, P = _dense_column_graph()
    else:
        g, P = gg.rmat(18).with_weights(), int(case.split("_p")[1])
    Gd = G(g, P)
    assert Gd.info()["num_pc_partials"] > 0
    # force_sc also splits the hub partitions' SC scatter into edge-range units (> 131072 active edges)
    ref, _, _ = O.pagerank(g, 0.85, max_iters=5)
    for pol in ("analytic", "force_pc", "force_sc"):
        r = Gd.run("pagerank", max_iters=5, mode=pol)
        assert pr_err(r.values.cpu().numpy(), ref) <= PR_TOL, pol
    root = int(gg.roots(g, 1)[0])
    level, parent = O.bfs(g, root)
    dist = u64_to_u32(O.sssp(g, root))
    for pol in ("analytic", "force_pc", "force_sc"):
        r = Gd.run("bfs", source=root, mode=pol)
        assert np.array_equal(r.values.cpu().numpy(), level), pol
        assert np.array_equal(r.parent.cpu().numpy(), parent), pol
        r = Gd.run("sssp", source=root, mode=pol)
        assert np.array_equal(r.values.cpu().numpy(), dist), pol


def test_traced_and_untraced_runs_agree():
    # tracing reads every plan's modes and frontier; the results, iterations and launches stay the same
    g = gg.rmat(14).with_weights()
    Gd = G(g, 512)
    root = int(gg.roots(g, 1)[0])
    for algo, kw in (("pagerank", dict(max_iters=30, tol=1e-9)), ("bfs", dict(source=root)),
                     ("sssp", dict(source=root)), ("ppr", dict(source=root, max_iters=50, tol=1e-10))):
        for pol in ("analytic", "force_sc"):
            # a warm-up with the same policy: the data rows a run must clear depend on the run before it
            Gd.run(algo, mode=pol, **kw)
            a = Gd.run(algo, mode=pol, profile=True, **kw)
            b = Gd.run(algo, mode=pol, profile=True, trace=True, **kw)
            assert np.array_equal(a.values.cpu().numpy().view(np.uint32), b.values.cpu().numpy().view(np.uint32))
            for key in ("iterations", "converged", "edges_scattered", "pc_partition_steps", "sc_partition_steps",
                        "kernel_launches"):
                assert a.stats[key] == b.stats[key], (algo, pol, key)
            assert a.stats["kernel_launches"][0] == a.stats["iterations"] + 1


def test_bounded_wait_gives_up_and_context_stays_usable():
    # the engine's bounded mbarrier wait, against a phase that nothing completes: it must give up after
    # its polls and raise the error word (no trap, no hang), and the device must stay usable afterwards
    import paper_1806_08092_gb300 as gp
    assert gp.probe_bounded_wait(1 << 16) is True
    assert gp.probe_bounded_wait(0) is True
    g = gg.rmat(10)
    root = int(gg.roots(g, 1)[0])
    assert np.array_equal(G(g, 64).run("bfs", source=root).values.cpu().numpy(), O.bfs(g, root)[0])


def _bits(t):
    return t.cpu().numpy().view(np.uint32)


def test_resume_from_checkpoint_matches_uninterrupted_run():
    # a run split at iteration `split` (continued on the same handle, and from an exported checkpoint on a
    # fresh handle of the same graph) gives the uninterrupted run's results bit for bit
    g = gg.rmat(14).with_weights()
    root = int(gg.roots(g, 1)[0])
    cases = (("pagerank", dict(max_iters=20), 8), ("pagerank", dict(max_iters=300, tol=1e-9), 10),
             ("bfs", dict(source=root), 3), ("sssp", dict(source=root), 4),
             ("ppr", dict(source=root, max_iters=80, tol=1e-10), 7),
             ("nibble", dict(source=root, epsilon=1e-4, max_iters=200), 3))
    for algo, kw, split in cases:
        Gd = G(g, 512)
        full = Gd.run(algo, **kw)
        total = kw.get("max_iters", 1000)
        first = Gd.run(algo, **{**kw, "max_iters": split})
        assert first.stats["iterations"] == split, algo
        blob = Gd.state_export()
        same = Gd.run(algo, resume=True, **{**kw, "max_iters": total - split})
        fresh = G(g, 512)
        fresh.state_import(blob)
        other = fresh.run(algo, resume=True, **{**kw, "max_iters": total - split})
        for r in (same, other):
            assert split + r.stats["iterations"] == full.stats["iterations"], algo
            assert r.stats["converged"] == full.stats["converged"], algo
            assert np.array_equal(_bits(r.values), _bits(full.values)), algo
            if algo == "bfs":
                assert np.array_equal(_bits(r.parent), _bits(full.parent))
    gs = gg.symmetrized(gg.rmat(13))
    Gs = G(gs, 256)
    full = Gs.run("cc")
    Gs.run("cc", max_iters=2)
    rest = Gs.run("cc", resume=True)
    assert 2 + rest.stats["iterations"] == full.stats["iterations"]
    assert np.array_equal(_bits(rest.values), _bits(full.values))


def test_checkpoint_errors():
    import paper_1806_08092_gb300 as gp
    g = gg.rmat(10)
    Gd = G(g, 64)
    with pytest.raises(gp.GpopError):
        Gd.state_export()  # nothing has run
    with pytest.raises(gp.GpopError):
        Gd.run("pagerank", resume=True, max_iters=3)  # no state to continue
    root = int(gg.roots(g, 1)[0])
    Gd.run("bfs", source=root, max_iters=2)
    blob = Gd.state_export()
    with pytest.raises(gp.GpopError):
        Gd.run("pagerank", resume=True, max_iters=3)  # the state is a BFS's
    with pytest.raises(gp.GpopError):
        G(gg.rmat(11), 64).state_import(blob)  # another vertex count
    bad = blob.copy()
    bad[0] ^= 0xFF
    with pytest.raises(gp.GpopError):
        G(g, 64).state_import(bad)  # not a checkpoint
    # another graph with the same vertex and edge counts: one edge's destination moved
    col = g.col.copy()
    row = int(np.flatnonzero(np.diff(g.row_ptr) == 1)[0])  # a vertex with a single out-edge
    e0 = int(g.row_ptr[row])
    col[e0] = (col[e0] + 1) % g.num_vertices if (col[e0] + 1) % g.num_vertices != row else (col[e0] + 2) % g.num_vertices
    other = gp.Graph.from_csr(g.row_ptr, col, partition_size=64)
    with pytest.raises(gp.GpopError, match="another graph"):
        other.state_import(blob)
    with pytest.raises(gp.GpopError, match="partition size"):
        G(g, 128).state_import(blob)  # the same graph, another partition size
    # a resumed run must repeat the options that shape the saved run's result
    fresh = G(g, 64)
    fresh.state_import(blob)
    other_root = int(gg.roots(g, 2)[1])
    with pytest.raises(gp.GpopError, match="source"):
        fresh.run("bfs", source=other_root, resume=True)
    assert fresh.run("bfs", source=root, resume=True).stats["converged"] == 1
    Gd.run("ppr", source=root, max_iters=3)
    with pytest.raises(gp.GpopError, match="damping"):
        Gd.run("ppr", source=root, damping=0.8, max_iters=3, resume=True)
    with pytest.raises(gp.GpopError, match="message format"):
        Gd.run("ppr", source=root, max_iters=3, resume=True, msg_bf16=True)
    Gd.run("nibble", source=root, epsilon=1e-4, max_iters=2)
    with pytest.raises(gp.GpopError, match="threshold"):
        Gd.run("nibble", source=root, epsilon=1e-5, max_iters=2, resume=True)


def test_partition_size_autotuner():
    # every candidate is built and timed through the library; the fastest is returned, and a candidate
    # the library rejects (not a power of two) is listed with the library's message and skipped
    from paper_1806_08092_gb300.autotune import pick_partition_size
    g = gg.rmat(13).with_weights()
    root = int(gg.roots(g, 1)[0])
    best, table = pick_partition_size(g.row_ptr, g.col, g.weights, runs=[("bfs", {"source": root}),
                                      ("sssp", {"source": root})], candidates=(256, 1000, 2048, 8192), reps=3)
    timed = [r for r in table if r[1] is not None]
    assert [r[0] for r in timed] == [256, 2048, 8192]
    assert best == min(timed, key=lambda r: r[1])[0]
    rejected = [r for r in table if r[1] is None]
    assert [r[0] for r in rejected] == [1000] and "power of two" in rejected[0][3]
    # the layout it picks gives the same exact results
    Gd = G(g, best)
    assert np.array_equal(Gd.run("bfs", source=root).values.cpu().numpy(), O.bfs(g, root)[0])


def test_bw_ratio_autotuner():
    # every candidate ratio is timed through the library on one layout; the results at any ratio are the
    # exact ones (the ratio only moves partitions between the modes)
    from paper_1806_08092_gb300.autotune import pick_bw_ratio
    g = gg.rmat(14).with_weights()
    root = int(gg.roots(g, 1)[0])
    Gd = G(g, 1024)
    best, table = pick_bw_ratio(Gd, runs=[("bfs", {"source": root}), ("sssp", {"source": root})],
                                candidates=(1, 2, 8, 64), reps=2)
    assert [t[0] for t in table] == [1, 2, 8, 64] and all(t[1] is not None for t in table)
    assert best == (min(table, key=lambda t: t[1])[0], 1)
    level, parent = O.bfs(g, root)
    for ratio in (1, 8, 64):
        r = Gd.run("bfs", source=root, bw_ratio=(ratio, 1))
        assert np.array_equal(r.values.cpu().numpy(), level) and np.array_equal(r.parent.cpu().numpy(), parent)
        t2 = O.gpop(g, 1024, "bfs", root, bw_ratio=(ratio, 1))
        assert np.array_equal(Gd.run("bfs", source=root, bw_ratio=(ratio, 1), trace=True).modes, t2.modes)


# --- interleaved scatter-gather (Sec. 3.3) --------------------------------------------------------

@pytest.mark.parametrize("name,g", SMALL, ids=[s[0] for s in SMALL])
@pytest.mark.parametrize("P,waves", [(32, 2), (256, 4), (4096, 2)])
def test_isg_cc_sssp_exact(name, g, P, waves):
    # the waves change the order in which partitions scatter, not the fixed point: labels and distances
    # stay bit-exact, in every mode policy
    gw = g.with_weights()
    Gd = G(gw, P)
    gs = gg.symmetrized(g)
    ref_cc = O.cc(gs)
    Gs = G(gs, P)
    for pol in POLICIES:
        assert np.array_equal(Gs.run("cc", mode=pol, isg_waves=waves).values.cpu().numpy(), ref_cc), pol
    for root in gg.roots(g, 2):
        root = int(root)
        ref = u64_to_u32(O.sssp(gw, root))
        for pol in POLICIES:
            r = Gd.run("sssp", source=root, mode=pol, isg_waves=waves)
            assert np.array_equal(r.values.cpu().numpy(), ref), pol
            assert r.stats["converged"] == 1


def test_isg_errors_and_iterations():
    import paper_1806_08092_gb300 as gp
    g = gg.rmat(14).with_weights()
    Gd = G(g, 512)
    root = int(gg.roots(g, 1)[0])
    for algo, kw in (("bfs", dict(source=root)), ("pagerank", dict(max_iters=2)), ("ppr", dict(source=root)),
                     ("nibble", dict(source=root))):
        with pytest.raises(gp.GpopError, match="interleaved"):
            Gd.run(algo, isg_waves=2, **kw)
    # multi-source BFS through the C ABI: its levels depend on the iteration structure
    import ctypes
    from paper_1806_08092_gb300 import _lib
    o = _lib.RunOpts()
    _lib.load().gpop_run_opts_default(ctypes.byref(o))
    o.isg_waves = 2
    src = np.array([root], dtype=np.uint32)
    out = torch.empty(g.num_vertices, dtype=torch.uint32, device="cuda")
    assert _lib.load().gpop_run_msbfs(Gd._h, ctypes.byref(o), ctypes.c_void_p(src.ctypes.data), 1,
                                      ctypes.c_void_p(out.data_ptr()), 1, None) == 1
    # the same distances with and without waves
    bsp = Gd.run("sssp", source=root)
    isg = Gd.run("sssp", source=root, isg_waves=2)
    assert np.array_equal(bsp.values.cpu().numpy(), isg.values.cpu().numpy())


# --- parallel Nibble (Alg. 4) ---------------------------------------------------------------------
# FP32 on the GPU against the FP64 oracle: PR values are probabilities (they sum to 1), compared in
# absolute terms.  The threshold PR >= eps deg is decided on FP32 values on the GPU and on FP64 values
# in the oracle, so a vertex whose PR lies within rounding of eps deg may fall on either side: frontier
# sizes agree to max(2, 2 %) per iteration and the run lengths to 2 iterations (exactly in the worked
# example).  Thresholds near 1 / volume keep the frontier at the threshold for many iterations, where
# such flips accumulate; the cases here end on their own.
NIBBLE_ABS_TOL = 1e-6


def nibble_close(r, ref, it, fr):
    n = min(r.stats["iterations"], it)
    assert abs(r.stats["iterations"] - it) <= 2
    d = np.abs(r.frontier[:n, 0].astype(np.int64) - fr[:n].astype(np.int64))
    assert (d <= np.maximum(2, fr[:n] // 50)).all(), d
    assert np.max(np.abs(r.values.cpu().numpy().astype(np.float64) - ref)) <= NIBBLE_ABS_TOL


@pytest.mark.parametrize("name,g", SMALL, ids=[s[0] for s in SMALL])
@pytest.mark.parametrize("P", [32, 1024])
def test_nibble_small(name, g, P):
    Gd = G(g, P)
    for seed in gg.roots(g, 2):
        seed = int(seed)
        for eps in (1e-3, max(1e-4, 10.0 / max(g.num_edges, 1))):
            ref, it, fr = O.nibble(g, seed, eps, max_iters=200)
            for pol in POLICIES:
                r = Gd.run("nibble", source=seed, epsilon=eps, max_iters=200, mode=pol, trace=True)
                nibble_close(r, ref, it, fr)


def test_nibble_worked_example_and_edge_cases():
    import paper_1806_08092_gb300 as gp
    # the path example of the oracle pins: dyadic values, exact in FP32
    r = G(gg.path(4), 32).run("nibble", source=0, epsilon=0.2, trace=True)
    assert r.stats["iterations"] == 5 and list(r.frontier[:, 0]) == [1, 2, 3, 2, 1]
    assert np.array_equal(r.values.cpu().numpy(), np.array([0.125, 0.1875, 0.1875, 0.5], dtype=np.float32))
    # a sink seed (the path's last vertex) scatters nothing and keeps half its mass
    r = G(gg.path(4), 32).run("nibble", source=3, epsilon=1e-9)
    x = r.values.cpu().numpy()
    assert r.stats["iterations"] == 1 and x[3] == 0.5 and x.sum() == 0.5
    st = gg.star(20)
    with pytest.raises(gp.GpopError):
        G(st, 32).run("nibble", source=0, epsilon=-1.0)
    with pytest.raises(gp.GpopError):
        G(st, 32).run("nibble", source=0, epsilon=float("nan"))
    with pytest.raises(gp.GpopError):
        G(st, 32).run("nibble", source=0, msg_bf16=True)


def test_nibble_large_partitions():
    g, P = gg.rmat(18), 16384
    Gd = G(g, P)
    seed = int(gg.roots(g, 1)[0])
    ref, it, fr = O.nibble(g, seed, 1e-7, max_iters=40)
    for pol in POLICIES:
        r = Gd.run("nibble", source=seed, epsilon=1e-7, max_iters=40, mode=pol, trace=True)
        nibble_close(r, ref, it, fr)


# --- multi-source BFS (gpop_run_msbfs) ------------------------------------------------------------

def _sources(g, n, seed=3):
    rng = np.random.default_rng(seed)
    src = rng.integers(0, g.num_vertices, size=n)
    if n > 4:
        src[3] = src[1]  # a repeated source
    return src


@pytest.mark.parametrize("name,g", SMALL, ids=[s[0] for s in SMALL])
@pytest.mark.parametrize("P", [32, 1024])
def test_msbfs_small(name, g, P):
    # 40 sources: one full 32-source pass and a ragged pass of 8
    Gd = G(g, P)
    src = _sources(g, 40)
    ref = O.msbfs(g, src)
    for pol in POLICIES:
        r = Gd.run_msbfs(src, mode=pol)
        assert np.array_equal(r.values.cpu().numpy(), ref), pol
    r = Gd.run_msbfs(src[:7], device_out=False)
    assert np.array_equal(r.values, ref[:7])


@pytest.mark.parametrize("case", ["rmat18_p8192", "rmat18_p16384", "dense_column"])
def test_msbfs_large_partitions(case):
    if case == "dense_column":
        g, P = _dense_column_graph()
    else:
        g, P = gg.rmat(18), int(case.split("_p")[1])
    Gd = G(g, P)
    src = _sources(g, 33, seed=5)
    ref = O.msbfs(g, src)
    for pol in POLICIES:
        r = Gd.run_msbfs(src, mode=pol)
        assert np.array_equal(r.values.cpu().numpy(), ref), pol


@pytest.mark.parametrize("scale,P", [(12, 64), (14, 512)])
def test_msbfs_modes_follow_union_frontier(scale, P):
    # frontier entering iteration t = vertices some source reached at level t - 1; each partition's mode is
    # Eq. (mode) on that frontier's V_a and E_a (exact integers on both sides)
    g = gg.rmat(scale)
    Gd = G(g, P)
    src = _sources(g, 32, seed=11)
    ref = O.msbfs(g, src)
    r = Gd.run_msbfs(src, trace=True)
    assert np.array_equal(r.values.cpu().numpy(), ref)
    Ep, npng = O.partition_stats(g, P)
    k = Ep.shape[0]
    deg = np.diff(g.row_ptr).astype(np.int64)
    lv = ref.astype(np.int64)
    depth = int(lv[lv != O.U32_INF].max()) + 1
    assert r.stats["iterations"] == depth
    for t in range(depth):
        front = (lv == t).any(axis=0)
        assert r.frontier[t, 0] == int(front.sum())
        assert r.frontier[t, 1] == int(deg[front].sum())
        part = np.arange(g.num_vertices) // P
        Va = np.bincount(part[front], minlength=k)
        Ea = np.bincount(part[front], weights=deg[front], minlength=k).astype(np.int64)
        exp = [O.mode_decide(k, int(Ep[q]), int(npng[q]), int(Va[q]), int(Ea[q])) for q in range(k)]
        assert np.array_equal(r.modes[t], np.array(exp, dtype=np.uint8)), t


def test_msbfs_edge_cases():
    import paper_1806_08092_gb300 as gp
    g = gg.rmat(10)
    Gd = G(g, 64)
    r = Gd.run_msbfs([])
    assert tuple(r.values.shape) == (0, g.num_vertices) and r.stats["iterations"] == 0
    with pytest.raises(gp.GpopError):
        Gd.run_msbfs([0, g.num_vertices])
    # one source repeated 32 times: every row the single BFS
    root = int(gg.roots(g, 1)[0])
    r = Gd.run_msbfs([root] * 32)
    assert np.array_equal(r.values.cpu().numpy(), np.tile(O.bfs(g, root)[0], (32, 1)))
    # max_iters caps each pass: iteration t discovers level t, deeper levels stay unreached
    ref = O.msbfs(g, [root])
    r = Gd.run_msbfs([root], max_iters=2)
    exp = np.where(ref <= 2, ref, np.uint32(O.U32_INF))
    assert np.array_equal(r.values.cpu().numpy(), exp)
    # a single-vertex graph
    one = gg.ring(1)
    r = G(one, 32).run_msbfs([0, 0, 0])
    assert np.array_equal(r.values.cpu().numpy(), np.zeros((3, 1), dtype=np.uint32))


# BF16 messages: each message is rounded to 8 mantissa bits (relative error <= 2^-9), and the PageRank
# fixed point amplifies a uniform relative perturbation of the messages by at most d / (1 - d) = 5.7
BF16_TOL = 2e-2


@pytest.mark.parametrize("pol", POLICIES)
def test_bf16_messages_pagerank_and_ppr(pol):
    g = gg.rmat(14)
    Gd = G(g, 256)
    ref, _, _ = O.pagerank(g, 0.85, max_iters=30)
    x32 = Gd.run("pagerank", max_iters=30, mode=pol).values.cpu().numpy()
    x16 = Gd.run("pagerank", max_iters=30, mode=pol, msg_bf16=True).values.cpu().numpy()
    e16, e32 = pr_err(x16, ref), pr_err(x32, ref)
    print(f"PageRank {pol}: L-inf rel error FP32 {e32:.2e}, BF16 messages {e16:.2e}")
    assert e32 <= PR_TOL and e16 <= BF16_TOL
    # an FP32 run after a BF16 run on the same graph is unaffected (bit-exact for all-PC PageRank)
    y32 = Gd.run("pagerank", max_iters=30, mode=pol).values.cpu().numpy()
    assert pr_err(y32, ref) <= PR_TOL
    if pol == "force_pc":
        assert np.array_equal(x32, y32)
    s = int(gg.roots(g, 1)[0])
    pref, _, _ = O.ppr(g, s, 0.15, max_iters=30)
    x = Gd.run("ppr", source=s, damping=0.85, max_iters=30, mode=pol, msg_bf16=True).values.cpu().numpy()
    sup = pref > 0
    assert np.max(np.abs(x[sup] - pref[sup]) / pref[sup]) <= BF16_TOL
    assert np.all(np.abs(x[~sup]) <= 1e-12)


def test_bf16_messages_only_for_pagerank_and_ppr():
    import paper_1806_08092_gb300 as gp
    g = gg.rmat(8).with_weights()
    Gd = G(g, 32)
    for algo in ("bfs", "sssp", "cc"):
        with pytest.raises(gp.GpopError, match="BF16"):
            Gd.run(algo, source=1, msg_bf16=True)


def test_pagerank_rmat16_p1024_10_iterations():
    # PageRank, 10 iterations, d = 0.85, RMAT scale 16, partitions of 1024 vertices
    g = gg.rmat(16)
    ref, _, _ = O.pagerank(g, 0.85, max_iters=10)
    r = G(g, 1024).run("pagerank", max_iters=10)
    assert r.stats["iterations"] == 10
    assert pr_err(r.values.cpu().numpy(), ref) <= PR_TOL
    assert r.stats["sc_partition_steps"] == 0  # all active: Eq. (mode) always picks PC


def test_pagerank_to_residual():
    g = gg.rmat(14)
    ref, it, res = O.pagerank(g, 0.85, max_iters=300, tol=1e-9)
    r = G(g, 1024).run("pagerank", max_iters=300, tol=1e-9)
    assert r.stats["converged"] == 1 and r.stats["residual"] < 1e-9
    assert pr_err(r.values.cpu().numpy(), ref) <= PR_TOL


def test_layout_partition_stats_match_oracle():
    for g, P in ((gg.rmat(12), 128), (gg.uniform(5000, 40000), 1024), (gg.star(100), 32)):
        Ep, npng = O.partition_stats(g, P)
        Gd = G(g, P)
        e, n = Gd.partition_stats()
        assert np.array_equal(e, Ep) and np.array_equal(n, npng)
        info = Gd.info()
        assert info["num_png"] == int(npng.sum()) and info["num_edges"] == g.num_edges


def test_repeated_runs_and_mode_switches_are_consistent():
    # PC rows left over from a previous run or iteration must not leak into later gathers
    g = gg.rmat(13).with_weights()
    Gd = G(g, 256)
    roots = gg.roots(g, 4)
    for i in range(3):
        for root in roots:
            root = int(root)
            for pol in ("force_pc", "analytic", "force_sc"):
                dist = u64_to_u32(O.sssp(g, root))
                assert np.array_equal(Gd.run("sssp", source=root, mode=pol).values.cpu().numpy(), dist)
    x = Gd.run("pagerank", max_iters=5).values.cpu().numpy()
    assert pr_err(x, O.pagerank(g, 0.85, max_iters=5)[0]) <= PR_TOL


def test_host_outputs_and_device_inputs():
    g = gg.rmat(11)
    rp = torch.from_numpy(g.row_ptr.view(np.int64)).cuda()
    col = torch.from_numpy(g.col.view(np.int32)).cuda()
    import paper_1806_08092_gb300 as gp
    Gd = gp.Graph.from_csr(rp.view(torch.uint64), col.view(torch.uint32), partition_size=128)
    root = int(gg.roots(g, 1)[0])
    r = Gd.run("bfs", source=root, device_out=False)
    level, parent = O.bfs(g, root)
    assert np.array_equal(r.values, level) and np.array_equal(r.parent, parent)


def test_errors_are_reported():
    import paper_1806_08092_gb300 as gp
    g = gg.rmat(8)
    bad = g.col.copy()
    bad[3] = g.num_vertices + 5
    with pytest.raises(gp.GpopError, match="INVALID_ARG"):
        gp.Graph.from_csr(g.row_ptr, bad, partition_size=32)
    for P in (16, 48, 32768):  # not a power of two in [32, 16384]
        with pytest.raises(gp.GpopError, match="partition_size"):
            gp.Graph.from_csr(g.row_ptr, g.col, partition_size=P)
    Gd = G(g, 32)
    with pytest.raises(gp.GpopError, match="weighted"):
        Gd.run("sssp", source=0)
    with pytest.raises(gp.GpopError, match="source"):
        Gd.run("bfs", source=g.num_vertices)
    with pytest.raises(gp.GpopError, match="NO_SELECTOR"):
        gp.selector_set(None)
        Gd.run("bfs", source=1, mode="learned")
