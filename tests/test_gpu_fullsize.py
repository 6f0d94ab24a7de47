"""Parity at full workload sizes, in the launch configuration bench.py times (partition size 16384).

RMAT scale 22 (4.2M vertices, ~65M edges): BFS levels and parents, SSSP distances (weights 1..255) and
CC labels (symmetrised graph) bit-exact against the full oracle, SSSP and CC also with interleaved
scatter-gather (Sec. 3.3, 2 and 4 waves).  RMAT scale 24 (16.8M vertices, ~263M
edges): PageRank 10 iterations, and PageRank to an L1 residual below 1e-9, element by element against
the FP64 oracle run to the same tolerance (L-inf relative <= 1e-5, iteration counts compared; BF16
messages reported), plus the fixed-point equation of Alg. 6 on sampled vertices.  The uniform random
graph of the same size (2^24 vertices, 16 x 2^24 edge draws): PageRank 10 iterations.  Seeded PPR at
the bench's partition size on RMAT 18 and 22, and parallel Nibble at eps = 0 (no threshold, so the
frontiers are exact) on a uniform 2^20 graph.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

P_BENCH = 16384


@pytest.fixture(scope="module")
def gp():
    import paper_1806_08092_gb300 as gp
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gp.build()
    return gp


@pytest.fixture(scope="module")
def rmat22():
    return gg.rmat(22).with_weights()


def test_rmat22_bfs_sssp_exact(gp, rmat22):
    g = rmat22
    G = gp.Graph.from_csr(g.row_ptr, g.col, g.weights, partition_size=P_BENCH)
    for root in gg.roots(g, 2):
        root = int(root)
        level, parent = O.bfs(g, root)
        r = G.run("bfs", source=root)
        assert np.array_equal(r.values.cpu().numpy(), level)
        assert np.array_equal(r.parent.cpu().numpy(), parent)
        d = O.sssp(g, root)
        assert int(d[d != O.U64_INF].max()) < 2**32 - 1
        dd = d.copy()
        dd[d == O.U64_INF] = O.U32_INF
        assert np.array_equal(G.run("sssp", source=root).values.cpu().numpy(), dd.astype(np.uint32))
        for w in (2, 4):  # interleaved scatter-gather: the same distances
            r = G.run("sssp", source=root, isg_waves=w, bw_ratio=(8, 1))
            assert np.array_equal(r.values.cpu().numpy(), dd.astype(np.uint32)), w
    G.close()


def test_rmat22_msbfs_64_sources(gp, rmat22):
    # 64 sources in two 32-source passes at the bench partition size: rows of four sources against the
    # full oracle BFS; every row against properties that fix BFS levels (source at 0, no edge spans more
    # than one level downwards, every reached vertex but the source has an in-neighbour one level up)
    g = rmat22
    G = gp.Graph.from_csr(g.row_ptr, g.col, None, partition_size=P_BENCH)
    src = np.asarray(gg.roots(g, 64), dtype=np.int64)
    r = G.run_msbfs(src)
    lv = r.values
    for j in (0, 31, 32, 63):
        assert np.array_equal(lv[j].cpu().numpy(), O.bfs(g, int(src[j]))[0])
    u = torch.from_numpy(g.src().astype(np.int64)).cuda()
    v = torch.from_numpy(g.col.astype(np.int64)).cuda()
    inf = O.U32_INF
    for j in range(64):
        L = lv[j].to(torch.int64)
        assert int(L[int(src[j])]) == 0
        lu, lw = L[u], L[v]
        reached = lu != inf
        assert bool((lw[reached] <= lu[reached] + 1).all())
        # a vertex at level l > 0 has an in-neighbour at level l - 1
        good = torch.zeros_like(L, dtype=torch.bool)
        good[v[reached & (lw == lu + 1)]] = True
        good[int(src[j])] = True
        assert bool((good | (L == inf)).all())
    G.close()


def test_rmat22_cc_exact(gp, rmat22):
    gs = gg.symmetrized(rmat22)
    G = gp.Graph.from_csr(gs.row_ptr, gs.col, partition_size=P_BENCH)
    ref = O.cc(gs)
    assert np.array_equal(G.run("cc").values.cpu().numpy(), ref)
    for w in (2, 4):  # interleaved scatter-gather: the same labels
        assert np.array_equal(G.run("cc", isg_waves=w, bw_ratio=(8, 1)).values.cpu().numpy(), ref), w
    G.close()


@pytest.fixture(scope="module")
def rmat24(gp):
    g = gg.rmat(24)
    G = gp.Graph.from_csr(g.row_ptr, g.col, partition_size=P_BENCH)
    yield g, G
    G.close()


def test_rmat24_pagerank_10_iterations(rmat24):
    g, G = rmat24
    ref, _, _ = O.pagerank(g, 0.85, max_iters=10)
    x = G.run("pagerank", max_iters=10).values.cpu().numpy().astype(np.float64)
    e32 = np.max(np.abs(x - ref) / ref)
    # BF16 messages (FP32 gather): bound derived in test_gpu_parity (2^-9 per message, x d/(1-d))
    x16 = G.run("pagerank", max_iters=10, msg_bf16=True).values.cpu().numpy().astype(np.float64)
    e16 = np.max(np.abs(x16 - ref) / ref)
    print(f"RMAT-24 PageRank 10 iterations, L-inf rel error vs FP64 oracle: FP32 {e32:.2e}, BF16 messages {e16:.2e}")
    assert e32 <= 1e-5 and e16 <= 2e-2


def test_rmat24_pagerank_converged_fixed_point_sampled(rmat24):
    g, G = rmat24
    r = G.run("pagerank", max_iters=300, tol=1e-9)
    assert r.stats["converged"] == 1 and r.stats["residual"] < 1e-9
    x = r.values.cpu().numpy().astype(np.float64)
    n = g.num_vertices
    deg = np.diff(g.row_ptr).astype(np.float64)
    # sampled destinations: the 64 largest in-degrees plus 4000 uniform draws
    indeg = np.bincount(g.col, minlength=n)
    rng = np.random.default_rng(24)
    sample = np.unique(np.concatenate([np.argsort(indeg)[-64:], rng.integers(0, n, 4000)]))
    want = np.zeros(n, dtype=bool)
    want[sample] = True
    src = g.src()
    m = want[g.col]
    y = np.zeros(n)
    np.add.at(y, g.col[m].astype(np.int64), x[src[m]] / deg[src[m]])
    fixed = (1 - 0.85) / n + 0.85 * y[sample]
    assert np.max(np.abs(x[sample] - fixed) / fixed) <= 1e-5
    # rank mass: sum x = (1-d) + d (sum x - sink mass) at the fixed point
    sink = deg == 0
    assert abs(x.sum() - ((1 - 0.85) + 0.85 * (x.sum() - x[sink].sum()))) <= 1e-5 * x.sum()


@pytest.fixture(scope="module")
def rmat24_converged(rmat24):
    # the FP64 oracle run to the bench's tolerance (about 90 power iterations of Alg. 6)
    g, _ = rmat24
    return O.pagerank(g, 0.85, max_iters=300, tol=1e-9)


def test_rmat24_pagerank_to_1e9_against_oracle(rmat24, rmat24_converged):
    g, G = rmat24
    ref, it_ref, res_ref = rmat24_converged
    r = G.run("pagerank", max_iters=300, tol=1e-9)
    x = r.values.cpu().numpy().astype(np.float64)
    err = float(np.max(np.abs(x - ref) / ref))
    print(f"RMAT-24 PageRank to L1 < 1e-9: GPU {r.stats['iterations']} iterations (residual "
          f"{r.stats['residual']:.3e}), oracle {it_ref} (residual {res_ref:.3e}); L-inf rel error {err:.2e}")
    assert res_ref < 1e-9 and r.stats["converged"] == 1 and r.stats["residual"] < 1e-9
    # the FP32 residual tracks the FP64 one until both fall below the tolerance
    assert abs(r.stats["iterations"] - it_ref) <= 2
    assert err <= 1e-5


def test_rmat24_pagerank_bf16_messages_at_convergence(rmat24, rmat24_converged):
    g, G = rmat24
    ref, _, _ = rmat24_converged
    r = G.run("pagerank", max_iters=300, tol=1e-9, msg_bf16=True)
    x = r.values.cpu().numpy().astype(np.float64)
    e16 = float(np.max(np.abs(x - ref) / ref))
    print(f"RMAT-24 PageRank with BF16 messages to L1 < 1e-9: {r.stats['iterations']} iterations, "
          f"L-inf rel error vs the FP64 oracle {e16:.2e} (reported; BF16 keeps 8 bits of a message)")
    assert r.stats["converged"] == 1
    assert e16 <= 2e-2  # 2^-9 per message, amplified at most d / (1 - d) by the iteration


def test_uniform24_pagerank_10_iterations(gp):
    g = gg.uniform(1 << 24, 16 << 24)
    G = gp.Graph.from_csr(g.row_ptr, g.col, partition_size=P_BENCH)
    ref, _, _ = O.pagerank(g, 0.85, max_iters=10)
    x = G.run("pagerank", max_iters=10).values.cpu().numpy().astype(np.float64)
    G.close()
    err = float(np.max(np.abs(x - ref) / ref))
    print(f"uniform 2^24 PageRank 10 iterations: L-inf rel error {err:.2e}")
    assert err <= 1e-5


def _ppr_error_profile(x, ref):
    """Largest relative error over the oracle's support, by floor of the oracle value."""
    out = {}
    for floor in (0.0, 1e-30, 1e-20, 1e-10):
        m = ref > floor
        out[floor] = float(np.max(np.abs(x[m] - ref[m]) / ref[m])) if m.any() else 0.0
    return out


@pytest.mark.parametrize("scale", [18, 22])
def test_ppr_bench_partition_size(gp, scale):
    g = gg.rmat(scale)
    G = gp.Graph.from_csr(g.row_ptr, g.col, partition_size=P_BENCH)
    s = int(gg.roots(g, 1)[0])
    ref, _, _ = O.ppr(g, s, 0.15, max_iters=40)
    x = G.run("ppr", source=s, damping=0.85, max_iters=40).values.cpu().numpy().astype(np.float64)
    G.close()
    prof = _ppr_error_profile(x, ref)
    print(f"RMAT-{scale} PPR 40 iterations, P = {P_BENCH}: max rel error by oracle floor {prof}; "
          f"support {(ref > 0).sum()}, smallest {ref[ref > 0].min():.2e}")
    assert np.all(np.abs(x[ref == 0]) <= 1e-12)
    assert prof[0.0] <= 1e-5


def test_nibble_eps0_uniform20_exact_frontiers(gp):
    # at eps = 0 every reached vertex with out-edges stays on (PR >= 0 always holds), so no FP32 rounding
    # can move a vertex across the threshold: the frontier sizes are exact, the values FP32 sums of the
    # lazy walk's probabilities
    g = gg.uniform(1 << 20, 16 << 20)
    G = gp.Graph.from_csr(g.row_ptr, g.col, partition_size=P_BENCH)
    seed = int(gg.roots(g, 1)[0])
    ref, it, fr = O.nibble(g, seed, 0.0, max_iters=8)
    r = G.run("nibble", source=seed, epsilon=0.0, max_iters=8, trace=True)
    G.close()
    x = r.values.cpu().numpy().astype(np.float64)
    assert r.stats["iterations"] == it
    assert np.array_equal(r.frontier[:, 0], fr)
    sup = ref > 0
    assert np.array_equal(x > 0, sup)
    err = float(np.max(np.abs(x[sup] - ref[sup]) / ref[sup]))
    print(f"uniform 2^20 Nibble eps = 0, {it} iterations: frontiers {[int(f) for f in fr]}; L-inf rel error {err:.2e}")
    assert err <= 1e-5


def test_rmat22_ppr_batch_64_seeds(gp, rmat22):
    # two passes of 32 seeds at partition size 1024 (the batched gather keeps 32 values per destination in
    # shared memory): four rows against the full oracle, all rows against the single-seed iteration's
    # invariant (a PPR vector's mass is at most 1 and its support contains the seed)
    g = rmat22
    G = gp.Graph.from_csr(g.row_ptr, g.col, partition_size=1024)
    seeds = [int(s) for s in gg.roots(g, 64)]
    r = G.run_ppr_batch(seeds, max_iters=40)
    vals = r.values.cpu().numpy()
    G.close()
    errs = []
    for j in (0, 31, 32, 63):
        ref, _, _ = O.ppr(g, seeds[j], 0.15, max_iters=40)
        sup = ref > 0
        errs.append(float(np.max(np.abs(vals[j][sup].astype(np.float64) - ref[sup]) / ref[sup])))
        assert np.all(vals[j][~sup] == 0)
    print(f"RMAT-22 batched PPR, 64 seeds, 40 iterations: L-inf rel error of rows 0/31/32/63 {errs}")
    assert max(errs) <= 1e-5
    mass = vals.astype(np.float64).sum(axis=1)
    assert np.all(mass <= 1.0 + 1e-5) and np.all(vals[np.arange(64), seeds] >= 0.15 - 1e-6)


def test_128_uneven_rmat_graphs_bfs_union(gp):
    # 128 RMAT graphs of scales 10 to 18 and edge factors 8 to 32 (drawn from a fixed seed) as one union:
    # every graph's levels from its own root against the oracle's BFS of that graph alone, and against the
    # properties that fix BFS levels
    rng = np.random.default_rng(128)
    gs = [gg.rmat(int(rng.integers(10, 19)), int(rng.choice([8, 16, 32]))) for _ in range(128)]
    G = gp.Graph.from_many([(g.row_ptr, g.col) for g in gs], partition_size=16384)
    off = G.union_offsets()
    src = [int(gg.roots(g, 1)[0]) for g in gs]
    lv = G.run_bfs_union(src).values.cpu().numpy()
    G.close()
    for i in range(128):
        assert np.array_equal(lv[off[i]:off[i + 1]], O.bfs(gs[i], src[i])[0]), i
    for i, g in enumerate(gs):
        L = lv[off[i]:off[i + 1]].astype(np.int64)
        assert L[src[i]] == 0
        u, v = g.src().astype(np.int64), g.col.astype(np.int64)
        reached = L[u] != O.U32_INF
        assert np.all(L[v][reached] <= L[u][reached] + 1)
