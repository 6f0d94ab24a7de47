"""Pins the CPU oracle to facts the paper and the mathematics fix (no GPU).

Each test pins one oracle function against something other than itself:
closed forms (ring, complete digraph, symmetric star, PPR on a ring), identities
(mass balance of Alg. 6), independent library routines (scipy.sparse.csgraph
BFS / Dijkstra / components, numpy dense power iteration and linear solve),
a hand-worked example under tests/golden/, and brute-force recounts.
"""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse import csgraph

import graphgen as gg
import oracle as O

D = 0.85


def dense_transition(g):
    """A^T D^-1 with multiplicities (column u scaled by 1/outdeg(u); sinks give zero columns)."""
    n = g.num_vertices
    M = np.zeros((n, n))
    deg = np.diff(g.row_ptr).astype(np.float64)
    src = g.src()
    np.add.at(M, (g.col.astype(np.int64), src.astype(np.int64)), 1.0 / deg[src])
    return M


def small_graphs():
    yield gg.rmat(7)
    yield gg.uniform(97, 600)
    yield gg.uniform(300, 900)                       # sparse: sinks and in-degree-0 vertices
    yield gg.star(9)
    yield gg.disjoint_rings([3, 5, 7])
    yield gg.multigraph(6, [0, 0, 0, 1, 2, 3, 3, 4, 5, 5], [1, 1, 2, 1, 3, 4, 4, 5, 0, 5])


# --- PageRank (Alg. 6) --------------------------------------------------------------------------

@pytest.mark.parametrize("g", [gg.ring(1), gg.ring(2), gg.ring(17), gg.complete(5), gg.complete(13)],
                         ids=lambda g: g.name)
def test_pagerank_uniform_on_regular_graphs(g):
    # every vertex has in-degree = out-degree, so x_t = 1/n exactly for all t
    x, it, _ = O.pagerank(g, D, max_iters=25) if g.num_edges else (np.ones(1), 25, 0)
    assert it == 25
    assert np.allclose(x, 1.0 / g.num_vertices, rtol=1e-14, atol=0)


@pytest.mark.parametrize("n", [2, 3, 10, 101])
def test_pagerank_star_fixed_point(n):
    # symmetric star: x_c = (1+d(n-1)) / (n(1+d)),  x_leaf = (1-d)/n + d x_c / (n-1)
    g = gg.star(n)
    x, it, res = O.pagerank(g, D, max_iters=5000, tol=1e-16)
    xc = (1 + D * (n - 1)) / (n * (1 + D))
    xl = (1 - D) / n + D * xc / (n - 1)
    assert res < 1e-13  # FP64 may settle into a rounding-level cycle
    assert abs(x[0] - xc) <= 1e-14 * xc
    assert np.allclose(x[1:], xl, rtol=1e-13, atol=0)
    assert abs(x.sum() - 1.0) < 1e-13


def test_pagerank_star_detects_wrong_damping():
    # planted mistake: the oracle run with d = 0.8 must miss the d = 0.85 closed form
    n = 10
    x, _, _ = O.pagerank(gg.star(n), 0.8, max_iters=5000, tol=1e-16)
    xc = (1 + D * (n - 1)) / (n * (1 + D))
    assert abs(x[0] - xc) > 1e-3 * xc


@pytest.mark.parametrize("g", list(small_graphs()), ids=lambda g: g.name)
def test_pagerank_mass_balance(g):
    # sum x_{t+1} = (1-d) + d (sum x_t - sink mass of x_t): sinks drop their mass (Alg. 6 scatters from no sink)
    sinks = np.diff(g.row_ptr) == 0
    prev = np.full(g.num_vertices, 1.0 / g.num_vertices)
    for t in range(1, 8):
        x, it, _ = O.pagerank(g, D, max_iters=t)
        assert it == t
        expect = (1 - D) + D * (prev.sum() - prev[sinks].sum())
        assert abs(x.sum() - expect) < 1e-13
        prev = x


@pytest.mark.parametrize("g", list(small_graphs()), ids=lambda g: g.name)
def test_pagerank_matches_dense_power_iteration(g):
    n = g.num_vertices
    M = dense_transition(g)
    x = np.full(n, 1.0 / n)
    for _ in range(30):
        x = (1 - D) / n + D * (M @ x)
    xo, _, _ = O.pagerank(g, D, max_iters=30)
    assert np.max(np.abs(xo - x) / x) < 1e-12


def test_pagerank_residual_history_is_l1_change():
    g = gg.rmat(8)
    xs = [np.full(g.num_vertices, 1.0 / g.num_vertices)]
    for t in range(1, 6):
        xs.append(O.pagerank(g, D, max_iters=t)[0])
    _, _, _, hist = O.pagerank(g, D, max_iters=5, history=True)
    for t in range(5):
        assert abs(hist[t] - np.abs(xs[t + 1] - xs[t]).sum()) < 1e-13 * hist[t]


# --- seeded personalised PageRank ---------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 4, 23])
def test_ppr_ring_closed_form(n):
    # directed ring seeded at 0: x_j = alpha (1-alpha)^j / (1 - (1-alpha)^n)
    a = 0.15
    x, _, res = O.ppr(gg.ring(n) if n > 1 else gg.multigraph(1, [0], [0]), 0, a, max_iters=20000, tol=1e-17)
    j = np.arange(n)
    expect = a * (1 - a) ** j / (1 - (1 - a) ** n)
    assert np.allclose(x, expect, rtol=1e-12, atol=1e-300)


@pytest.mark.parametrize("g", list(small_graphs()), ids=lambda g: g.name)
def test_ppr_linear_solve(g):
    # fixed point solves (I - (1-alpha) A^T D^-1) x = alpha e_s (sinks drop mass)
    a = 0.15
    s = int(gg.roots(g, 1)[0])
    M = dense_transition(g)
    e = np.zeros(g.num_vertices)
    e[s] = 1.0
    expect = np.linalg.solve(np.eye(g.num_vertices) - (1 - a) * M, a * e)
    x, _, res = O.ppr(g, s, a, max_iters=20000, tol=1e-16)
    assert np.max(np.abs(x - expect)) < 1e-13


# --- parallel Nibble (Alg. 4) ------------------------------------------------------------------

def sink_free(n, m, seed):
    # uniform edges plus the cycle 0 -> 1 -> ... -> 0: every vertex has an out-edge
    rng = np.random.default_rng(seed)
    u = np.concatenate([rng.integers(0, n, m), np.arange(n)])
    v = np.concatenate([rng.integers(0, n, m), (np.arange(n) + 1) % n])
    keep = u != v
    return gg.multigraph(n, u[keep].tolist(), v[keep].tolist())


@pytest.mark.parametrize("g", [gg.ring(9), gg.complete(6), sink_free(60, 200, 1)], ids=lambda g: g.name)
def test_nibble_without_threshold_is_the_lazy_walk(g):
    # eps = 0 and no sinks: every reached vertex stays on, so t iterations apply the lazy walk
    # W = (I + A^T D^-1) / 2 to the seed's indicator (half the mass stays, half spreads over out-edges)
    n = g.num_vertices
    A = np.zeros((n, n))
    np.add.at(A, (g.src().astype(np.int64), g.col.astype(np.int64)), 1.0)
    W = 0.5 * (np.eye(n) + (A / A.sum(axis=1, keepdims=True)).T)
    for t in (1, 2, 7, 25):
        pr, it, _ = O.nibble(g, 0, 0.0, max_iters=t)
        assert it == t
        exp = np.linalg.matrix_power(W, t) @ np.eye(n)[0]
        assert np.max(np.abs(pr - exp)) < 1e-14


@pytest.mark.parametrize("eps", [0.0, 1e-6, 1e-4, 1e-3])
def test_nibble_conserves_mass(eps):
    # a kept vertex with out-edges keeps half its PR and sends the other half; a vertex off the frontier
    # keeps all of it: the total stays 1 whatever the threshold truncates
    g = gg.rmat(10)
    for s in gg.roots(g, 3):
        pr, it, fr = O.nibble(g, int(s), eps, max_iters=60)
        assert abs(pr.sum() - 1.0) < 1e-12
        assert (pr >= 0).all() and fr[0] == 1


def test_nibble_one_step_closed_form():
    # a threshold no vertex meets: one iteration, the seed keeps 1/2 and each out-neighbour gets
    # 1 / (2 deg) per edge
    g = gg.rmat(9)
    s = int(gg.roots(g, 1)[0])
    pr, it, fr = O.nibble(g, s, 10.0, max_iters=100)
    deg = int(g.row_ptr[s + 1] - g.row_ptr[s])
    exp = np.zeros(g.num_vertices)
    np.add.at(exp, g.col[g.row_ptr[s]:g.row_ptr[s + 1]].astype(np.int64), 1.0 / (2 * deg))
    exp[s] += 0.5
    assert it == 1 and list(fr) == [1]
    assert np.max(np.abs(pr - exp)) < 1e-15


def test_nibble_path_worked_example():
    # directed path 0 -> 1 -> 2 -> 3 (vertex 3 is a sink), seed 0, eps = 0.2, worked by hand from Alg. 4:
    #  it 1: {0} sends 0.5 to 1; PR0 = 0.5 kept                           -> PR .5 .5 0 0,        on {0,1}
    #  it 2: 0 sends .25 to 1, 1 sends .25 to 2; both halve to .25, kept -> PR .25 .5 .25 0,     on {0,1,2}
    #  it 3: sends .125, .25, .125; 0 and 2 halve below .2 (cond1 fails), 1 kept at .25;
    #        gather: PR1 = .375, PR2 = .375, PR3 = .125 (a sink: never on) -> on {1,2}
    #  it 4: 1 and 2 send .1875 each and fall below .2; 2 receives (.375, on), 3 receives
    #                                                                     -> PR .125 .1875 .375 .3125, on {2}
    #  it 5: 2 sends .1875 to the sink and falls below .2                -> PR .125 .1875 .1875 .5,   empty
    pr, it, fr = O.nibble(gg.path(4), 0, 0.2, max_iters=100)
    assert it == 5 and list(fr) == [1, 2, 3, 2, 1]
    assert np.array_equal(pr, [0.125, 0.1875, 0.1875, 0.5])


# --- BFS (Alg. 5), CC, SSSP (Alg. 7) against scipy ---------------------------------------------

def scipy_csr(g, weighted=False):
    data = g.weights.astype(np.float64) if weighted else np.ones(g.num_edges)
    return sp.csr_matrix((data, g.col.astype(np.int64), g.row_ptr.astype(np.int64)),
                         shape=(g.num_vertices, g.num_vertices))


def bfs_graphs():
    yield gg.rmat(10)
    yield gg.uniform(1000, 3000)
    yield gg.path(40)
    yield gg.ring(33)
    yield gg.star(50)
    yield gg.disjoint_rings([4, 9])


@pytest.mark.parametrize("g", list(bfs_graphs()), ids=lambda g: g.name)
def test_bfs_levels_and_min_parent(g):
    for root in gg.roots(g, 3):
        level, parent = O.bfs(g, int(root))
        dist = csgraph.shortest_path(scipy_csr(g), unweighted=True, indices=int(root))
        exp_level = np.full(g.num_vertices, O.U32_INF, dtype=np.uint64)
        exp_level[~np.isinf(dist)] = dist[~np.isinf(dist)].astype(np.uint64)
        assert np.array_equal(level.astype(np.uint64), exp_level)
        # brute-force parent: smallest in-neighbour one level up
        src, dst = g.src().astype(np.int64), g.col.astype(np.int64)
        lv = level.astype(np.int64)
        ok = (lv[src] != O.U32_INF) & (lv[dst] == lv[src] + 1) & (dst != int(root))
        exp_parent = np.full(g.num_vertices, O.U32_INF, dtype=np.int64)
        np.minimum.at(exp_parent, dst[ok], src[ok])
        exp_parent[int(root)] = int(root)
        assert np.array_equal(parent.astype(np.int64), exp_parent)


def test_bfs_path_closed_form():
    level, parent = O.bfs(gg.path(25), 0)
    assert np.array_equal(level, np.arange(25))
    assert np.array_equal(parent, np.concatenate([[0], np.arange(24)]))


@pytest.mark.parametrize("g", [gg.rmat(10), gg.uniform(700, 2000), gg.disjoint_rings([4, 9, 1])],
                         ids=lambda g: g.name)
def test_msbfs_against_scipy_all_sources(g):
    # 40 sources with repeats (more than one 32-source pass of the GPU path)
    rng = np.random.default_rng(7)
    src = rng.integers(0, g.num_vertices, size=40)
    src[5] = src[17]
    lv = O.msbfs(g, src)
    dist = csgraph.shortest_path(scipy_csr(g), unweighted=True, indices=src.astype(np.int64))
    exp = np.full(dist.shape, O.U32_INF, dtype=np.uint64)
    exp[~np.isinf(dist)] = dist[~np.isinf(dist)].astype(np.uint64)
    assert lv.shape == (40, g.num_vertices)
    assert np.array_equal(lv.astype(np.uint64), exp)


def test_msbfs_ring_closed_form():
    # directed ring of n: level from s to v is (v - s) mod n
    n = 29
    src = np.array([0, 3, 28, 3])
    lv = O.msbfs(gg.ring(n), src)
    v = np.arange(n)
    for j, s in enumerate(src):
        assert np.array_equal(lv[j], (v - s) % n)


@pytest.mark.parametrize("g", [gg.symmetrized(gg.rmat(11)), gg.symmetrized(gg.uniform(2000, 1500)),
                               gg.disjoint_rings([5, 1, 8, 2])], ids=lambda g: g.name)
def test_cc_against_scipy(g):
    label = O.cc(g)
    ncomp, comp = csgraph.connected_components(scipy_csr(g), directed=True, connection="weak")
    exp = np.zeros(g.num_vertices, dtype=np.int64)
    mins = np.full(ncomp, g.num_vertices, dtype=np.int64)
    np.minimum.at(mins, comp, np.arange(g.num_vertices))
    exp = mins[comp]
    assert np.array_equal(label.astype(np.int64), exp)


def test_cc_rings_closed_form():
    label = O.cc(gg.disjoint_rings([3, 4, 5]))
    assert list(label) == [0] * 3 + [3] * 4 + [7] * 5


@pytest.mark.parametrize("g", [gg.rmat(10).with_weights(), gg.uniform(800, 4000).with_weights(),
                               gg.rmat(9).with_weights(hi=9)], ids=lambda g: g.name)
def test_sssp_against_scipy_dijkstra(g):
    for root in gg.roots(g, 3):
        dist = O.sssp(g, int(root))
        ref = csgraph.dijkstra(scipy_csr(g, weighted=True), indices=int(root))
        exp = np.full(g.num_vertices, O.U64_INF, dtype=np.uint64)
        exp[~np.isinf(ref)] = ref[~np.isinf(ref)].astype(np.uint64)
        assert np.array_equal(dist, exp)


def test_sssp_weighted_path_prefix_sums():
    g = gg.path(30).with_weights()
    dist = O.sssp(g, 0)
    assert np.array_equal(dist, np.concatenate([[0], np.cumsum(g.weights)]).astype(np.uint64))


# --- hand-worked golden example (tests/golden/partition_example.txt) ----------------------------

def golden_graph(ex, weighted=True):
    e = np.array(ex["edge"], dtype=np.int64)
    g = gg.from_edges(8, e[:, 0], e[:, 1])
    # weights in CSR order: rows sorted by destination, matching the listing order per source
    wmap = {(a, b): w for a, b, w in ex["edge"]}
    w = np.array([wmap[(int(s), int(d))] for s, d in zip(g.src(), g.col)], dtype=np.int32)
    return gg.CSR(8, g.row_ptr, g.col, w if weighted else None, "golden")


def test_golden_partition_stats(golden_example):
    g = golden_graph(golden_example)
    Ep, npng = O.partition_stats(g, 2)
    for p, e, m in golden_example["stats"]:
        assert (int(Ep[p]), int(npng[p])) == (e, m)


def test_golden_mode_decisions(golden_example):
    g = golden_graph(golden_example)
    Ep, npng = O.partition_stats(g, 2)
    for p, va, ea, num, den, expect in golden_example["mode"]:
        assert O.mode_decide(4, int(Ep[p]), int(npng[p]), va, ea, num, den) == expect
    for mode, p, va, ea, expect in golden_example["bytes"]:
        assert O.mode_bytes(mode, 4, int(Ep[p]), int(npng[p]), va, ea) == pytest.approx(expect, rel=0, abs=1e-12)


def test_golden_traversals(golden_example):
    g = golden_graph(golden_example)
    level, parent = O.bfs(g, 0)
    assert list(level) == golden_example["bfs_level"]
    assert list(parent) == golden_example["bfs_parent"]
    assert list(O.sssp(g, 0)) == golden_example["sssp_dist"]
    assert list(O.cc(g)) == golden_example["cc_label"]
    for policy in ("analytic", "force_sc", "force_pc"):
        r = O.gpop(g, 2, "bfs", 0, policy=policy)
        assert list(r.level) == golden_example["bfs_level"]
        r = O.gpop(g, 2, "sssp", 0, policy=policy)
        assert list(r.values) == golden_example["sssp_dist"]


def test_partition_stats_brute_force():
    for g in (gg.rmat(9), gg.uniform(513, 3000), gg.multigraph(5, [0, 0, 1, 4, 4], [1, 1, 4, 4, 0])):
        for P in (1, 4, 64, 1024):
            Ep, npng = O.partition_stats(g, P)
            k = (g.num_vertices + P - 1) // P
            src = g.src()
            pairs = set(zip(src.tolist(), (g.col // P).tolist()))
            exp_np = np.zeros(k, dtype=np.int64)
            for u, q in pairs:
                exp_np[u // P] += 1
            exp_E = np.bincount(src // P, minlength=k)
            assert np.array_equal(Ep.astype(np.int64), exp_E)
            assert np.array_equal(npng.astype(np.int64), exp_np)


def test_pagerank_all_active_always_pc():
    # (12 r + 4) E + 4k <= 2 (8 r E + 12 E + 4 V_a) whenever all of p is active, so Eq. (mode) picks PC
    for g in (gg.rmat(12), gg.uniform(5000, 20000)):
        for P in (64, 256, 1024):
            r = O.gpop(g, P, "pagerank", max_iters=3)
            Ep, _ = O.partition_stats(g, P)
            has_edges = Ep > 0
            assert np.all(r.modes[:, has_edges] == 2)
            assert np.all(r.modes[:, ~has_edges] == 0)


# --- Tier 2 engine (Alg. 2/3, Eq. (mode)) against Tier 1 ---------------------------------------

TIER2_GRAPHS = [gg.rmat(11), gg.uniform(1500, 9000), gg.star(70), gg.path(50),
                gg.disjoint_rings([3, 30, 7]),
                gg.multigraph(9, [0, 0, 0, 1, 2, 3, 3, 4, 5, 5, 7, 8], [1, 1, 2, 1, 3, 4, 4, 5, 0, 5, 8, 7])]


@pytest.mark.parametrize("g,P,policy", [(g, P, pol) for g in TIER2_GRAPHS for P in (1, 16, 256)
                                        for pol in ("analytic", "force_sc", "force_pc")],
                         ids=lambda v: getattr(v, "name", str(v)))
def test_tier2_matches_tier1(g, P, policy):
    roots = gg.roots(g, 2)
    # PageRank: same iteration, FP64, only summation order may differ
    xr, _, _ = O.pagerank(g, D, max_iters=12)
    r = O.gpop(g, P, "pagerank", max_iters=12, policy=policy)
    assert r.iterations == 12
    assert np.max(np.abs(r.values - xr) / xr) < 1e-12
    for s in roots:
        s = int(s)
        level, parent = O.bfs(g, s)
        r = O.gpop(g, P, "bfs", s, policy=policy)
        assert np.array_equal(r.level, level)
        par = parent.astype(np.uint64)
        par[parent == O.U32_INF] = O.U64_INF
        assert np.array_equal(r.values, par)
        gw = g.with_weights()
        r = O.gpop(gw, P, "sssp", s, policy=policy)
        assert np.array_equal(r.values, O.sssp(gw, s))
        xp, _, _ = O.ppr(g, s, 0.15, max_iters=40)
        r = O.gpop(g, P, "ppr", s, damping=0.85, max_iters=40, policy=policy)
        assert np.max(np.abs(r.values - xp)) < 1e-14
    gs = gg.symmetrized(g)
    r = O.gpop(gs, P, "cc", policy=policy)
    assert np.array_equal(r.values, O.cc(gs).astype(np.uint64))


def test_tier2_frontier_trace_is_bfs_layers():
    g = gg.rmat(12)
    s = int(gg.roots(g, 1)[0])
    level, _ = O.bfs(g, s)
    r = O.gpop(g, 64, "bfs", s)
    deg = np.diff(g.row_ptr)
    L = int(level[level != O.U32_INF].max())
    assert r.iterations == L + 1
    for t in range(r.iterations):
        layer = level == t
        assert r.frontier_vertices[t] == layer.sum()
        assert r.frontier_edges[t] == deg[layer].sum()


def test_tier2_pagerank_stops_on_residual():
    g = gg.rmat(10)
    x, it, res = O.pagerank(g, D, max_iters=500, tol=1e-9)
    r = O.gpop(g, 32, "pagerank", max_iters=500, tol=1e-9)
    assert r.iterations == it and r.residual < 1e-9
    assert np.max(np.abs(r.values - x) / x) < 1e-12
