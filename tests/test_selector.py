"""Learned SC/PC selector: the FP64 CPU reference is pinned by finite differences (no GPU); the GPU forward /
backward kernels match it within FP32 tolerance; training reduces the loss; the learned policy leaves every
application's result unchanged (both modes compute the same answer, Sec. 3.2)."""
import numpy as np
import pytest

import graphgen as gg
import oracle as O
from oracle import mlp

RNG = np.random.default_rng(1234)


def random_problem(n=300, seed=0):
    rng = np.random.default_rng(seed)
    w = rng.normal(0, 0.4, mlp.NW)
    X = rng.normal(0, 1, (n, 8))
    Y = np.sin(X[:, 0]) + 0.5 * X[:, 1] * X[:, 2] - X[:, 7]
    return w, X, Y


def test_cpu_backprop_matches_central_differences():
    w, X, Y = random_problem(40)
    g = mlp.grad(w, X, Y)
    h = 1e-6
    idx = list(range(0, mlp.NW, 7)) + [mlp.NW - 1]
    for i in idx:
        e = np.zeros(mlp.NW)
        e[i] = h
        fd = (mlp.loss(w + e, X, Y) - mlp.loss(w - e, X, Y)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), i


def test_cpu_forward_linear_regime_closed_form():
    # with all pre-activations positive the network is affine: y = W3 (W2 (W1 x + b1) + b2) + b3
    rng = np.random.default_rng(3)
    W1 = np.abs(rng.normal(size=(32, 8)))
    W2 = np.abs(rng.normal(size=(32, 32)))
    W3 = rng.normal(size=32)
    b1, b2, b3 = np.ones(32), np.ones(32), 0.25
    w = np.concatenate([W1.ravel(), b1, W2.ravel(), b2, W3, [b3]])
    X = np.abs(rng.normal(size=(5, 8)))
    expect = ((X @ W1.T + b1) @ W2.T + b2) @ W3 + b3
    assert np.allclose(mlp.forward(w, X), expect, rtol=1e-13)


def test_cpu_grad_detects_dropped_bias_term():
    # planted mistake: dropping b2's gradient would fail the finite-difference pin on those coordinates
    w, X, Y = random_problem(30, seed=5)
    g = mlp.grad(w, X, Y)
    i = 32 * 8 + 32 + 32 * 32 + 3  # a b2 coordinate
    h = 1e-6
    e = np.zeros(mlp.NW)
    e[i] = h
    fd = (mlp.loss(w + e, X, Y) - mlp.loss(w - e, X, Y)) / (2 * h)
    assert abs(fd) > 1e-4 and abs(fd - g[i]) < 1e-6 * max(1, abs(fd))


torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def gp():
    import paper_1806_08092_gb300 as gp
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gp.build()
    return gp


@pytest.mark.gpu
def test_gpu_gradient_matches_fp64_reference(gp):
    for n in (1, 63, 64, 65, 1000):
        w, X, Y = random_problem(n, seed=n)
        w32, X32, Y32 = w.astype(np.float32), X.astype(np.float32), Y.astype(np.float32)
        pred, g, loss = gp.selector_grad(w32, X32, Y32)
        ref_pred = mlp.forward(w32.astype(np.float64), X32.astype(np.float64))
        ref_g = mlp.grad(w32.astype(np.float64), X32.astype(np.float64), Y32.astype(np.float64))
        assert np.max(np.abs(pred - ref_pred)) <= 1e-4 * max(1.0, np.max(np.abs(ref_pred)))
        scale = np.max(np.abs(ref_g))
        assert np.max(np.abs(g - ref_g)) <= 1e-4 * scale, n
        assert loss == pytest.approx(mlp.loss(w32, X32, Y32), rel=1e-4)


@pytest.mark.gpu
def test_gpu_training_reduces_loss_and_is_deterministic(gp):
    rng = np.random.default_rng(7)
    X = rng.normal(0, 1, (2000, 8)).astype(np.float32)
    Y = (np.tanh(X[:, 0] - 0.5 * X[:, 3]) + 0.3 * X[:, 5]).astype(np.float32)
    p1, l1 = gp.selector_train(X, Y, epochs=600, lr=3e-3, seed=11)
    p2, l2 = gp.selector_train(X, Y, epochs=600, lr=3e-3, seed=11)
    assert np.array_equal(p1, p2) and l1 == l2
    base = float(np.var(Y))
    assert l1 < 0.1 * base
    # the stored statistics standardise the features the way the reference does
    mean, sd = p1[mlp.NW:mlp.NW + 8], p1[mlp.NW + 8:mlp.NW + 16]
    Z = (X - mean) / sd
    assert mlp.loss(p1[:mlp.NW].astype(np.float64), Z, Y) == pytest.approx(l1, rel=1e-3)


@pytest.mark.gpu
def test_learned_mode_leaves_results_unchanged(gp):
    # any selector output only changes how messages travel, never what the gather computes
    g = gg.rmat(13).with_weights()
    rng = np.random.default_rng(2)
    params = np.zeros(gp.SELECTOR_PARAMS, dtype=np.float32)
    params[:mlp.NW] = rng.normal(0, 0.5, mlp.NW)
    params[mlp.NW + 8:mlp.NW + 16] = 1.0                 # std
    params[mlp.NW + 16:mlp.NW + 24] = -1e30              # fmin
    params[mlp.NW + 24:mlp.NW + 32] = 1e30               # fmax
    gp.selector_set(params)
    try:
        G = gp.Graph.from_csr(g.row_ptr, g.col, g.weights, partition_size=128)
        for root in gg.roots(g, 2):
            root = int(root)
            level, parent = O.bfs(g, root)
            r = G.run("bfs", source=root, mode="learned", trace=True)
            assert np.array_equal(r.values.cpu().numpy(), level)
            assert np.array_equal(r.parent.cpu().numpy(), parent)
            d = O.sssp(g, root)
            r2 = G.run("sssp", source=root, mode="learned")
            dd = d.copy()
            dd[d == O.U64_INF] = O.U32_INF
            assert np.array_equal(r2.values.cpu().numpy(), dd.astype(np.uint32))
        x = G.run("pagerank", max_iters=8, mode="learned").values.cpu().numpy()
        ref = O.pagerank(g, 0.85, max_iters=8)[0]
        assert np.max(np.abs(x - ref) / ref) <= 1e-5
        got = gp.selector_get()
        assert np.array_equal(got, params)
    finally:
        gp.selector_set(None)


@pytest.mark.gpu
def test_learned_policy_with_a_network_equal_to_the_model(gp):
    # hand-set network whose output is feature 7 (the log of Eq. (mode)'s cost ratio) through off-diagonal
    # weights: h1_0 = relu(f7), h1_1 = relu(-f7), h2_2 = relu(h1_0), h2_5 = relu(h1_1), y = h2_2 - h2_5; the
    # learned policy must then pick Eq. (mode)'s modes in every iteration (a misplaced weight would not)
    W1 = np.zeros((32, 8)); W1[0, 7], W1[1, 7] = 1.0, -1.0
    W2 = np.zeros((32, 32)); W2[2, 0], W2[5, 1] = 1.0, 1.0
    W3 = np.zeros(32); W3[2], W3[5] = 1.0, -1.0
    params = np.zeros(gp.SELECTOR_PARAMS, dtype=np.float32)
    params[:mlp.NW] = np.concatenate([W1.ravel(), np.zeros(32), W2.ravel(), np.zeros(32), W3, [0.0]])
    params[mlp.NW + 8:mlp.NW + 16] = 1.0                 # std (mean 0)
    params[mlp.NW + 16:mlp.NW + 24] = -1e30              # fmin
    params[mlp.NW + 24:mlp.NW + 32] = 1e30               # fmax
    g = gg.rmat(15).with_weights()
    G = gp.Graph.from_csr(g.row_ptr, g.col, g.weights, partition_size=256)
    gp.selector_set(params)
    try:
        for root in gg.roots(g, 2):
            for algo in ("bfs", "sssp"):
                a = G.run(algo, source=int(root), trace=True)
                b = G.run(algo, source=int(root), mode="learned", trace=True)
                assert np.array_equal(a.modes, b.modes), algo
                assert b.stats["pc_partition_steps"] + b.stats["sc_partition_steps"] > 0
    finally:
        gp.selector_set(None)


def features_np(Va, Ea, Ep, npng, k, row_bins, num=2, den=1):
    """Selector features in float64 (the engine computes the same quantities in FP32/FP64 on the device)."""
    cpc = 4.0 * (3 * npng + k + Ep) * den
    csc = 4.0 * (Va + 3.0 * Ea + 2.0 * (npng / Ep) * Ea) * num
    return np.stack([np.log1p(Va), np.log1p(Ea), np.log1p(Ep), npng / Ep, np.log1p(row_bins), np.log1p(npng),
                     np.log1p(np.full_like(Va, k)), np.log(cpc / csc)], axis=1)


def regret(choose_pc, t_pc, t_sc):
    return float(np.sum(np.where(choose_pc, t_pc, t_sc) - np.minimum(t_pc, t_sc)))


@pytest.mark.gpu
def test_trained_selector_beats_the_model_when_bandwidths_differ(gp):
    # planted truth: PC streams at 4x the SC bandwidth (Eq. (mode) assumes 2x), so Eq. (mode) sends a band
    # of partitions to SC that PC would finish sooner; the trained MLP must recover that boundary
    rng = np.random.default_rng(21)
    n = 6000
    Ep = rng.integers(1000, 200000, n).astype(np.float64)
    r = rng.uniform(0.3, 1.0, n)
    npng = np.floor(r * Ep)
    Ea = np.floor(Ep * rng.uniform(0.0005, 1.0, n) ** 2)
    Ea = np.maximum(Ea, 1)
    Va = np.maximum(np.floor(Ea / 16), 1)
    k, rb = 1024, np.minimum(npng, 1024)
    t_pc = 4.0 * (3 * npng + k + Ep) / 4.0
    t_sc = 4.0 * (Va + 3 * Ea + 2 * r * Ea) / 1.0
    X = features_np(Va, Ea, Ep, npng, k, rb).astype(np.float32)
    Y = np.log(t_pc / t_sc).astype(np.float32)
    tr, te = slice(0, 4000), slice(4000, n)
    params, loss = gp.selector_train(X[tr], Y[tr], epochs=1500, lr=3e-3, seed=5)
    mean, sd = params[mlp.NW:mlp.NW + 8], params[mlp.NW + 8:mlp.NW + 16]
    pred = mlp.forward(params[:mlp.NW].astype(np.float64), (X[te] - mean) / sd)
    mlp_regret = regret(pred <= 0, t_pc[te], t_sc[te])
    model_regret = regret(X[te, 7] <= 0, t_pc[te], t_sc[te])
    assert model_regret > 0
    assert mlp_regret < 0.25 * model_regret, (mlp_regret, model_regret)


@pytest.mark.gpu
def test_log_both_records_and_results(gp):
    g = gg.rmat(14).with_weights()
    G = gp.Graph.from_csr(g.row_ptr, g.col, g.weights, partition_size=256)
    root = int(gg.roots(g, 1)[0])
    r = G.run("bfs", source=root, mode="log_both", log_capacity=100000, trace=True)
    level, parent = O.bfs(g, root)
    assert np.array_equal(r.values.cpu().numpy(), level)
    assert np.array_equal(r.parent.cpu().numpy(), parent)
    log = r.log
    n_sc, n_pc = (r.modes == 1).sum(), (r.modes == 2).sum()
    assert log.shape == (n_sc + n_pc, gp.LOG_RECORD_FLOATS)
    assert np.all(log[:, 8] > 0) and np.all(log[:, 9] > 0)
    # the logged chosen mode is Eq. (mode)'s, and the features agree with the host-side formulas
    Ep, npng = O.partition_stats(g, 256)
    for rec in log[:50]:
        q, it = int(rec[11]), int(rec[12])
        assert r.modes[it - 1, q] == int(rec[10])
        assert rec[2] == pytest.approx(np.log1p(Ep[q]), rel=1e-5)
        assert rec[3] == pytest.approx(npng[q] / Ep[q], rel=1e-5)
