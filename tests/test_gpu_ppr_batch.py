"""Batched seeded PPR (gpop_run_ppr_batch) against the FP64 oracle, seed by seed.

Every row of a batch must match the oracle's PPR vector of its seed after the same number of iterations:
L-inf relative error <= 1e-5 on the oracle's support and absolute <= 1e-12 elsewhere (the tolerance of
the single-seed application).  Passes of 32 seeds, ragged last passes, repeated seeds, the tolerance
stop, host output, and the argument errors.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PR_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def gp():
    import paper_1806_08092_gb300 as gp
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gp.build()
    return gp


def check_rows(g, seeds, vals, iters, alpha=0.15):
    for j, s in enumerate(seeds):
        ref, _, _ = O.ppr(g, int(s), alpha, max_iters=iters)
        x = vals[j].astype(np.float64)
        sup = ref > 0
        err = float(np.max(np.abs(x[sup] - ref[sup]) / ref[sup]))
        assert err <= PR_TOL, (j, int(s), err)
        assert np.all(np.abs(x[~sup]) <= 1e-12), (j, int(s))


SMALL = [("ring", gg.ring(100)), ("star", gg.star(200)), ("rings", gg.disjoint_rings([33, 1, 64, 7])),
         ("uniform_ragged", gg.uniform(3001, 20000)), ("sparse_sinks", gg.uniform(2500, 3000)),
         ("rmat13", gg.rmat(13))]


@pytest.mark.parametrize("name,g", SMALL, ids=[s[0] for s in SMALL])
@pytest.mark.parametrize("P", [32, 1024])
def test_ppr_batch_matches_oracle_per_seed(gp, name, g, P):
    G = gp.Graph.from_csr(g.row_ptr, g.col, partition_size=P)
    # 37 seeds: a full pass of 32 and a ragged pass of 5, with one seed repeated across the passes
    seeds = list(gg.roots(g, 36)) if g.num_vertices > 40 else [int(i) % g.num_vertices for i in range(36)]
    seeds = [int(s) for s in seeds] + [int(seeds[3])]
    r = G.run_ppr_batch(seeds, max_iters=30)
    assert r.stats["iterations"] == 60  # two passes of 30
    vals = r.values.cpu().numpy()
    check_rows(g, seeds, vals, 30)
    assert np.array_equal(vals[3], vals[36])  # the repeated seed, in another pass: the same vector
    G.close()


def test_ppr_batch_equals_single_seed_runs_and_tolerance(gp):
    g = gg.rmat(14)
    G = gp.Graph.from_csr(g.row_ptr, g.col, partition_size=512)
    seeds = [int(s) for s in gg.roots(g, 8)]
    r = G.run_ppr_batch(seeds, max_iters=200, tol=1e-10)
    assert r.stats["converged"] == 1 and r.stats["residual"] < 1e-10
    it = r.stats["iterations"]
    vals = r.values.cpu().numpy()
    # every seed ran the pass's iteration count: its oracle vector at that count
    check_rows(g, seeds, vals, it)
    # and the single-seed engine after the same count agrees within FP32 rounding
    for j, s in enumerate(seeds[:3]):
        x1 = G.run("ppr", source=s, max_iters=it).values.cpu().numpy().astype(np.float64)
        sup = x1 > 0
        assert np.array_equal(sup, vals[j] > 0)
        assert np.max(np.abs(vals[j][sup] - x1[sup]) / x1[sup]) <= 2 * PR_TOL
    # host output gives the same rows
    h = G.run_ppr_batch(seeds[:5], max_iters=it, device_out=False).values
    assert isinstance(h, np.ndarray) and np.array_equal(h, G.run_ppr_batch(seeds[:5], max_iters=it).values.cpu().numpy())
    G.close()


def test_ppr_batch_errors(gp):
    g = gg.rmat(12)
    big = gp.Graph.from_csr(g.row_ptr, g.col, partition_size=2048)
    with pytest.raises(gp.GpopError, match="1024"):
        big.run_ppr_batch([0, 1], max_iters=3)
    big.close()
    G = gp.Graph.from_csr(g.row_ptr, g.col, partition_size=256)
    with pytest.raises(gp.GpopError, match="seed out of range"):
        G.run_ppr_batch([0, g.num_vertices], max_iters=3)
    with pytest.raises(gp.GpopError, match="damping"):
        G.run_ppr_batch([0], damping=1.0, max_iters=3)
    r = G.run_ppr_batch([], max_iters=3)
    assert r.stats["iterations"] == 0 and tuple(r.values.shape) == (0, g.num_vertices)
    G.close()
