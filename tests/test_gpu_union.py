"""Many graphs of uneven size as one disjoint union (gpop_graph_build_union, gpop_run_bfs_union).

Each graph's BFS levels from its own source, read out of the union's batched traversal, must equal the
oracle's queue BFS on that graph alone, bit for bit; any other application run on the union must give,
on each graph's vertices, the results of that graph alone.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gp():
    import paper_1806_08092_gb300 as gp
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gp.build()
    return gp


def uneven_graphs(count, scales, efs, seed):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        s, ef = int(rng.choice(scales)), int(rng.choice(efs))
        g = gg.rmat(s, ef) if i % 5 else gg.uniform(1 << s, ef << s, seed=1000 + i)
        out.append(g.with_weights())
    return out


@pytest.mark.parametrize("P", [64, 1024])
def test_union_bfs_equals_each_graph_alone(gp, P):
    gs = uneven_graphs(45, scales=(5, 6, 7, 8, 9, 10, 11), efs=(2, 4, 8, 16), seed=P)  # 45 graphs: two passes
    gs.append(gg.path(7).with_weights())  # and a path with an unreachable-free tail and a ring
    gs.append(gg.ring(33).with_weights())
    G = gp.Graph.from_many([(g.row_ptr, g.col, g.weights) for g in gs], partition_size=P)
    off = G.union_offsets()
    assert len(off) == len(gs) + 1 and off[-1] == sum(g.num_vertices for g in gs)
    src = [int(gg.roots(g, 1)[0]) for g in gs]
    r = G.run_bfs_union(src)
    lv = r.values.cpu().numpy()
    for i, g in enumerate(gs):
        assert np.array_equal(lv[off[i]:off[i + 1]], O.bfs(g, src[i])[0]), i
    # the union is an ordinary graph: SSSP and CC on it restricted to a graph equal that graph's own results
    for i in (0, 7, len(gs) - 1):
        d = O.sssp(gs[i], src[i])
        d32 = d.copy()
        d32[d == O.U64_INF] = O.U32_INF
        x = G.run("sssp", source=int(off[i]) + src[i]).values.cpu().numpy()[off[i]:off[i + 1]]
        assert np.array_equal(x, d32.astype(np.uint32)), i
    G.close()


def test_union_errors(gp):
    g0, g1 = gg.rmat(6), gg.rmat(7)
    G = gp.Graph.from_many([(g0.row_ptr, g0.col), (g1.row_ptr, g1.col)], partition_size=32)
    with pytest.raises(gp.GpopError, match="source out of its graph"):
        G.run_bfs_union([0, g1.num_vertices])  # graph 1's source must be one of its own vertices
    plain = gp.Graph.from_csr(g0.row_ptr, g0.col, partition_size=32)
    assert len(plain.union_offsets()) == 0
    with pytest.raises(gp.GpopError, match="union"):
        plain.run_bfs_union([0])
    G.close()
    plain.close()
