"""Host logic of the partition-size autotuner on CPU: a stand-in Graph with fixed device times."""
import pytest

from paper_1806_08092_gb300 import GpopError
from paper_1806_08092_gb300 import autotune


class _FakeRun:
    def __init__(self, ms):
        self.stats = {"device_ms": ms}


class _FakeGraph:
    times = {}
    closed = []

    def __init__(self, P):
        self.P = P

    @classmethod
    def from_csr(cls, row_ptr, col, weights, partition_size):
        if partition_size not in cls.times:
            raise GpopError(1, "partition_size must be a power of two in [32, 16384]")
        return cls(partition_size)

    def run(self, algo, **kw):
        t = self.times[self.P][algo]
        if t is None:
            raise GpopError(2, "run buffers: out of memory")
        return _FakeRun(t)

    def close(self):
        self.closed.append(self.P)


def test_picks_the_fastest_and_lists_rejected(monkeypatch):
    _FakeGraph.times = {1024: {"bfs": 3.0, "sssp": 9.0}, 4096: {"bfs": 2.0, "sssp": 7.5}, 16384: {"bfs": 2.5, "sssp": 7.4}}
    _FakeGraph.closed = []
    monkeypatch.setattr(autotune, "Graph", _FakeGraph)
    best, table = autotune.pick_partition_size(None, None, None, runs=[("bfs", {}), ("sssp", {})],
                                               candidates=(1024, 3000, 4096, 16384), reps=3)
    assert best == 4096  # 9.5 ms against 12.0 and 9.9
    assert [(r[0], r[1]) for r in table] == [(1024, 12.0), (3000, None), (4096, 9.5), (16384, 9.9)]
    assert "power of two" in table[1][3]
    assert _FakeGraph.closed == [1024, 4096, 16384]  # every built layout is released


def test_no_candidate_raises(monkeypatch):
    _FakeGraph.times = {}
    monkeypatch.setattr(autotune, "Graph", _FakeGraph)
    with pytest.raises(ValueError):
        autotune.pick_partition_size(None, None, None, candidates=(3000,))


def test_a_candidate_whose_runs_fail_is_listed_and_skipped(monkeypatch):
    _FakeGraph.times = {2048: {"bfs": 3.0}, 16384: {"bfs": None}}
    _FakeGraph.closed = []
    monkeypatch.setattr(autotune, "Graph", _FakeGraph)
    best, table = autotune.pick_partition_size(None, None, None, runs=[("bfs", {})], candidates=(2048, 16384))
    assert best == 2048
    assert table[1][0] == 16384 and table[1][1] is None and "out of memory" in table[1][3]
    assert _FakeGraph.closed == [2048, 16384]  # the failing layout is released too


class _FakeRatioGraph:
    """A built graph whose run time depends on the bandwidth ratio (U-shaped, minimum at 8)."""
    def __init__(self):
        self.calls = []

    def run(self, algo, bw_ratio=(2, 1), **kw):
        self.calls.append((algo, bw_ratio))
        r = bw_ratio[0] / bw_ratio[1]
        if r == 0:
            raise GpopError(1, "bandwidth ratio must be positive")
        return _FakeRun({"bfs": 1.0, "sssp": 3.0}[algo] * (1.0 + abs(__import__("math").log2(r / 8.0)) / 4))


def test_bw_ratio_picks_the_fastest_and_lists_rejected():
    G = _FakeRatioGraph()
    best, table = autotune.pick_bw_ratio(G, runs=[("bfs", {}), ("sssp", {})], candidates=(0, 2, 8, 32), reps=3)
    assert best == (8, 1)
    assert table[0][0] == 0 and table[0][1] is None and "positive" in table[0][2]
    assert [t[0] for t in table[1:]] == [2, 8, 32] and table[2][1] == 4.0
    # every candidate's runs are timed at its own ratio: one warm-up + reps per run
    assert G.calls.count(("bfs", (8, 1))) == 4 and G.calls.count(("sssp", (32, 1))) == 4
