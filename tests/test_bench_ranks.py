"""Host logic of bench.py's multi-replica path on CPU: two gloo ranks, max of times, sum of counted edges."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, e = bench.reduce_over_ranks(1.5 + rank, 1e9 * (rank + 1), dist, "cpu")
    out[rank] = (t, e)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_reduction():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        for r in range(2):
            assert out[r] == (2.5, 3e9)


def test_single_rank_passthrough():
    import bench
    assert bench.reduce_over_ranks(2.0, 5.0, None, "cpu") == (2.0, 5.0)


def test_engine_code_sha_ignores_comments_only(tmp_path):
    import bench
    a = tmp_path / "a.cu"
    a.write_text("// header\n__global__ void k(int *x) {\n    x[0] = 1;  // set\n}\n")
    b = tmp_path / "b.cu"
    b.write_text("/* another\n   header */\n\n__global__ void k(int *x) {\n      x[0] = 1;\n}\n")
    c = tmp_path / "c.cu"
    c.write_text("__global__ void k(int *x) {\n    x[0] = 2;\n}\n")
    assert bench.engine_code_sha(str(a)) == bench.engine_code_sha(str(b))
    assert bench.engine_code_sha(str(a)) != bench.engine_code_sha(str(c))

