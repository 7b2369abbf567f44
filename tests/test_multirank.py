"""Host logic of the benchmark's N > 1 path, on CPU with two gloo ranks.

With N GPUs every rank solves its own problem instance (replicas; the method has
no data-path exchange): the ranks draw different seeded inputs, and the reported
whole-job throughput is the flops of all ranks over the slowest rank's time.
"""
import hashlib
import os
import socket

import pytest
import torch.multiprocessing as mp

WL = dict(n=24, spec="uniform:1:10", beta=0.3, nev=4, nex=2)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _digest(*arrays) -> str:
    h = hashlib.sha256()
    for a in arrays:
        h.update(a.tobytes())
    return h.hexdigest()


def _worker(rank: int, world: int, port: int, q) -> None:
    import torch.distributed as dist

    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r reports (r + 1) TFLOP over (r + 1) x 100 ms
        v = bench.whole_job_tflops(dist, (rank + 1) * 1e12, (rank + 1) * 100.0, "cpu")
        m = bench.reduce_scalar(dist, float(rank), "max", "cpu")
        s = bench.reduce_scalar(dist, float(rank + 1), "sum", "cpu")
        A, B, _, W0, V0, w = bench.make_inputs(WL, rank)
        A2, B2, _, W02, V02, w2 = bench.make_inputs(WL, rank)
        q.put((rank, v, m, s, _digest(A, B, W0, V0, w), _digest(A2, B2, W02, V02, w2)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_and_draw_independent_replicas():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    try:
        for _ in range(2):
            rank, v, m, s, d1, d2 = q.get(timeout=120)
            out[rank] = (v, m, s, d1, d2)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert all(p.exitcode == 0 for p in procs)
    assert sorted(out) == [0, 1]
    for rank in (0, 1):
        v, m, s, d1, d2 = out[rank]
        # (1 + 2) TFLOP over the slowest rank's 0.2 s
        assert v == pytest.approx(15.0, rel=1e-12)
        assert m == 1.0 and s == 3.0
        assert d1 == d2  # seeded: the same inputs on a second draw
    assert out[0][3] != out[1][3]  # replicas: each rank its own problem


def test_single_process_reduction_is_identity():
    import bench

    assert bench.reduce_scalar(None, 2.5, "max", "cpu") == 2.5
    assert bench.whole_job_tflops(None, 3e12, 200.0, "cpu") == pytest.approx(15.0, rel=1e-12)
