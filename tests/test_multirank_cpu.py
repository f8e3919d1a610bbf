"""The multi-rank host logic of bench.py on CPU: two gloo ranks (one process
each), weak scaling with no data-path collective -- only the max-over-ranks
reduction of the step time and the whole-job value."""
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


def _rank_main(rank, world, port, ms, out):
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        bench.rank_barrier()
        m = bench.max_over_ranks(ms[rank], "cpu")
        out[rank] = (m, bench.weak_value(8192, world, m))
        bench.rank_barrier()
    finally:
        dist.destroy_process_group()


def test_weak_scaling_takes_the_slowest_rank():
    world, port = 2, _free_port()
    ms = [5.5, 6.25]
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_rank_main, args=(world, port, ms, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        m, v = res[r]
        assert m == max(ms)
        assert v == pytest.approx(8192 * world / (max(ms) * 1e-3))


def test_single_process_needs_no_group():
    import bench
    assert not (dist.is_available() and dist.is_initialized())
    assert bench.max_over_ranks(3.0, "cpu") == 3.0
    bench.rank_barrier()
    assert bench.weak_value(100, 1, 2.0) == pytest.approx(5e4)
