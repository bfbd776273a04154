"""The N > 1 path of bench.py on the host: two ranks over gloo on the CPU
(the GPU runs here use one GPU). Each rank evaluates its own parameter
points; the only collectives are the barrier and the max over ranks of the
timed interval; rank 0 alone reports, and alone runs the reference arm."""
import importlib.util
import os
import socket

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import io
    import contextlib
    import torch.distributed as dist
    bench = _bench()
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        bench.barrier(world)
        m = bench.max_over_ranks(0.25 + rank, world)
        g, b = bench.angle_sets(3, bench.rank_seed(rank))
        seen = [None] * world
        dist.all_gather_object(seen, (g.tolist(), b.tolist()))
        buf = io.StringIO()

        class A:
            gpus, steps, warmup = world, 1, 0
        with contextlib.redirect_stdout(buf):
            if rank != 0:  # the reference arm does no work off rank 0
                bench.run_reference(A, rank, world)
        out[rank] = (m, seen, buf.getvalue())
    finally:
        dist.destroy_process_group()


def test_two_ranks_over_gloo():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    world, port = 2, _free_port()
    manager = mp.get_context("spawn").Manager()
    out = manager.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    assert set(out.keys()) == {0, 1}
    for r in range(world):
        m, seen, printed = out[r]
        assert m == 1.25  # max over ranks of 0.25 + rank
        (g0, b0), (g1, b1) = seen
        assert not np.allclose(g0, g1) and not np.allclose(b0, b1)  # disjoint parameter points
    assert out[1][2] == ""  # nothing printed by rank 1
    bench = _bench()
    assert bench.whole_job_rate(2, 10, 0.5) == 40.0
