"""The multi-rank host logic of bench.py on CPU: two gloo ranks (world size
2, 127.0.0.1) take the maximum of their timings, aggregate the whole job's
throughput from the slowest rank, reconstruct different frames, and only
rank 0 of the reference arm produces output."""
import importlib.util
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    b = _bench()
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, wsz, _ = b.dist_env()
    ms = b.max_over_ranks(dist, [10.0 + 5.0 * rank, 100.0 - rank])
    from paper_1904_04884_gb300 import workloads
    w = workloads.TINY
    frame = b.rank_hologram(np.zeros((w.ny, w.nx), np.float32), w, rank)

    class Args:
        gpus, steps, warmup = world, 1, 0
    buf = io.StringIO()
    if rank == 1:                     # the reference arm: non-zero ranks do no work
        with redirect_stdout(buf):
            b.run_reference(Args, rank, world)
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, r, wsz, ms, float(np.abs(frame).sum()), buf.getvalue()))


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, r, wsz, ms, frame_abs, text in res:
        assert r == rank and wsz == 2
        assert ms == [15.0, 100.0]                     # max over ranks, element-wise
    assert res[0][4] == 0.0 and res[1][4] > 0.0        # rank 1 solves its own frame
    assert res[1][5] == ""                             # rank 1 of the reference arm is silent


def test_job_value_is_weak_scaling():
    b = _bench()
    one = b.job_value(1e6, 5, 1, 1000.0)
    assert b.job_value(1e6, 5, 2, 1000.0) == 2 * one
    assert b.job_value(1e6, 5, 2, 2000.0) == one
