"""Host logic of the multi-GPU bench (replicas only): world_size-2 ranks over
gloo on the CPU -- barrier, max-over-ranks timing, whole-job throughput, and
the reference arm's rank-0-only output."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    bench.barrier(world)
    local_ms = 10.0 + 5.0 * rank
    worst = bench.max_over_ranks(local_ms, world)
    value = bench.PRODUCTS * world / (worst / 1e3)

    class A:
        steps, warmup, gpus = 1, 0, world

    buf = io.StringIO()
    called = []
    bench.oracle_setup = lambda: called.append(rank) or None
    bench.oracle_step = lambda st: 1.0
    with redirect_stdout(buf):
        bench.run_reference(A, world, rank)
    q.put((rank, worst, value, buf.getvalue(), called))
    dist.destroy_process_group()


def test_two_rank_max_and_rank0_output():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, v0, out0, c0), (r1, w1, v1, out1, c1) = res
    assert w0 == w1 == 15.0                     # both ranks see the slowest rank's time
    assert v0 == v1 == pytest.approx(2 * 32 / 0.015)
    assert '"impl": "reference"' in out0 and out1 == ""   # only rank 0 runs and prints the reference arm
    assert c0 == [0] and c1 == []
