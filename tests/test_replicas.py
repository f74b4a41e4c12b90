"""Multi-GPU form on the host: replicas only (instances and simulations are
independent; a rank exchanges nothing but its timings and unit counts).
world_size 2 over gloo on 127.0.0.1, no GPU: the bench's rank set-up, barrier,
max-over-ranks timing and summed unit counts, and the reference arm, which
only rank 0 runs."""
from __future__ import annotations

import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as tmp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    w, r, local = bench.dist_setup()
    bench.init_ranks(w, local, backend="gloo")
    bench.barrier(w)
    mx = bench.max_over_ranks(1.5 + r, w)            # the job's time is the slowest rank's
    sm = bench.sum_over_ranks(10.0 * (r + 1), w)     # the job's units are every rank's
    # reference arm: rank 0 alone prints its line, the other rank returns at once
    args = type("A", (), dict(workload="c0", frames=None, warmup=0, steps=1, gpus=w))()
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(args, w, r)
    bench.barrier(w)
    dist.destroy_process_group()
    out.put((r, mx, sm, buf.getvalue()))


def test_two_replicas_over_gloo():
    world = 2
    port = _free_port()
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(world):
        r, mx, sm, text = q.get(timeout=240)
        res[r] = (mx, sm, text)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0][0] == res[1][0] == 2.5
    assert res[0][1] == res[1][1] == 30.0
    assert res[1][2] == ""                              # rank 1 ran no reference work
    line = json.loads(res[0][2].strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
