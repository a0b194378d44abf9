"""Host logic of the multi-process bench path, on CPU with two gloo ranks: the timed region's
max-over-ranks reduction, and the reference arm running on rank 0 only.  (Replicas only: the path
has no data exchange, so the only collective is this reduction of a timing.)"""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        got = bench.max_over_ranks(dist, 10.0 + 5.0 * rank)
        bench.barrier(dist)
        q.put((rank, got))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=5) for _ in range(2))
    assert res == [(0, 15.0), (1, 15.0)]


def _ref_worker(rank, world, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import contextlib
    import io
    import json
    import sys
    import bench
    sys.argv = ["bench.py", "--impl", "reference", "--gpus", str(world), "--steps", "1", "--warmup", "0", "--size", "small"]
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        rc = bench.main()
    lines = [json.loads(x) for x in buf.getvalue().splitlines() if x.startswith("{")]
    q.put((rank, rc, lines))


def test_reference_arm_runs_on_rank0_only():
    """Under torchrun every rank starts bench.py --impl reference: rank 0 times the oracle and prints
    the one JSON line; the others exit 0 without work."""
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_ref_worker, args=(r, 2, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(600)
        assert p.exitcode == 0
    res = dict((r, (rc, lines)) for r, rc, lines in (q.get(timeout=5) for _ in range(2)))
    assert res[1] == (0, [])
    rc0, lines0 = res[0]
    assert rc0 == 0 and len(lines0) == 1
    line = lines0[0]
    assert line["impl"] == "reference" and line["unit"] == "beam-steps/s" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0
