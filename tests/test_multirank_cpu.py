"""World-size-2 gloo tests of the multi-process host logic (CPU only): the
max-over-ranks timing of the benchmark and the all-gather of exported sketch
images used for the cross-box OR-merge of Sec. 4.2 (equal sizes on every
rank, a mismatch reported on every rank), and a rank that dies before the
exchange."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1901_07306_gb300 import exchange
        t = exchange.reduce_max(10.0 * (rank + 1))
        imgs = exchange.all_gather_images(bytes([rank, 7]) * 500)
        try:
            exchange.all_gather_images(bytes([rank]) * (1000 + rank))
            mismatch = "no error"
        except ValueError:
            mismatch = "ValueError"
        q.put((rank, t, [len(x) for x in imgs], [x[:2] for x in imgs], mismatch))
    finally:
        dist.destroy_process_group()


def _dead_worker(rank, world, port, q):
    import torch.distributed as dist
    from datetime import timedelta
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=timedelta(seconds=5))
    if rank == 1:
        return                                      # a watch point that dies before the exchange
    from paper_1901_07306_gb300 import exchange
    try:
        exchange.all_gather_images(b"x" * 10)
        q.put((rank, "no error"))
    except Exception as e:                          # the survivor sees an error, not a hang
        q.put((rank, type(e).__name__))


def test_reduce_max_and_gather_images():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict((r, rest) for r, *rest in (q.get(timeout=120) for _ in procs))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        t, lens, heads, mismatch = out[r]
        assert t == 20.0
        assert lens == [1000, 1000] and heads == [b"\x00\x07", b"\x01\x07"]
        assert mismatch == "ValueError"


def test_dead_rank_surfaces_as_error():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_dead_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    rank, what = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
    assert rank == 0 and what != "no error"
