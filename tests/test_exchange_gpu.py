"""The WP -> GS exchange of Sec. 4.2 through the library, checked against the
oracle of the union stream.

* host form: two processes (gloo ranks, both on the one GPU; their kernels
  never wait on each other) each scan their own watch point's stream, export
  the sketch, all-gather the images and OR them on the GPU; the global
  detection equals the oracle's detection of the concatenated streams.
* device form: sp_copy_sketch images gathered over a one-rank NCCL group
  (the code path of a multi-GPU run) and ORed with sp_merge_device, and
  directly between contexts; bit-exact against the oracle."""
import os
import socket

import numpy as np
import pytest

import oracle as O
from paper_1901_07306_gb300 import workloads as W

pytestmark = pytest.mark.gpu

KW = dict(theta=1024, seed=61)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _stream(rank):
    """A watch point's window: background, plus its half of the peers of 6
    global hosts with 1,600 peers each (800 per watch point: below theta on
    each, a super point in the union)."""
    pairs, _ = W.single_window(seed=60 + rank, n=1 << 19, n_background=8192, n_planted=0)
    hosts = W.uniform_pairs(6, seed=70)[:, 0]
    glob = np.stack([np.repeat(hosts, 1600), W.uniform_pairs(6 * 1600, seed=71)[:, 1]], 1).astype(np.uint32)
    return np.ascontiguousarray(np.concatenate([pairs, glob[rank::2]]))


def _rank_main(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1901_07306_gb300 import build
        build.build()
        from paper_1901_07306_gb300 import exchange, sp
        with sp.SuperPoint(n_routers=1 + world + 1, **KW) as ctx:
            flat = torch.from_numpy(_stream(rank).reshape(-1).view(np.int32).copy()).cuda()
            ctx.update(flat, router=0)
            images = exchange.all_gather_images(sp.sp_export(ctx.ctx, 0))
            gs = world + 1                                        # routers 1 .. world hold the images
            rc = exchange.merge_remote_images(sp, ctx.ctx, images, 1, gs)
            recs, n, drc = ctx.detect(router=gs)
            seav, ldca = ctx.sketch_image(gs)
            q.put((rank, rc, drc, recs["ip"].tolist(), recs["z0"].tolist(), seav.tobytes(), ldca.tobytes()))
    finally:
        dist.destroy_process_group()


def test_host_form_two_ranks_on_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict((r, rest) for r, *rest in (q.get(timeout=300) for _ in procs))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    union = np.concatenate([_stream(0), _stream(1)])
    osk = O.Sketch(O.Params(**KW)).update(union)
    want, n_want, _ = osk.detect()
    assert n_want > 0
    for r in range(2):
        rc, drc, ips, z0, seav, ldca = out[r]
        assert rc == 0 and drc == 0
        assert seav == osk.seav.tobytes() and ldca == osk.ldca.tobytes()
        assert ips == want["ip"].tolist() and z0 == want["z0"].tolist()


@pytest.fixture(scope="module")
def sp():
    from paper_1901_07306_gb300 import build
    build.build()
    from paper_1901_07306_gb300 import sp as mod
    return mod


def test_device_form_between_contexts(sp):
    import torch
    from paper_1901_07306_gb300 import exchange
    streams = [_stream(r) for r in range(3)]
    ctxs = [sp.SuperPoint(scan_mode=m, **KW) for m in (1, 2, 2)]    # direct and binned (pending planes) scans
    gs = sp.SuperPoint(n_routers=2, **KW)
    try:
        for c, x in zip(ctxs, streams):
            c.update(torch.from_numpy(x.reshape(-1).view(np.int32).copy()).cuda())
        n = sp.sp_copy_sketch_bytes(gs.ctx)
        imgs = torch.empty((3, n), dtype=torch.uint8, device="cuda")
        for i, c in enumerate(ctxs):
            sp.sp_copy_sketch(c.ctx, 0, imgs[i])
        torch.cuda.synchronize()
        gs.update(torch.from_numpy(streams[0].reshape(-1).view(np.int32).copy()).cuda(), router=1)
        exchange.merge_gathered(sp, gs.ctx, imgs, 1, skip=(0,))   # router 1 already holds stream 0
        osk = O.Sketch(O.Params(**KW)).update(np.concatenate(streams))
        seav, ldca = gs.sketch_image(1)
        assert np.array_equal(seav, osk.seav) and np.array_equal(ldca, osk.ldca)
        got, n_got, rc = gs.detect(router=1)
        want, n_want, _ = osk.detect()
        assert rc == sp.SP_OK and n_got == n_want and np.array_equal(got["ip"], want["ip"])
        with pytest.raises(sp.SPError):
            sp.sp_merge_device(gs.ctx, [imgs[0][1:]], 1)             # misaligned image
    finally:
        for c in ctxs + [gs]:
            c.close()


def _nccl_one_rank(port, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    os.environ["NCCL_NVLS_ENABLE"] = "0"
    torch.cuda.set_device(0)
    dist.init_process_group("nccl", rank=0, world_size=1, device_id=torch.device("cuda", 0))
    try:
        from paper_1901_07306_gb300 import exchange, sp
        with sp.SuperPoint(n_routers=2, **KW) as ctx:
            ctx.update(torch.from_numpy(_stream(0).reshape(-1).view(np.int32).copy()).cuda(), router=0)
            gathered = exchange.all_gather_sketches(sp, ctx.ctx, 0)
            exchange.merge_gathered(sp, ctx.ctx, gathered, 1)
            recs, n, rc = ctx.detect(router=1)
            seav, ldca = ctx.sketch_image(1)
            q.put((tuple(gathered.shape), rc, recs["ip"].tolist(), seav.tobytes(), ldca.tobytes()))
    finally:
        dist.destroy_process_group()


def test_device_form_over_nccl_one_rank(sp):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    p = ctx.Process(target=_nccl_one_rank, args=(_free_port(), q))
    p.start()
    shape, rc, ips, seav, ldca = q.get(timeout=300)
    p.join(timeout=120)
    assert p.exitcode == 0
    osk = O.Sketch(O.Params(**KW)).update(_stream(0))
    want, _, _ = osk.detect()
    assert shape[0] == 1 and rc == 0
    assert seav == osk.seav.tobytes() and ldca == osk.ldca.tobytes() and ips == want["ip"].tolist()
