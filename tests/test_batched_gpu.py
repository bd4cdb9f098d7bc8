"""GPU parity of the batched scan: many routers' batches of uneven size in
one call (and one persistent launch), against the oracle's per-router
sketches; the device-table form captured in a CUDA graph and replayed with a
rewritten table; the autotuner."""
import ctypes

import numpy as np
import pytest

import oracle as O
from paper_1901_07306_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TINY = dict(r=12, isb=(0, 7, 14), ibn=(8, 8, 8), k_log2=8, lr=3, lc_log2=6)


@pytest.fixture(scope="module")
def sp():
    from paper_1901_07306_gb300 import build
    build.build()
    from paper_1901_07306_gb300 import sp as mod
    return mod


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available()
    return t


def oparams(kw):
    keys = ("r", "isb", "ibn", "k_log2", "lr", "lc_log2", "theta", "seed")
    return O.Params(**{k: v for k, v in kw.items() if k in keys})


def dev(torch, pairs):
    flat = np.ascontiguousarray(pairs, np.uint32).reshape(-1).view(np.int32)
    return torch.from_numpy(flat.copy()).cuda()


def same_sketch(ctx, osk, router):
    seav, ldca = ctx.sketch_image(router)
    return np.array_equal(seav, osk.seav) and np.array_equal(ldca, osk.ldca)


def _batches(seed, n_routers, n_batches, lo_log2, hi_log2):
    rng = np.random.default_rng(seed)
    routers = rng.integers(0, n_routers, n_batches).tolist()
    sizes = np.exp(rng.uniform(np.log(2.0**lo_log2), np.log(2.0**hi_log2), n_batches)).astype(int)
    sizes[rng.integers(0, n_batches)] = 0                      # an empty batch
    data = [W.uniform_pairs(int(n), seed=seed * 1000 + i, n_hosts=max(1, int(n) // 8)) for i, n in enumerate(sizes)]
    return routers, data


@pytest.mark.parametrize("kw", [dict(TINY, theta=16), dict(theta=256)])
def test_batched_small_batches_one_launch(sp, torch, kw):
    kw = dict(kw, seed=11, n_routers=6)
    routers, data = _batches(11, 6, 40, 4, 16)
    with sp.SuperPoint(**kw) as ctx:
        tensors = [dev(torch, x) for x in data]
        sp.sp_update_batched(ctx.ctx, routers, tensors)
        op = oparams(kw)
        for r in range(6):
            mine = [x for rr, x in zip(routers, data) if rr == r]
            want = O.Sketch(op).update(np.concatenate(mine) if mine else np.empty((0, 2), np.uint32))
            assert same_sketch(ctx, want, r), r


def test_batched_mixes_binned_and_direct_routers(sp, torch):
    """Router 2 receives more than 2^22 pairs over three batches (binned
    rounds); the other routers' small batches share the persistent launch."""
    kw = dict(theta=256, seed=12, n_routers=4)
    rng = np.random.default_rng(12)
    big = [W.uniform_pairs(n, seed=120 + i, n_hosts=50000) for i, n in enumerate((1 << 21, 1 << 21, 300001))]
    small = [W.uniform_pairs(int(n), seed=130 + i, n_hosts=500) for i, n in enumerate(rng.integers(100, 5000, 9))]
    routers = [2, 0, 2, 1, 3, 2, 0, 1, 3, 0, 1, 3]
    data = [big[0], small[0], big[1], small[1], small[2], big[2]] + small[3:]
    with sp.SuperPoint(**kw) as ctx:
        tensors = [dev(torch, x) for x in data]
        sp.sp_update_batched(ctx.ctx, routers, tensors)
        op = oparams(kw)
        for r in range(4):
            mine = np.concatenate([x for rr, x in zip(routers, data) if rr == r])
            osk = O.Sketch(op).update(mine)
            assert same_sketch(ctx, osk, r), r
        got, n, rc = ctx.detect(router=2)
        want, _, _ = O.Sketch(op).update(np.concatenate(big)).detect()
        assert np.array_equal(got["ip"], want["ip"]) and np.array_equal(got["z0"], want["z0"])


def test_device_table_graph_replay(sp, torch):
    """One CUDA graph = reset + batched scan from a device table + detect.
    Replayed after rewriting the table (other streams, other sizes, other
    routers), every replay matches the oracle."""
    kw = dict(TINY, theta=16, seed=13, n_routers=3)
    op = oparams(kw)
    pool = [dev(torch, W.uniform_pairs(20000, seed=140 + i, n_hosts=400)) for i in range(6)]
    host_pool = [p.cpu().numpy().view(np.uint32).reshape(-1, 2) for p in pool]
    table = torch.zeros(8 * sp.BATCH.itemsize, dtype=torch.uint8, device="cuda")

    def write_table(entries):
        rec = np.zeros(8, sp.BATCH)
        for i, (k, n, r) in enumerate(entries):
            rec[i] = (pool[k].data_ptr(), n, r, 0)
        table.copy_(torch.from_numpy(rec.view(np.uint8)))

    with sp.SuperPoint(**kw) as ctx:
        write_table([(0, 100, 0)] * 8)
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):            # warm up: allocations happen before capture
            sp.sp_set_stream(ctx.ctx, side)
            for r in range(3):
                sp.sp_reset(ctx.ctx, r)
            sp.sp_update_batched_device(ctx.ctx, table, 8)
            sp.sp_detect_async(ctx.ctx, 1, 0)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            sp.sp_set_stream(ctx.ctx, torch.cuda.current_stream())
            for r in range(3):
                sp.sp_reset(ctx.ctx, r)
            sp.sp_update_batched_device(ctx.ctx, table, 8)
            sp.sp_detect_async(ctx.ctx, 1, 0)
        sp.sp_set_stream(ctx.ctx, torch.cuda.current_stream())
        rng = np.random.default_rng(13)
        for replay in range(3):
            entries = [(int(rng.integers(0, 6)), int(rng.integers(0, 20001)), int(rng.integers(0, 3)))
                       for _ in range(8)]
            write_table(entries)
            g.replay()
            torch.cuda.synchronize()
            for r in range(3):
                mine = [host_pool[k][:n] for k, n, rr in entries if rr == r]
                osk = O.Sketch(op).update(np.concatenate(mine) if mine else np.empty((0, 2), np.uint32))
                assert same_sketch(ctx, osk, r), (replay, r)
            recs, n, rc = sp.sp_results(ctx.ctx)
            mine = [host_pool[k][:n_] for k, n_, rr in entries if rr == 1]
            want, _, _ = O.Sketch(op).update(np.concatenate(mine) if mine else np.empty((0, 2), np.uint32)).detect()
            assert np.array_equal(recs["ip"], want["ip"]) and np.array_equal(recs["z0"], want["z0"])


def test_device_table_bad_router_is_reported(sp, torch):
    kw = dict(TINY, theta=16, seed=14, n_routers=2)
    pairs = W.uniform_pairs(5000, seed=14, n_hosts=100)
    buf = dev(torch, pairs)
    rec = np.zeros(2, sp.BATCH)
    rec[0] = (buf.data_ptr(), 5000, 7, 0)                    # router out of range
    rec[1] = (buf.data_ptr(), 5000, 1, 0)
    table = torch.from_numpy(rec.view(np.uint8).copy()).cuda()
    with sp.SuperPoint(**kw) as ctx:
        sp.sp_update_batched_device(ctx.ctx, table, 2)
        sp.sp_detect_async(ctx.ctx, 0, 0)
        with pytest.raises(sp.SPError) as e:
            sp.sp_results(ctx.ctx)
        assert e.value.code == sp.SP_ERR_ROUTER
        assert same_sketch(ctx, O.Sketch(oparams(kw)).update(pairs), 1)


def test_autotune_then_scan(sp, torch):
    kw = dict(theta=256, seed=15, n_routers=2)
    sample = dev(torch, W.uniform_pairs(1 << 20, seed=15, n_hosts=1 << 16))
    with sp.SuperPoint(**kw) as ctx:
        threads, blocks = sp.sp_autotune(ctx.ctx, sample)
        assert threads in (128, 256, 512) and 1 <= blocks <= 2048 // threads
        seav, ldca = ctx.sketch_image(0)
        assert not seav.any() and not ldca.any()              # the tuner left router 0 empty
        routers, data = _batches(15, 2, 12, 6, 15)
        sp.sp_update_batched(ctx.ctx, routers, [dev(torch, x) for x in data])
        for r in range(2):
            mine = [x for rr, x in zip(routers, data) if rr == r]
            assert same_sketch(ctx, O.Sketch(oparams(kw)).update(np.concatenate(mine)), r)


def test_many_batches_of_one_router_binned(sp, torch):
    """40 batches of one router (> 2^22 pairs in total): two binning launches
    of up to 32 streams each append to the same lists; one stream starts 8
    bytes off a 16-byte boundary (plain loads inside a TMA launch)."""
    kw = dict(theta=256, seed=16, n_routers=2, scan_mode=0)
    rng = np.random.default_rng(16)
    sizes = rng.integers(60000, 180000, 40)
    data = [W.uniform_pairs(int(n), seed=160 + i, n_hosts=20000) for i, n in enumerate(sizes)]
    assert sum(sizes) >= (1 << 22)
    tensors = [dev(torch, x) for x in data]
    raw = torch.empty(2 * int(sizes[7]) + 2, dtype=torch.int32, device="cuda")
    raw[2:].copy_(tensors[7])
    tensors[7] = raw[2:]                                        # 8-byte aligned only
    assert tensors[7].data_ptr() % 16 == 8
    with sp.SuperPoint(**kw) as ctx:
        sp.sp_update_batched(ctx.ctx, [1] * 40, tensors)
        osk = O.Sketch(oparams(kw)).update(np.concatenate(data))
        assert same_sketch(ctx, osk, 1)
        seav, ldca = ctx.sketch_image(0)
        assert not seav.any() and not ldca.any()


@pytest.mark.parametrize("n_batches,lo,hi", [(2048, 4096, 4096), (3000, 500, 6000)])
def test_thousands_of_small_batches_of_one_router(sp, torch, n_batches, lo, hi):
    """Thousands of small batches of one router in one call (> 2^22 pairs in
    total, so the router takes the binned rounds): the rounds must stay
    within the allocated list capacity whatever the number of binning
    launches they need, and the sketch and result list stay bit-exact."""
    kw = dict(theta=1024, seed=17, n_routers=2, scan_mode=0)
    rng = np.random.default_rng(17)
    sizes = rng.integers(lo, hi + 1, n_batches)
    assert sizes.sum() >= (1 << 22)
    pairs, planted = W.single_window(seed=17, n=int(sizes.sum()), n_background=1 << 17, n_planted=8,
                                     planted_degree=3000)
    flat = dev(torch, pairs)
    cuts = np.concatenate([[0], np.cumsum(sizes)])
    tensors = [flat[2 * int(a):2 * int(b)] for a, b in zip(cuts[:-1], cuts[1:])]
    with sp.SuperPoint(**kw) as ctx:
        sp.sp_update_batched(ctx.ctx, [1] * n_batches, tensors)
        osk = O.Sketch(oparams(kw)).update(pairs)
        assert same_sketch(ctx, osk, 1)
        got, n, rc = ctx.detect(router=1)
        want, n_want, _ = osk.detect()
        assert rc == sp.SP_OK and n == n_want
        assert np.array_equal(got["ip"], want["ip"]) and np.array_equal(got["z0"], want["z0"])
        assert set(planted.tolist()) <= set(got["ip"].tolist())


def test_batched_host_copies_into_arena(sp, torch):
    """sp_update_batched_host: host batches (pinned, uneven sizes, odd pair
    counts) copied into a caller arena on a copy stream and scanned in one
    call; every router's sketch equals the oracle's; an arena too small is
    refused before anything is copied."""
    kw = dict(theta=256, seed=18, n_routers=3)
    routers, data = _batches(18, 3, 30, 3, 15)
    host = [torch.from_numpy(np.ascontiguousarray(x, np.uint32).reshape(-1).view(np.int32).copy()).pin_memory()
            for x in data]
    words = sum((h.numel() + 3) // 4 * 4 for h in host)
    arena = torch.empty(words, dtype=torch.int32, device="cuda")
    copy = torch.cuda.Stream()
    with sp.SuperPoint(**kw) as ctx:
        with pytest.raises(sp.SPError) as e:
            sp.sp_update_batched_host(ctx.ctx, routers, host, arena[: words - 4], copy)
        assert e.value.code == sp.SP_ERR_PARAM
        sp.sp_update_batched_host(ctx.ctx, routers, host, arena, copy)
        for r in range(3):
            mine = [x for rr, x in zip(routers, data) if rr == r]
            assert same_sketch(ctx, O.Sketch(oparams(kw)).update(np.concatenate(mine)), r), r


def test_reserve_then_batched_and_host_updates(sp, torch):
    """sp_reserve allocates up front what updates would allocate on first use;
    afterwards the batched scan (binned and direct routers, then a call with
    more batches than a reserved table holds, which grows a used table) and
    the host path give the oracle's sketches.  A range outside the context is
    refused."""
    kw = dict(theta=256, seed=19, n_routers=4)
    big = [W.uniform_pairs(n, seed=190 + i, n_hosts=50000) for i, n in enumerate((1 << 21, (1 << 21) + 7))]
    small = [W.uniform_pairs(64 + 3 * i, seed=200 + i, n_hosts=40) for i in range(1500)]
    with sp.SuperPoint(**kw) as ctx:
        with pytest.raises(sp.SPError) as e:
            sp.sp_reserve(ctx.ctx, 2, 3)
        assert e.value.code == sp.SP_ERR_ROUTER
        sp.sp_reserve(ctx.ctx, 0, 0)                       # no router: only the shared buffers
        sp.sp_reserve(ctx.ctx)
        sp.sp_reserve(ctx.ctx)                             # idempotent
        sp.sp_update_batched(ctx.ctx, [1, 0, 1], [dev(torch, big[0]), dev(torch, small[0]), dev(torch, big[1])])
        sp.sp_update_batched(ctx.ctx, [2] * len(small), [dev(torch, x) for x in small])
        host = torch.from_numpy(np.ascontiguousarray(big[0], np.uint32).reshape(-1).view(np.int32).copy()).pin_memory()
        sp.sp_update_host(ctx.ctx, 3, host)
        op = oparams(kw)
        want = {0: small[0], 1: np.concatenate(big), 2: np.concatenate(small), 3: big[0]}
        for r, pairs in want.items():
            assert same_sketch(ctx, O.Sketch(op).update(pairs), r), r
