"""GPU parity of the sliding time window (Sec. 5): at every slice t the
context's window sketch (exported bits) and its detection list equal the
oracle's discrete sketch of the window's slices W(t, k) -- byte for byte."""
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


def dev(torch, pairs):
    flat = np.ascontiguousarray(pairs, np.uint32).reshape(-1).view(np.int32)
    return torch.from_numpy(flat.copy()).cuda()


def oparams(kw):
    keys = ("r", "isb", "ibn", "k_log2", "lr", "lc_log2", "theta", "seed")
    return O.Params(**{k: v for k, v in kw.items() if k in keys})


def same_sketch(ctx, osk, router=0):
    seav, ldca = ctx.sketch_image(router)
    return np.array_equal(seav, osk.seav) and np.array_equal(ldca, osk.ldca)


def test_window_equals_concatenation_every_slice(sp, torch):
    sizes = np.random.default_rng(4).integers(2000, 30000, 14)
    slices, sp_hosts, sched = W.sliding_stream(seed=4, sizes=sizes, n_sp=6, sp_degree_per_slice=(100, 400),
                                               n_background=3000)
    k = 4
    kw = dict(theta=256, seed=4, window_slices=k)
    op = oparams(kw)
    with sp.SuperPoint(**kw) as ctx:
        for t, sl in enumerate(slices):
            if t:
                ctx.slide()
            ctx.update(dev(torch, sl))
            got, n, rc = ctx.detect()
            osk = O.sliding_window_sketch(op, slices, t, k)
            assert same_sketch(ctx, osk), t
            want, n_want, _ = osk.detect()
            assert n == n_want and np.array_equal(got["ip"], want["ip"]) and np.array_equal(got["z0"], want["z0"])


def test_no_stamp_aliasing_past_255_slices(sp, torch):
    """Slice ids cycle through 255 values; the per-slide sweep must retire
    every stamp before its id comes back."""
    k = 3
    kw = dict(TINY, theta=16, seed=5, window_slices=k)
    op = oparams(kw)
    rng = np.random.default_rng(5)
    hosts = rng.integers(0, 2**32, 64, dtype=np.uint32)      # a small, recurring population
    slices = [np.stack([hosts[rng.integers(0, 64, 400)], rng.integers(0, 2**32, 400, dtype=np.uint32)], 1)
              for _ in range(300)]
    check = {0, 1, 2, 3, 100, 253, 254, 255, 256, 257, 299}
    with sp.SuperPoint(**kw) as ctx:
        for t, sl in enumerate(slices):
            if t:
                ctx.slide()
            if t % 7 != 3:                                     # some slices carry nothing
                ctx.update(dev(torch, sl))
            else:
                slices[t] = np.empty((0, 2), np.uint32)
            if t in check:
                assert same_sketch(ctx, O.sliding_window_sketch(op, slices, t, k)), t


def test_boundary_super_point_found_only_by_sliding(sp, torch):
    """Sec. 5.1: 900 + 900 peers across the boundary of two discrete windows
    of 4 slices: neither discrete window reports the host, the sliding
    window that straddles the boundary does (and both match the oracle)."""
    rng = np.random.default_rng(245)
    aip = 0xC0A80042
    per = [0, 0, 450, 450, 450, 450, 0, 0]
    slices = []
    for n in per:
        bg = W.uniform_pairs(20000, seed=int(rng.integers(1 << 30)), n_hosts=4000)
        own = np.stack([np.full(n, aip, np.uint32), rng.integers(0, 2**32, n, dtype=np.uint32)], 1)
        slices.append(np.concatenate([bg, own]))
    kw = dict(seed=245)
    op = oparams(kw)
    with sp.SuperPoint(**kw) as disc, sp.SuperPoint(**dict(kw, window_slices=4)) as slid:
        found_disc, found_slid = set(), {}
        for t, sl in enumerate(slices):
            if t:
                slid.slide()
            slid.update(dev(torch, sl))
            got, _, _ = slid.detect()
            want, _, _ = O.sliding_window_sketch(op, slices, t, 4).detect()
            assert np.array_equal(got["ip"], want["ip"])
            found_slid[t] = aip in set(got["ip"].tolist())
            disc.update(dev(torch, sl))
            if t % 4 == 3:                                     # end of a discrete window
                got, _, _ = disc.detect()
                want, _, _ = O.Sketch(op).update(O.window_pairs(slices, t, 4)).detect()
                assert np.array_equal(got["ip"], want["ip"])
                found_disc |= set(got["ip"].tolist())
                disc.slide()                                   # discrete: next window starts empty
        assert aip not in found_disc
        assert found_slid[5]


def test_sliding_merge_and_reset(sp, torch):
    k = 3
    kw = dict(TINY, theta=16, seed=9, window_slices=k, n_routers=3)
    op = oparams(kw)
    a = [W.uniform_pairs(3000, seed=100 + t, n_hosts=200) for t in range(6)]
    b = [W.uniform_pairs(2500, seed=200 + t, n_hosts=300) for t in range(6)]
    with sp.SuperPoint(**kw) as ctx:
        for t in range(6):
            if t:
                ctx.slide(0)
                ctx.slide(1)
                ctx.slide(2)
            ctx.update(dev(torch, a[t]), router=0)
            ctx.update(dev(torch, b[t]), router=1)
        ctx.merge([0, 1], 2)
        both = [np.concatenate([x, y]) for x, y in zip(a, b)]
        assert same_sketch(ctx, O.sliding_window_sketch(op, both, 5, k), router=2)
        ctx.slide(0)
        with pytest.raises(sp.SPError) as e:
            ctx.merge([0, 1], 2)                               # slice clocks differ
        assert e.value.code == sp.SP_ERR_STATE
        ctx.reset(1)
        ctx.update(dev(torch, a[0]), router=1)
        assert same_sketch(ctx, O.Sketch(op).update(a[0]), router=1)
        assert sp.sp_import(ctx.ctx, 1, sp.sp_export(ctx.ctx, 1)) == sp.SP_ERR_STATE


@pytest.mark.parametrize("scan_mode", [1, 2])
def test_every_update_form_mid_slice_reads(sp, torch, scan_mode):
    """The slice's bits reach the counters however they were scanned (direct
    or binned; device, host, batched or device-table updates), and a detect
    or an export in the middle of a slice commits what came so far without
    losing what comes after it in the same slice."""
    k = 3
    kw = dict(TINY, theta=16, seed=21, window_slices=k, n_routers=2, scan_mode=scan_mode)
    op = oparams(kw)
    rng = np.random.default_rng(21)
    parts = [[W.uniform_pairs(int(rng.integers(500, 4000)), seed=1000 + 10 * t + j, n_hosts=150)
              for j in range(4)] for t in range(7)]
    keep = []
    with sp.SuperPoint(**kw) as ctx:
        for t in range(7):
            if t:
                ctx.slide(0)
                ctx.slide(1)
            p = parts[t]
            form = t % 4
            if form == 0:
                ctx.update(dev(torch, p[0]))
                ctx.update_host(np.ascontiguousarray(p[1]))
            elif form == 1:
                bufs = [dev(torch, x) for x in p[:2]]
                sp.sp_update_batched(ctx.ctx, [0, 0], bufs)
                keep.append(bufs)
            elif form == 2:
                bufs = [dev(torch, x) for x in p[:2]]
                rec = np.zeros(2, sp.BATCH)
                rec[0] = (bufs[0].data_ptr(), len(p[0]), 0, 0)
                rec[1] = (bufs[1].data_ptr(), len(p[1]), 0, 0)
                table = torch.from_numpy(rec.view(np.uint8).copy()).cuda()
                sp.sp_update_batched_device(ctx.ctx, table, 2)
                keep.append((bufs, table))
            else:
                ctx.update(dev(torch, np.concatenate(p[:2])))
            # window so far: earlier slices whole, this slice's first two parts
            so_far = [np.concatenate(x[:4]) for x in parts[:t]] + [np.concatenate(p[:2])]
            osk = O.sliding_window_sketch(op, so_far, t, k)
            got, n, _ = ctx.detect()
            want, n_want, _ = osk.detect()
            assert n == n_want and np.array_equal(got["ip"], want["ip"]), t
            assert same_sketch(ctx, osk), t
            ctx.update(dev(torch, p[2]))
            ctx.update_host(np.ascontiguousarray(p[3]))
            whole = [np.concatenate(x[:4]) for x in parts[:t + 1]]
            assert same_sketch(ctx, O.sliding_window_sketch(op, whole, t, k)), t
            assert same_sketch(ctx, O.Sketch(op), router=1), t     # router 1 never received pairs
        torch.cuda.synchronize()


def test_per_slice_cuda_graph_replay(sp, torch):
    """Sec. 5 per-slice step recorded once as a CUDA graph -- slide, scan of
    the slice through a one-entry device batch table, detect -- and replayed
    slice after slice with the table rewritten: the slice clock lives on the
    device, so every replay advances the window, and the window's sketch and
    results equal the oracle's at every slice (past the window length, so
    slices also leave it)."""
    sizes = np.random.default_rng(71).integers(2000, 20000, 12)
    slices, sp_hosts, sched = W.sliding_stream(seed=71, sizes=sizes, n_sp=6, sp_degree_per_slice=(100, 400),
                                               n_background=3000)
    k = 4
    kw = dict(theta=256, seed=71, window_slices=k)
    op = oparams(kw)
    pool = [dev(torch, x) for x in slices]
    table = torch.zeros(sp.BATCH.itemsize, dtype=torch.uint8, device="cuda")

    def write_table(t):
        rec = np.zeros(1, sp.BATCH)
        rec[0] = (pool[t].data_ptr(), slices[t].shape[0], 0, 0)
        table.copy_(torch.from_numpy(rec.view(np.uint8)))

    def check(ctx, t):
        torch.cuda.synchronize()
        osk = O.sliding_window_sketch(op, slices, t, k)
        assert same_sketch(ctx, osk), t
        got, n, rc = sp.sp_results(ctx.ctx)
        want, n_want, _ = osk.detect()
        assert n == n_want and np.array_equal(got["ip"], want["ip"]) and np.array_equal(got["z0"], want["z0"]), t

    with sp.SuperPoint(**kw) as ctx:
        c = ctx.ctx
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):                    # slices 0 and 1 without a graph
            sp.sp_set_stream(c, side)
            for t in (0, 1):
                if t:
                    sp.sp_slide(c, 0)
                write_table(t)
                sp.sp_update_batched_device(c, table, 1)
                sp.sp_detect_async(c, 0, 0)
        torch.cuda.synchronize()
        sp.sp_set_stream(c, torch.cuda.current_stream())
        check(ctx, 1)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            sp.sp_set_stream(c, torch.cuda.current_stream())
            sp.sp_slide(c, 0)
            sp.sp_update_batched_device(c, table, 1)
            sp.sp_detect_async(c, 0, 0)
        sp.sp_set_stream(c, torch.cuda.current_stream())
        for t in range(2, len(slices)):
            write_table(t)
            g.replay()
            check(ctx, t)


def test_reset_range_in_a_sliding_context(sp, torch):
    """sp_reset_range on sliding routers forgets their slices and clocks
    (per router), leaving the others' windows intact."""
    kw = dict(TINY, theta=16, seed=81, window_slices=3, n_routers=3)
    op = oparams(kw)
    a = W.uniform_pairs(5000, seed=81, n_hosts=300)
    b = W.uniform_pairs(5000, seed=82, n_hosts=300)
    with sp.SuperPoint(**kw) as ctx:
        for r in range(3):
            ctx.update(dev(torch, a), router=r)
            ctx.slide(r)
            ctx.update(dev(torch, b), router=r)
        sp.sp_reset_range(ctx.ctx, 1, 2)
        assert same_sketch(ctx, O.Sketch(op).update(a).update(b), router=0)
        for r in (1, 2):
            seav, ldca = ctx.sketch_image(r)
            assert not seav.any() and not ldca.any(), r
        ctx.update(dev(torch, b), router=1)                     # slice 0 of a fresh window
        assert same_sketch(ctx, O.Sketch(op).update(b), router=1)
