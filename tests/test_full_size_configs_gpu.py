"""Bit-exact parity with the oracle at the full sizes of the distributed,
sliding-window and serving workloads.

* distributed (Sec. 4.2): 16 routers x 2^24 pairs from an overlapping host
  population, 64 uneven batches per router in one sp_update_batched call
  (binned rounds per router), OR-merge into a global router, detect; profile
  D3 (r = 16, LC = 2^18).  Every router's sketch, the merged sketch and the
  result list equal the oracle's.
* sliding window (Sec. 5): 2^28 pairs in 128 lognormal slices of 2^19-2^22
  pairs, window of 32 slices advanced one slice at a time.  The window's
  sketch and result list at slices 31, 64, 127 and at the slice whose window
  holds the most super points equal the oracle's discrete sketch of the
  window's 32 slices.
* serving: 64 routers, batches of 2^12-2^22 pairs (log-uniform), arriving all
  at once, a detect every 2^24 global pairs.  Every window equals the oracle
  and the plain one-launch-per-batch path, and some routers receive at least
  2^22 pairs in one engine step (the binned form inside the batched call).

The oracle sketches of large streams are built in shards on all host cores
and OR-merged, which equals the sketch of the whole stream (Sec. 4.2; the
oracle's merge = concatenation pin)."""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle as O
from paper_1901_07306_gb300 import workloads as W

pytestmark = pytest.mark.gpu

D3 = dict(r=16, isb=(0, 4, 8, 12), ibn=(7, 7, 7, 7), lc_log2=18)
PROFILE_S = dict(r=12, isb=(0, 5, 10, 15), ibn=(7, 7, 7, 7), lc_log2=14)
THREADS = max(1, min(16, os.cpu_count() or 1))


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
    return torch.from_numpy(flat).cuda()


def oracle_sketch(params, pairs):
    """The oracle's sketch of a large stream: shards on every host core,
    OR-merged (equal to the sketch of the whole stream)."""
    pairs = np.ascontiguousarray(pairs, np.uint32).reshape(-1, 2)
    bounds = np.linspace(0, pairs.shape[0], THREADS + 1).astype(np.int64)
    with ThreadPoolExecutor(THREADS) as ex:
        parts = list(ex.map(lambda t: O.Sketch(params).update(pairs[bounds[t]:bounds[t + 1]]), range(THREADS)))
    out = parts[0]
    for s in parts[1:]:
        out.merge(s)
    return out


def assert_same_sketch(ctx, osk, router):
    seav, ldca = ctx.sketch_image(router)
    assert np.array_equal(seav, osk.seav), f"SEAV of router {router}"
    assert np.array_equal(ldca, osk.ldca), f"LDCA of router {router}"


def assert_same_results(got, want):
    assert len(got) == len(want)
    for f in ("ip", "z0", "flags"):
        assert np.array_equal(got[f], want[f]), f
    assert np.array_equal(got["est"].view(np.uint64), want["est"].view(np.uint64))


def test_distributed_16_routers_full_size(sp, torch):
    n_routers, per = 16, 1 << 24
    routers, sp_hosts = W.distributed(seed=3, n_per_router=per)
    rng = np.random.default_rng(3)
    flats = [dev(torch, pr) for pr in routers]
    batches = []
    for r, pr in enumerate(routers):
        w = np.exp(rng.uniform(0, np.log(16.0), 64))
        cuts = np.floor(np.cumsum(w / w.sum())[:-1] * pr.shape[0]).astype(np.int64)
        bounds = [0, *cuts.tolist(), pr.shape[0]]
        for a, b in zip(bounds[:-1], bounds[1:]):
            batches.append((r, flats[r][2 * a:2 * b]))
    batches = [batches[i] for i in rng.permutation(len(batches))]
    kw = dict(theta=1024, seed=3, n_routers=n_routers + 1, **D3)
    op = oparams(kw)
    with sp.SuperPoint(**kw) as ctx:
        sp.sp_update_batched(ctx.ctx, [r for r, _ in batches], [t for _, t in batches])
        with ThreadPoolExecutor(THREADS) as ex:
            osks = list(ex.map(lambda x: O.Sketch(op).update(x), routers))
        for r in range(n_routers):
            assert_same_sketch(ctx, osks[r], r)
        sp.sp_merge(ctx.ctx, list(range(n_routers)), n_routers)
        merged = osks[0].copy()
        for s in osks[1:]:
            merged.merge(s)
        assert_same_sketch(ctx, merged, n_routers)
        got, n, rc = ctx.detect(router=n_routers)
        want, n_want, overflow = merged.detect()
        assert rc == sp.SP_OK and not overflow and n == n_want
        assert_same_results(got, want)
        assert set(sp_hosts.tolist()) <= set(got["ip"].tolist())   # every global super point


def test_sliding_2e28_pairs_window_32(sp, torch):
    k = 32
    sizes = W.slice_sizes(4, n_slices=128, total=1 << 28, lo=1 << 19, hi=1 << 22)
    slices, sp_hosts, sched = W.sliding_stream(seed=4, sizes=sizes, n_sp=64, sp_degree_per_slice=(64, 512))
    assert sum(x.shape[0] for x in slices) == 1 << 28
    dslices = [dev(torch, x) for x in slices]
    kw = dict(theta=1024, seed=4, window_slices=k)
    op = oparams(kw)
    checkpoints = (31, 64, 127)
    seen = {}

    def run_to(ctx, last, keep):
        ctx.reset()
        counts = []
        for t in range(last + 1):
            if t:
                ctx.slide()
            ctx.update(dslices[t])
            recs, n, rc = ctx.detect()
            assert rc == sp.SP_OK, (t, rc)
            counts.append(n)
            if t in keep:
                seen[t] = (ctx.sketch_image(), recs)
        return counts

    with sp.SuperPoint(**kw) as ctx:
        counts = run_to(ctx, len(slices) - 1, checkpoints)
        busiest = int(np.argmax(counts))
        if busiest not in seen:                   # a second pass, stopped at the busiest window
            run_to(ctx, busiest, (busiest,))
    for t in sorted(seen):
        (seav, ldca), recs = seen[t]
        osk = oracle_sketch(op, O.window_pairs(slices, t, k))
        assert np.array_equal(seav, osk.seav) and np.array_equal(ldca, osk.ldca), f"window sketch at slice {t}"
        want, n_want, overflow = osk.detect()
        assert not overflow and counts[t] == n_want, t
        assert_same_results(recs, want)


def test_serving_64_routers_full_size(sp, torch):
    from paper_1901_07306_gb300 import serving as S
    n_routers = 64
    heavy = W.uniform_pairs(64, seed=55)[:, 0]            # 64 hosts that talk to many peers everywhere

    def stream(router, n, seed):
        """Uniform background; 2% of the pairs come from the heavy hosts."""
        rng = np.random.default_rng(seed)
        pairs = W.uniform_pairs(n, seed=seed, n_hosts=max(1, n // 4))
        m = n // 50
        pairs[:m, 0] = heavy[rng.integers(0, heavy.size, m)]
        return pairs

    reqs = S.poisson_requests(5, n_routers, 200, rate_pairs_per_s=1e13, lo_log2=12, hi_log2=22, streams=stream)
    kw = dict(PROFILE_S, theta=1024, seed=5)
    op = oparams(kw)

    def serve(batched, steps=None):
        rs = [S.Request(router=r.router, pairs=r.pairs, arrival=0.0) for r in reqs]   # all at once
        srv = S.SketchServer(n_routers, kw, budget_bytes=2 << 30, detect_every=1 << 24, batched=batched)
        if steps is not None:
            issue = srv.ops.issue_step
            srv.ops.issue_step = lambda step: (steps.append(step), issue(step))[1]
        try:
            wins = srv.run(rs)
        finally:
            srv.close()
        return rs, wins

    steps = []
    rb, wb = serve(True, steps)
    rp, wp = serve(False)
    assert [r.window for r in rb] == [r.window for r in rp]
    biggest = max(max(np.bincount([r.router for r in st], weights=[r.n_pairs for r in st])) for st in steps)
    assert biggest >= 1 << 22                     # some router took the binned form inside a batched step
    assert len(wb) == len(wp) >= 6
    assert all(w.n_found >= 32 for w in wb[:-1])          # the heavy hosts are found in every full window
    for a, b in zip(wb, wp):
        assert a.n_found == b.n_found and np.array_equal(a.records, b.records), a.index
    for w in wb:
        mine = [r.pairs.numpy().view(np.uint32).reshape(-1, 2) for r in rb if r.window == w.index]
        want, n_want, overflow = oracle_sketch(op, np.concatenate(mine)).detect()
        assert not overflow and w.n_found == n_want, w.index
        assert_same_results(w.records, want[:len(w.records)])
