"""sp_detect_noalloc: detect with no device allocation, for callers that may
not allocate at that point (device memory owned by another allocator or
budgeted up front, latency-critical loops).  Its output must equal the
context-based sp_detect on the same sketch, bit for bit, call after call:
the scratch array it shares across calls keeps the previous contents, so a
stale status or a wrong estimate table would show up on a later call.

This file is collected last so that a failure here leaves every other test
already run."""
import ctypes

import numpy as np
import pytest

from paper_1901_07306_gb300 import workloads as W

pytestmark = pytest.mark.gpu


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


def _sketch_and_reference(sp, torch, seed, n_planted, threshold, **kw):
    """A sketch built through a context, its sp_detect output, and device
    copies of its SEAV/LDCA in the exported layout."""
    pairs, planted = W.single_window(seed=seed, n=1 << 18, n_background=16384, n_planted=n_planted,
                                     planted_degree=2500)
    params = sp.make_params(seed=seed, **kw)
    with sp.SuperPoint(params) as ctx:
        flat = torch.from_numpy(pairs.reshape(-1).view(np.int32).copy()).cuda()
        ctx.update(flat)
        want, n, rc = ctx.detect(threshold=threshold)
        assert rc == sp.SP_OK
        seav, ldca = ctx.sketch_image()
    dseav = torch.from_numpy(seav).cuda()
    dldca = torch.from_numpy(ldca.view(np.int32)).cuda()
    return params, dseav, dldca, want, n


def _noalloc(sp, torch, params, dseav, dldca, threshold, cap):
    out = torch.zeros(max(cap, 1) * sp.CANDIDATE.itemsize, dtype=torch.uint8, device="cuda")
    status = torch.full((2,), -1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = sp.lib.sp_detect_noalloc(ctypes.byref(params), dseav.data_ptr(), dldca.data_ptr(), threshold,
                                  out.data_ptr(), cap, status.data_ptr(), stream)
    torch.cuda.synchronize()
    count, flags = (int(x) for x in status.cpu().numpy().view(np.uint32))
    recs = out.cpu().numpy().view(sp.CANDIDATE)[:min(count, cap)]
    return rc, count, flags, recs


def _same(got, want):
    assert len(got) == len(want)
    for f in ("ip", "z0", "flags"):
        assert np.array_equal(got[f], want[f]), f
    assert np.array_equal(got["est"].view(np.uint64), want["est"].view(np.uint64))


def test_noalloc_detect_matches_context_detect_twice(sp, torch):
    a = _sketch_and_reference(sp, torch, seed=21, n_planted=12, threshold=1024)
    b = _sketch_and_reference(sp, torch, seed=22, n_planted=3, threshold=2000)
    # first call: many results; second call: another sketch with fewer, so
    # leftovers of the first call in the shared scratch would be visible
    for (params, dseav, dldca, want, n), thr in ((a, 1024), (b, 2000)):
        rc, count, flags, recs = _noalloc(sp, torch, params, dseav, dldca, thr, sp.SP_NOALLOC_MAX_RESULTS)
        assert rc == sp.SP_OK and flags == 0
        assert count == n
        _same(recs, want)


def test_noalloc_limits_and_overflow(sp, torch):
    params, dseav, dldca, want, n = _sketch_and_reference(sp, torch, seed=23, n_planted=10, threshold=1024)
    rc, *_ = _noalloc(sp, torch, params, dseav, dldca, 0, sp.SP_NOALLOC_MAX_RESULTS + 1)
    assert rc == sp.SP_ERR_PARAM
    big_k = sp.make_params(seed=23, k_log2=13, lc_log2=10)
    rc, *_ = _noalloc(sp, torch, big_k, dseav, dldca, 0, 16)
    assert rc == sp.SP_ERR_PARAM
    # a cap below the count: flag 1, count still exact, records a subset
    rc, count, flags, recs = _noalloc(sp, torch, params, dseav, dldca, 0, 4)
    assert rc == sp.SP_OK and count == n and flags & 1 and len(recs) == 4
    assert set(recs["ip"].tolist()) <= set(want["ip"].tolist())


def test_noalloc_estimate_table_of_each_k(sp, torch):
    """The estimate tables of every supported k live side by side in the
    shared array; calls with k = 256, 4096 and 1024 in a row each read their
    own table (the est bits are compared, so a wrong table offset fails)."""
    cases = [dict(k_log2=8, lc_log2=16), dict(k_log2=12, lc_log2=14), dict()]
    for i, kw in enumerate(cases):
        params, dseav, dldca, want, n = _sketch_and_reference(sp, torch, seed=31 + i, n_planted=6,
                                                              threshold=1024, **kw)
        rc, count, flags, recs = _noalloc(sp, torch, params, dseav, dldca, 1024, sp.SP_NOALLOC_MAX_RESULTS)
        assert rc == sp.SP_OK and flags == 0 and count == n, kw
        _same(recs, want)


def test_noalloc_sort_beyond_one_block(sp, torch):
    """About 20,000 results: the sort merges runs of 8,192 keys across the
    grid, using the caller's output records as its second buffer (nothing
    allocated); the list equals the context's, bit for bit."""
    rng = np.random.default_rng(53)
    hosts = rng.permutation(np.unique(rng.integers(0, 2**32, 26000, dtype=np.uint32))[:20000])
    pairs = np.stack([np.repeat(hosts, 64), rng.integers(0, 2**32, hosts.size * 64, dtype=np.uint32)], 1)
    params = sp.make_params(r=16, isb=(0, 8), ibn=(9, 9), theta=32, seed=53)
    with sp.SuperPoint(params) as ctx:
        ctx.update(torch.from_numpy(np.ascontiguousarray(pairs).reshape(-1).view(np.int32).copy()).cuda())
        want, n, rc = ctx.detect()
        assert rc == sp.SP_OK and n > 8192
        seav, ldca = ctx.sketch_image()
    dseav = torch.from_numpy(seav).cuda()
    dldca = torch.from_numpy(ldca.view(np.int32)).cuda()
    for _ in range(2):
        rc, count, flags, recs = _noalloc(sp, torch, params, dseav, dldca, 0, sp.SP_NOALLOC_MAX_RESULTS)
        assert rc == sp.SP_OK and flags == 0 and count == n
        _same(recs, want)
