"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Sketches (SEAV bytes, LDCA words) and detection lists (ip, z0, est, flags,
in order) must be bit-identical: the scheme is integer-only up to the
estimate, and the estimate comes from the same libm on both sides.
"""
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


def dev(torch, pairs, offset_pairs=0):
    """Pairs on the GPU as int32; offset_pairs > 0 shifts the start by whole
    pairs (8 bytes) to exercise the unaligned-head path."""
    flat = np.ascontiguousarray(pairs, np.uint32).reshape(-1).view(np.int32)
    buf = torch.empty(flat.size + 2 * offset_pairs + 4, dtype=torch.int32, device="cuda")
    buf[2 * offset_pairs:2 * offset_pairs + flat.size].copy_(torch.from_numpy(flat))
    return buf[2 * offset_pairs:2 * offset_pairs + flat.size]


_CORE = {}


def _core_link():
    if "pairs" not in _CORE:
        _CORE["pairs"] = W.core_link(seed=2)
    return _CORE["pairs"]


def oracle_params(kw):
    keys = ("r", "isb", "ibn", "k_log2", "lr", "lc_log2", "theta", "seed")
    return O.Params(**{k: v for k, v in kw.items() if k in keys})


def assert_same_sketch(ctx, osk, router=0):
    seav, ldca = ctx.sketch_image(router)
    assert seav.shape == osk.seav.shape and ldca.shape == osk.ldca.shape
    bad = np.nonzero(seav != osk.seav)[0]
    assert bad.size == 0, f"SEAV differs at {bad[:8]}"
    bad = np.nonzero(ldca != osk.ldca)[0]
    assert bad.size == 0, f"LDCA differs at {bad[:8]}"


def assert_same_results(got, want):
    assert len(got) == len(want)
    for f in ("ip", "z0", "flags"):
        assert np.array_equal(got[f], want[f]), f
    assert np.array_equal(got["est"].view(np.uint64), want["est"].view(np.uint64))


MODES = [1, 2]   # SP_SCAN_DIRECT, SP_SCAN_BINNED


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("n,offset", [(0, 0), (1, 0), (1, 1), (2, 1), (3, 0), (1001, 0), (1001, 1),
                                       (65537, 0), (200003, 1)])
def test_scan_parity_sizes_and_alignment(sp, torch, n, offset, mode):
    kw = dict(TINY, theta=16, seed=7, scan_mode=mode)
    pairs = W.uniform_pairs(n, seed=n + 3, n_hosts=max(1, n // 20))
    with sp.SuperPoint(**kw) as ctx:
        ctx.update(dev(torch, pairs, offset))
        torch.cuda.synchronize()
        assert_same_sketch(ctx, O.Sketch(oracle_params(kw)).update(pairs))


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("n", [4099, 200003])
def test_scan_parity_smallest_binned_planes(sp, torch, n, mode):
    """The smallest sketch the binned scan takes: k = 32 bit planes of
    LR x LC = 2 x 32 bits (the plane word index is a shift by 32, and one
    LDC is a single word), bit-exact in both scan forms."""
    kw = dict(r=12, isb=(0, 7, 14), ibn=(8, 8, 8), k_log2=5, lr=2, lc_log2=5, theta=16, seed=19, scan_mode=mode)
    pairs = W.uniform_pairs(n, seed=n + 11, n_hosts=max(1, n // 20))
    with sp.SuperPoint(**kw) as ctx:
        ctx.update(dev(torch, pairs))
        torch.cuda.synchronize()
        assert_same_sketch(ctx, O.Sketch(oracle_params(kw)).update(pairs))


# (profile, workload) pairs sized so that no SEA is overloaded: the oracle
# enumerates the full cartesian product of hot SEs, as the paper states it
PROFILES = [
    (dict(), dict(n=1 << 17, n_background=4096, n_planted=8, planted_degree=600), 64),      # profile D
    (dict(r=0, isb=(0, 8, 16, 24), ibn=(9, 9, 9, 9), lc_log2=12),                          # L = 32
     dict(n=1 << 14, n_background=64, n_planted=4, planted_degree=3000), 1024),
    (dict(r=16, isb=(0, 8), ibn=(9, 9), lr=1, lc_log2=0, k_log2=5),                        # SR = 2, LC = 1, k = 32
     dict(n=1 << 17, n_background=4096, n_planted=8, planted_degree=600), 64),
    (dict(r=16, isb=(0, 3, 6, 9, 12), ibn=(4, 4, 4, 4, 5), lr=8, lc_log2=10, k_log2=12),
     dict(n=1 << 17, n_background=4096, n_planted=8, planted_degree=600), 64),
    (dict(r=12, isb=(0, 10), ibn=(11, 11), lr=2, lc_log2=14, k_log2=16),             # 4 KiB SEA (limit), k = 2^16
     dict(n=1 << 17, n_background=4096, n_planted=8, planted_degree=600), 9),
]


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("kw,wl,theta", PROFILES)
def test_scan_and_detect_parity_profiles(sp, torch, kw, wl, theta, mode):
    kw = dict(kw, theta=theta, seed=1234, scan_mode=mode)
    pairs, planted = W.single_window(seed=5, **wl)
    with sp.SuperPoint(**kw) as ctx:
        ctx.update(dev(torch, pairs))
        got, n, rc = ctx.detect()
        osk = O.Sketch(oracle_params(kw)).update(pairs)
        assert_same_sketch(ctx, osk)
        want, n_want, over = osk.detect()
        assert rc == sp.SP_OK and not over
        assert n == n_want
        assert_same_results(got, want)
        assert set(planted.tolist()) <= set(got["ip"].tolist())


@pytest.mark.parametrize("mode", MODES)
def test_single_window_full_size(sp, torch, mode):
    """2^20 pairs, 20 planted hosts x 3,000 peers, theta 1024, profile D."""
    pairs, planted = W.single_window(seed=1)
    kw = dict(seed=1, scan_mode=mode)
    with sp.SuperPoint(**kw) as ctx:
        ctx.update(dev(torch, pairs))
        got, n, rc = ctx.detect(threshold=1024)
        osk = O.Sketch(oracle_params(kw)).update(pairs)
        assert_same_sketch(ctx, osk)
        want, _, _ = osk.detect(1024)
        assert rc == sp.SP_OK
        assert_same_results(got, want)
        assert set(planted.tolist()) <= set(got["ip"].tolist())


def test_threshold_sweep_and_warning(sp, torch):
    pairs, _ = W.single_window(seed=9, n=1 << 18, n_background=16384, n_planted=12,
                               planted_degree=2500)
    kw = dict(seed=9)
    with sp.SuperPoint(**kw) as ctx:
        ctx.update(dev(torch, pairs))
        osk = O.Sketch(oracle_params(kw)).update(pairs)
        for thr in (1024, 1500, 2000, 3000, 6000, 600):
            got, n, rc = ctx.detect(threshold=thr)
            want, n2, _ = osk.detect(thr)
            assert n == n2
            assert_same_results(got, want)
            assert rc == (sp.SP_WARN_THETA_BELOW_INIT if thr < 1024 else sp.SP_OK)


@pytest.mark.parametrize("mode", MODES)
def test_chunked_updates_and_reset(sp, torch, mode):
    pairs = W.uniform_pairs(300000, seed=41, n_hosts=2000)
    kw = dict(TINY, theta=32, seed=41, scan_mode=mode)
    with sp.SuperPoint(**kw) as ctx:
        for part in np.array_split(pairs, 7):
            ctx.update(dev(torch, part))
        assert_same_sketch(ctx, O.Sketch(oracle_params(kw)).update(pairs))
        ctx.reset()
        torch.cuda.synchronize()
        seav, ldca = ctx.sketch_image()
        assert not seav.any() and not ldca.any()


@pytest.mark.parametrize("mode", MODES)
def test_merge_parity(sp, torch, mode):
    """Sec. 4.2: OR of the routers' sketches = sketch of the union stream."""
    routers, sp_hosts = W.distributed(seed=3, n_routers=4, n_per_router=1 << 16, n_global_sp=6,
                                      sp_range=(1200, 2000), theta=1024)
    kw = dict(theta=256, seed=77, n_routers=5, scan_mode=mode)
    with sp.SuperPoint(**kw) as ctx:
        for i, r in enumerate(routers):
            ctx.update(dev(torch, r), router=i)
        ctx.merge([0, 1, 2, 3], 4)
        op = oracle_params(kw)
        whole = O.Sketch(op).update(np.concatenate(routers))
        assert_same_sketch(ctx, whole, router=4)
        for i, r in enumerate(routers):
            assert_same_sketch(ctx, O.Sketch(op).update(r), router=i)
        got, n, rc = ctx.detect(router=4, threshold=1024)
        want, _, _ = whole.detect(1024)
        assert_same_results(got, want)
        # merging into a router listed among the sources is idempotent
        ctx.merge([4, 0], 4)
        assert_same_sketch(ctx, whole, router=4)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_update_host_double_buffer(sp, torch, mode):
    pairs = W.uniform_pairs((1 << 22) + 12345, seed=8, n_hosts=100000)   # > one staging buffer
    kw = dict(theta=1024, seed=8, scan_mode=mode)
    host = torch.from_numpy(pairs.reshape(-1).view(np.int32)).pin_memory()
    with sp.SuperPoint(**kw) as ctx:
        ctx.update_host(host)
        torch.cuda.synchronize()
        assert_same_sketch(ctx, O.Sketch(oracle_params(kw)).update(pairs))
        # pageable memory works too
        ctx.reset()
        ctx.update_host(pairs)
        torch.cuda.synchronize()
        assert_same_sketch(ctx, O.Sketch(oracle_params(kw)).update(pairs))


@pytest.mark.parametrize("mode", MODES)
def test_export_import_roundtrip_and_checksum(sp, torch, mode):
    pairs = W.uniform_pairs(100000, seed=2, n_hosts=500)
    kw = dict(TINY, theta=16, seed=2, n_routers=2, scan_mode=mode)
    with sp.SuperPoint(**kw) as ctx:
        ctx.update(dev(torch, pairs[:60000]))
        img = sp.sp_export(ctx.ctx, 0)
        assert sp.sp_import(ctx.ctx, 1, img) == sp.SP_OK
        ctx.update(dev(torch, pairs[60000:]), router=1)    # resume after checkpoint
        assert_same_sketch(ctx, O.Sketch(oracle_params(kw)).update(pairs), router=1)
        bad = bytearray(img)
        bad[len(bad) // 2] ^= 0x10
        assert sp.sp_import(ctx.ctx, 0, bytes(bad)) == sp.SP_ERR_CHECKSUM
        assert sp.sp_import(ctx.ctx, 0, img[:-1]) == sp.SP_ERR_CHECKSUM
    with sp.SuperPoint(**dict(kw, seed=3)) as other:   # other hash seed: rejected
        assert sp.sp_import(other.ctx, 0, img) == sp.SP_ERR_CHECKSUM


def test_candidate_overflow_and_truncation(sp, torch):
    pairs, planted = W.single_window(seed=4, n=1 << 18, n_background=8192, n_planted=16,
                                     planted_degree=2000)
    kw = dict(seed=4, max_candidates=5)
    with sp.SuperPoint(**kw) as ctx:
        ctx.update(dev(torch, pairs))
        got, n, rc = ctx.detect()
        assert rc == sp.SP_ERR_CANDIDATE_OVERFLOW and n >= 16 and len(got) == 5
        want, n_want, _ = O.Sketch(oracle_params(kw)).update(pairs).detect()
        assert n == n_want
        assert set(got["ip"].tolist()) <= set(want["ip"].tolist())
    with sp.SuperPoint(**dict(kw, max_candidates=0)) as ctx:
        ctx.update(dev(torch, pairs))
        got, n, rc = sp.sp_detect(ctx.ctx, 0, 0, cap=3)
        assert rc == sp.SP_ERR_TRUNCATED and len(got) == 3
        assert_same_results(got, want[:3])


def test_join_bound(sp, torch):
    """A saturated SEAV makes the candidate product explode; the join bound
    stops the detect with SP_ERR_CANDIDATE_OVERFLOW instead of running on."""
    pairs = W.uniform_pairs(1 << 20, seed=6, n_hosts=1 << 16)
    kw = dict(r=4, isb=(0, 7, 14, 21), ibn=(8, 8, 8, 8), theta=1, seed=6, max_join=1 << 12)
    with sp.SuperPoint(**kw) as ctx:
        ctx.update(dev(torch, pairs))
        got, n, rc = ctx.detect(threshold=1)
        assert rc == sp.SP_ERR_CANDIDATE_OVERFLOW


def test_errors(sp, torch):
    with sp.SuperPoint(**TINY) as ctx:
        with pytest.raises(sp.SPError) as e:
            sp.sp_update(ctx.ctx, 3, dev(torch, np.zeros((4, 2), np.uint32)))
        assert e.value.code == sp.SP_ERR_ROUTER
        t = torch.zeros(9, dtype=torch.int32, device="cuda")
        assert sp.lib.sp_update(ctx.ctx, 0, t.data_ptr() + 4, 2) == sp.SP_ERR_PARAM
        assert sp.lib.sp_results(ctx.ctx, None, 0, sp.ctypes.byref(sp.ctypes.c_uint64())) == sp.SP_ERR_STATE
    with pytest.raises(sp.SPError):
        sp.SuperPoint(**dict(TINY, theta=0))


def test_binned_pending_planes(sp, torch):
    """Several binned updates accumulate in the plane buffer; detect, merge,
    export and reset see exactly the oracle's sketch at every point."""
    kw = dict(theta=256, seed=31, n_routers=3, scan_mode=2)
    op = oracle_params(kw)
    a = W.uniform_pairs(1 << 18, seed=31, n_hosts=20000)
    b, _ = W.single_window(seed=32, n=1 << 18, n_background=8192, n_planted=6, planted_degree=900)
    with sp.SuperPoint(**kw) as ctx:
        ctx.update(dev(torch, a), router=0)
        ctx.update(dev(torch, b[:100000]), router=0)          # accumulate on pending planes
        ctx.update(dev(torch, b[100000:]), router=0)
        ora = O.Sketch(op).update(a).update(b)
        got, n, rc = ctx.detect(router=0)
        want, _, _ = ora.detect()
        assert_same_results(got, want)
        assert_same_sketch(ctx, ora, router=0)
        ctx.update(dev(torch, a), router=1)
        ctx.update(dev(torch, b), router=2)
        ctx.merge([1, 2], 0)                                   # sources still pending
        assert_same_sketch(ctx, ora, router=0)
        ctx.update(dev(torch, b), router=1)
        ctx.reset(1)                                           # drops the pending planes
        ctx.update(dev(torch, a[:5000]), router=1)
        assert_same_sketch(ctx, O.Sketch(op).update(a[:5000]), router=1)


def test_binned_list_overflow_skew(sp, torch):
    """Every pair has the same opposite IP, so all of them fall into one bit
    plane: the per-block lists overflow and the rest goes through L2 REDs."""
    n = 1 << 20
    rng = np.random.default_rng(12)
    pairs = np.stack([rng.integers(0, 2**32, n, dtype=np.uint32),
                      np.full(n, 0x0A000001, np.uint32)], 1)
    pairs[: n // 2, 1] = rng.integers(0, 2**32, n // 2, dtype=np.uint32)   # half skewed
    kw = dict(seed=12, scan_mode=2)
    with sp.SuperPoint(**kw) as ctx:
        ctx.update(dev(torch, pairs))
        assert_same_sketch(ctx, O.Sketch(oracle_params(kw)).update(pairs))


@pytest.mark.parametrize("mode", [0, 1])
def test_core_link_full_size(sp, torch, mode):
    """The 2^26-pair core-link workload in the launch configuration the
    benchmark times (one scan call, one detect), bit-exact against the oracle
    over the whole sketch and result list."""
    pairs, planted = _core_link()
    kw = dict(seed=2, scan_mode=mode)
    with sp.SuperPoint(**kw) as ctx:
        ctx.update(dev(torch, pairs))
        got, n, rc = ctx.detect(threshold=1024)
        if "oracle" not in _CORE:
            osk = O.Sketch(oracle_params(kw)).update(pairs)
            _CORE["oracle"] = (osk, osk.detect(1024)[0])
        osk, want = _CORE["oracle"]
        assert_same_sketch(ctx, osk)
        assert rc == sp.SP_OK
        assert_same_results(got, want)
        recall = len(set(planted.tolist()) & set(got["ip"].tolist())) / len(planted)
        assert recall > 0.95


def _shape_count(sp):
    return len(sp.sp_binned_shapes())


@pytest.mark.parametrize("shape", range(6))
def test_every_binned_shape_is_bit_exact(sp, torch, shape):
    """Every compiled staging shape of the binned scan gives the oracle's
    sketch: unaligned head, a ragged last tile, appending launches (host
    path chunks and a batched call of many streams), pending planes, a
    skewed stream that overflows rows and lists, and a detect."""
    if shape >= _shape_count(sp):
        pytest.skip("fewer compiled shapes")
    kw = dict(theta=256, seed=41, n_routers=2, scan_mode=2)
    op = oracle_params(kw)
    a, planted = W.single_window(seed=41, n=(1 << 20) + 12345, n_background=16384, n_planted=6, planted_degree=900)
    n = 1 << 18
    rng = np.random.default_rng(41)
    skew = np.stack([rng.integers(0, 2**32, n, dtype=np.uint32), np.full(n, 0x0A000001, np.uint32)], 1)
    parts = np.array_split(W.uniform_pairs(600000, seed=42, n_hosts=30000), 40)
    with sp.SuperPoint(**kw) as ctx:
        sp.sp_set_binned_shape(ctx.ctx, shape)
        assert sp.sp_get_binned_shape(ctx.ctx)["index"] == shape
        ctx.update(dev(torch, a, 1), router=0)                              # 8 bytes off a 16-byte boundary
        ctx.update(dev(torch, skew), router=0)                              # on pending planes, rows overflow
        host = torch.from_numpy(a.reshape(-1).view(np.int32).copy()).pin_memory()
        ctx.update_host(host, router=1)
        sp.sp_update_batched(ctx.ctx, [1] * len(parts), [dev(torch, x) for x in parts])
        osk0 = O.Sketch(op).update(a).update(skew)
        assert_same_sketch(ctx, osk0, router=0)
        osk1 = O.Sketch(op).update(a).update(np.concatenate(parts))
        assert_same_sketch(ctx, osk1, router=1)
        got, n_got, rc = ctx.detect(router=1)
        want, _, _ = osk1.detect()
        assert_same_results(got, want)


def test_autotune_binned_picks_a_shape_and_stays_exact(sp, torch):
    pairs, planted = W.core_link(seed=43, n=1 << 22)
    kw = dict(seed=43, scan_mode=2)
    with sp.SuperPoint(**kw) as ctx:
        best = sp.sp_autotune_binned(ctx.ctx, dev(torch, pairs))
        assert 0 <= best["index"] < _shape_count(sp) and sp.sp_get_binned_shape(ctx.ctx) == best
        seav, ldca = ctx.sketch_image(0)
        assert not seav.any() and not ldca.any()                           # the tuner left router 0 empty
        ctx.update(dev(torch, pairs))
        osk = O.Sketch(oracle_params(kw)).update(pairs)
        assert_same_sketch(ctx, osk)
        got, n, rc = ctx.detect()
        assert_same_results(got, osk.detect()[0])
        with pytest.raises(sp.SPError) as e:
            sp.sp_set_binned_shape(ctx.ctx, _shape_count(sp))
        assert e.value.code == sp.SP_ERR_PARAM
    with sp.SuperPoint(**dict(kw, k_log2=12, lc_log2=14)) as ctx:            # k > 1024: no binned scan
        with pytest.raises(sp.SPError) as e:
            sp.sp_autotune_binned(ctx.ctx, dev(torch, pairs[:1000]))
        assert e.value.code == sp.SP_ERR_STATE


def _many_hosts(n_hosts, seed):
    """n_hosts hosts with 64 distinct peers each, shuffled: at theta = 32 each
    is a super point, so the detection returns about n_hosts results."""
    rng = np.random.default_rng(seed)
    hosts = np.unique(rng.integers(0, 2**32, n_hosts + n_hosts // 4 + 64, dtype=np.uint32))[:n_hosts]
    hosts = rng.permutation(hosts)
    pairs = np.stack([np.repeat(hosts, 64), rng.integers(0, 2**32, hosts.size * 64, dtype=np.uint32)], 1)
    return np.ascontiguousarray(pairs[rng.permutation(pairs.shape[0])]), hosts


@pytest.mark.parametrize("n_hosts", [12000, 20000, 150000])
def test_detect_sort_beyond_one_block(sp, torch, n_hosts):
    """More results than one block sorts in shared memory (8,192): runs of
    8,192 sorted per block, then merged across the grid (one round, two
    rounds, five rounds at more than 65,536 results); the list equals the
    oracle's, in order, bit for bit."""
    kw = dict(r=16, isb=(0, 8), ibn=(9, 9), theta=32, seed=51)
    pairs, hosts = _many_hosts(n_hosts, 51 + n_hosts)
    with sp.SuperPoint(**kw) as ctx:
        ctx.update(dev(torch, pairs))
        got, n, rc = ctx.detect()
        osk = O.Sketch(oracle_params(kw)).update(pairs)
        want, n_want, overflow = osk.detect()
        assert not overflow and rc == sp.SP_OK and n == n_want > 8192
        assert_same_results(got, want)
        if n_hosts > 65536:
            assert n > 65536
            assert len(set(hosts.tolist()) - set(got["ip"].tolist())) <= n_hosts // 100


def test_reset_range(sp, torch):
    """sp_reset_range zeroes exactly the routers of the range (one launch),
    drops their pending binned planes, and leaves the others intact."""
    kw = dict(theta=256, seed=61, n_routers=4, scan_mode=2)
    op = oracle_params(kw)
    data = [W.uniform_pairs(50000 + 1000 * r, seed=610 + r, n_hosts=5000) for r in range(4)]
    with sp.SuperPoint(**kw) as ctx:
        for r in range(4):
            ctx.update(dev(torch, data[r]), router=r)
        sp.sp_reset_range(ctx.ctx, 1, 2)
        for r in range(4):
            seav, ldca = ctx.sketch_image(r)
            if r in (1, 2):
                assert not seav.any() and not ldca.any(), r
            else:
                assert_same_sketch(ctx, O.Sketch(op).update(data[r]), router=r)
        ctx.update(dev(torch, data[0]), router=2)               # the router works on after the reset
        assert_same_sketch(ctx, O.Sketch(op).update(data[0]), router=2)
        with pytest.raises(sp.SPError) as e:
            sp.sp_reset_range(ctx.ctx, 3, 2)
        assert e.value.code == sp.SP_ERR_ROUTER


def _random_profile(rng):
    """A random parameter set inside the library's limits that satisfies the
    coverage and overlap constraints of Sec. 3.2 (checked by the oracle)."""
    while True:
        r = int(rng.integers(4, 20))
        L = 32 - r
        sr = int(rng.integers(2, 6))
        step = -(-L // sr)
        ibn = [int(min(12, L, step + rng.integers(1, 4))) for _ in range(sr)]
        isb = [(i * step + int(rng.integers(0, 2))) % L for i in range(sr)]
        k_log2 = int(rng.integers(5, 12))
        lr = int(rng.integers(1, 9))
        lc_log2 = int(rng.integers(5, 15))
        if (lr << lc_log2) > (1 << 20) or sum(1 << b for b in ibn) > 4096:
            continue
        kw = dict(r=r, isb=tuple(isb), ibn=tuple(ibn), k_log2=k_log2, lr=lr, lc_log2=lc_log2)
        if O.check_params(oracle_params(dict(kw, theta=64, seed=1))) == 0:
            return kw


@pytest.mark.parametrize("case", range(12))
def test_random_profiles_both_scan_forms(sp, torch, case):
    """Seeded random profiles: every scan form gives the oracle's sketch and
    detection bit for bit (one-word LDCs, 32-bit LDCA rows, up to 8 rows,
    k up to 2048 -- the binned form applies up to k = 1024)."""
    rng = np.random.default_rng(700 + case)
    kw = dict(_random_profile(rng), theta=int(rng.choice([48, 64, 256])), seed=700 + case)
    pairs, _ = W.single_window(seed=710 + case, n=int(rng.integers(1 << 14, 1 << 17)), n_background=2048,
                               n_planted=4, planted_degree=400)
    osk = O.Sketch(oracle_params(kw)).update(pairs)
    want, n_want, overflow = osk.detect()
    for mode in (1, 2):
        with sp.SuperPoint(**dict(kw, scan_mode=mode)) as ctx:
            ctx.update(dev(torch, pairs, case % 2))
            assert_same_sketch(ctx, osk)
            got, n, rc = ctx.detect()
            if not overflow:
                assert n == n_want and rc in (sp.SP_OK, sp.SP_ERR_TRUNCATED)
                assert_same_results(got, want[:len(got)])


@pytest.mark.parametrize("mode", MODES)
def test_wide_planes_two_blocks_per_plane(sp, torch, mode):
    """LC = 2^18 (profile D3): a binned plane of four rows is 128 KiB, so two
    blocks share each plane, two rows apiece.  In the binned form three
    updates (one of 4,099 pairs) accumulate into the planes before the fold;
    in both forms the sketch and the detection equal the oracle's."""
    kw = dict(r=16, isb=(0, 4, 8, 12), ibn=(7, 7, 7, 7), lc_log2=18, theta=256, seed=31, scan_mode=mode)
    a, _ = W.single_window(seed=31, n=(1 << 20) + 3, n_background=1 << 15, n_planted=6, planted_degree=900)
    b, _ = W.single_window(seed=32, n=(1 << 19) + 5, n_background=1 << 14, n_planted=6, planted_degree=700)
    c = W.uniform_pairs(4099, seed=33, n_hosts=300)
    with sp.SuperPoint(**kw) as ctx:
        ctx.update(dev(torch, a))
        ctx.update(dev(torch, c))
        ctx.update(dev(torch, b, 1))
        osk = O.Sketch(oracle_params(kw)).update(np.concatenate([a, c, b]))
        assert_same_sketch(ctx, osk)
        got, n, rc = ctx.detect()
        want, n_want, _ = osk.detect()
        assert rc == sp.SP_OK and n == n_want
        assert_same_results(got, want)


def test_fold_of_a_freshly_zeroed_ldca(sp, torch):
    """After a reset the fold writes the binned planes without reading the
    LDCA.  It must still OR whenever something else wrote the LDCA first: a
    binning launch that spilled past a full list, a merge into the router, an
    import, a direct update.  Each case against the oracle."""
    n = 1 << 19
    rng = np.random.default_rng(41)
    skew = np.stack([rng.integers(0, 2**32, n, dtype=np.uint32), np.full(n, 0x0A000001, np.uint32)], 1)
    a = W.uniform_pairs(1 << 18, seed=41, n_hosts=20000)
    b = W.uniform_pairs(1 << 18, seed=42, n_hosts=30000)
    kw = dict(seed=41, n_routers=4, scan_mode=2)
    op = oracle_params(kw)
    with sp.SuperPoint(**kw) as ctx:
        ctx.update(dev(torch, skew), router=0)                 # lists overflow: spilled bits in the LDCA
        ctx.update(dev(torch, a), router=1)
        assert_same_sketch(ctx, O.Sketch(op).update(skew), router=0)
        assert_same_sketch(ctx, O.Sketch(op).update(a), router=1)
        ctx.merge([1], 2)                                      # router 2's LDCA now holds a's bits
        ctx.update(dev(torch, b), router=2)
        assert_same_sketch(ctx, O.Sketch(op).update(a).update(b), router=2)
        image = sp.sp_export(ctx.ctx, 1)
        sp.sp_reset_range(ctx.ctx, 0, 4)                       # every router fresh again
        ctx.update(dev(torch, b), router=0)                    # no spill this time
        assert_same_sketch(ctx, O.Sketch(op).update(b), router=0)
        assert sp.sp_import(ctx.ctx, 3, image) == sp.SP_OK     # router 3 = a's sketch
        ctx.update(dev(torch, b), router=3)
        assert_same_sketch(ctx, O.Sketch(op).update(a).update(b), router=3)
    with sp.SuperPoint(**dict(kw, scan_mode=0)) as ctx:        # auto: a small direct update, then a binned one
        ctx.update(dev(torch, a[:4096]))
        big = W.uniform_pairs((1 << 22) + 11, seed=43, n_hosts=1 << 20)
        ctx.update(dev(torch, big))
        assert_same_sketch(ctx, O.Sketch(oracle_params(dict(kw, scan_mode=0))).update(a[:4096]).update(big))
