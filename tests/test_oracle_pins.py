"""Pins of the CPU oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: every expected value is a
closed form, a published vector, a hand-worked example, a brute force over a
tiny input with a different algorithm, or an invariant the paper states.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_1901_07306_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# A tiny profile for brute force: r = 12 leaves L = 20 LP bits, 2^20 LPs per
# SEA; rows cover LP bits 0-7, 7-14 and 14-21 mod 20 = {14..19, 0, 1}, so
# consecutive rows share bits 7, 14 and {0, 1}.
TINY = dict(r=12, isb=(0, 7, 14), ibn=(8, 8, 8), k_log2=8, lr=3, lc_log2=6)


def _golden_lines(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


# ---------------------------------------------------------------- Eq. 1 --
def test_tau_closed_form():
    # tau = ceil(log2(theta / 8)), clamped at 0 (Eq. 1)
    assert O.tau(1024) == 7
    assert O.tau(8) == 0 and O.tau(1) == 0 and O.tau(9) == 1 and O.tau(16) == 1
    assert O.tau(17) == 2 and O.tau(2**32 - 1) == 29
    for theta in list(range(1, 5000)) + [2**20, 2**20 + 1, 3 * 2**25]:
        # ceil(log2(theta)) - 3 from the bit length, independently of the loop
        expect = max(0, (theta - 1).bit_length() - 3)
        assert O.tau(theta) == expect, theta


def test_lsb_definition():
    assert O.lsb(0) == 32
    for x in [1, 2, 3, 4, 96, 2**31, 0xFFFFFFFF, 0x80000000, 0x00010000]:
        assert O.lsb(x) == (x & -x).bit_length() - 1


# ------------------------------------------------------------ hash family --
def test_splitmix64_published_vector():
    want = [int(v[0], 16) for v in _golden_lines("splitmix64_seed0.txt")]
    assert O.splitmix64_stream(0, 4) == want


def test_mas_closed_forms():
    # (a x + b) mod 2^64, top 32 bits
    assert O.mas(2**32, 0, 12345) == 12345
    assert O.mas(0, 0xDEADBEEF_00000000, 7) == 0xDEADBEEF
    assert O.mas(1, 0, 0xFFFFFFFF) == 0
    assert O.mas(2**64 - 1, 0, 1) == 0xFFFFFFFF   # -1 mod 2^64
    assert O.mas(2**64 - 1, 0, 2) == 0xFFFFFFFF   # wrap to 2^64 - 2
    assert O.mas(2**63, 0, 2) == 0                # 2^64 wraps to 0
    assert O.mas(2**63, 2**63, 1) == 0            # carry out of bit 63 is dropped
    rng = np.random.default_rng(5)
    for _ in range(200):
        a, b = (int(v) for v in rng.integers(0, 2**64, 2, dtype=np.uint64))
        x = int(rng.integers(0, 2**32))
        assert O.mas(a, b, x) == ((a * x + b) % 2**64) >> 32


def test_hash_params_draw_order():
    # (a, b) for H1, H3, LH_0.. are consecutive SplitMix64 outputs
    a, b = O.hash_params(0, 2)
    s = O.splitmix64_stream(0, 8)
    assert [int(v) for v in a] == s[0::2]
    assert [int(v) for v in b] == s[1::2]


def test_mas_is_universal_statistically():
    # Dietzfelbinger multiply-add-shift: Pr[h(x) = h(y)] <= 2^-l over (a, b)
    rng = np.random.default_rng(6)
    l = 8
    hits, trials = 0, 20000
    for t in range(trials):
        a, b = (int(v) for v in rng.integers(0, 2**64, 2, dtype=np.uint64))
        hx = O.mas(a, b, 12345) >> (32 - l)
        hy = O.mas(a, b, 12346) >> (32 - l)
        hits += hx == hy
    p = 2.0**-l
    assert hits <= trials * p + 4 * math.sqrt(trials * p)


# ----------------------------------------------------------- Eq. 2 / Eq. 3 --
def test_idx_hand_worked_examples():
    p = O.Params()  # r = 14, ISB = 0, 5, 10, 15, IBN = 7
    for row, lp, want in _golden_lines("eq2_idx_examples.txt"):
        assert O.idx(p, int(row), int(lp, 16)) == int(want, 16), (row, lp)


def test_rp_lp_split():
    for r in [0, 1, 14, 20, 24]:
        for ip in [0, 1, 0xFFFFFFFF, 0x12345678, 0x80000001]:
            assert O.rp(r, ip) == ip % (1 << r)
            assert O.lp(r, ip) == ip // (1 << r)


def test_param_constraints():
    assert O.check_params(O.Params()) == 0
    assert O.check_params(O.Params(**TINY)) == 0
    # constraint 1: LP bit 17 uncovered (rows end at bit 16)
    assert O.check_params(O.Params(isb=(0, 5, 10), ibn=(7, 7, 7))) == 5
    # constraint 2: rows 0 and 1 do not share a bit
    assert O.check_params(O.Params(isb=(0, 7, 10, 15), ibn=(7, 7, 7, 7))) == 6
    # the paper's own example rule IBN = ceil(L / SR) + a, ISB = i * ceil(L / SR)
    L, sr, a = 18, 4, 2
    step = -(-L // sr)
    p = O.Params(isb=tuple(i * step for i in range(sr)), ibn=(step + a,) * sr)
    assert p.isb == (0, 5, 10, 15) and p.ibn == (7, 7, 7, 7)
    assert O.check_params(p) == 0
    assert O.check_params(O.Params(theta=0)) == 10
    assert O.check_params(O.Params(k_log2=4)) == 7


# --------------------------------------------------------- Eq. 4 / Z_theta --
def test_z_theta_closed_form():
    # -k ln(z / k) >= theta  <=>  z <= k exp(-theta / k)
    assert O.z_theta(10, 1024) == 376   # floor(1024 / e)
    for k_log2 in [5, 8, 10, 12]:
        k = 1 << k_log2
        for theta in [1, 2, 10, 100, 1000, 1024, 3000, 5000, 10**6]:
            bound = k * math.exp(-theta / k)
            if abs(bound - round(bound)) < 1e-9:
                continue
            assert O.z_theta(k_log2, theta) == math.floor(bound), (k, theta)


def test_est_formula_values():
    # Eq. 4: Est = -k ln(z0 / k)
    assert O.est(10, 1024) == 0.0
    assert abs(O.est(10, 512) - 1024 * math.log(2)) < 1e-9
    assert abs(O.est(10, 376) - 1025.9278461) < 1e-6


# ------------------------------------------------------------ update scan --
def _sketch(pairs, **kw):
    return O.Sketch(O.Params(**kw)).update(pairs)


def test_single_pair_sets_expected_bits():
    # theta = 1 gives tau = 0: every pair is sampled (Sec. 3.1)
    p = dict(TINY, theta=1)
    s = _sketch(np.array([[0xC0A80001, 0x08080808]], np.uint32), **p)
    assert int(np.unpackbits(s.seav).sum()) == 3            # one bit per SEA row
    assert int(np.unpackbits(s.ldca.view(np.uint8)).sum()) == 3  # one bit per LDCA row
    # with theta huge the pair is almost never sampled but LDCA is still set
    q = dict(TINY, theta=2**31)
    s = _sketch(np.array([[1, 2]], np.uint32), **q)
    assert int(np.unpackbits(s.ldca.view(np.uint8)).sum()) == 3


def test_sampling_boundary_is_inclusive():
    """Sec. 3.1 (reading 2: lsb(H1(oip)) >= tau): a pair whose H1 has its
    lowest set bit exactly at tau is sampled -- its SE bit is set in every
    SEA row -- and one whose lowest set bit is at tau - 1 is not."""
    p = O.Params(**dict(TINY, theta=64))            # tau = 3
    tau = O.tau(p.theta)
    assert tau == 3
    at = next(o for o in range(1, 1 << 20) if O.lsb(O.h1(p, o)) == tau)
    below = next(o for o in range(1, 1 << 20) if O.lsb(O.h1(p, o)) == tau - 1)
    for oip, sampled in ((at, True), (below, False)):
        s = _sketch(np.array([[0x0A0B0C0D, oip]], np.uint32), **dict(TINY, theta=64))
        assert int(np.unpackbits(s.seav).sum()) == (p.sr if sampled else 0), oip
        assert int(np.unpackbits(s.ldca.view(np.uint8)).sum()) == p.lr   # the LDCA takes every pair


def test_sampling_rate_matches_tau():
    # lsb(H1(oip)) >= tau happens with probability 2^-tau for a uniform H1
    p = O.Params(**dict(TINY, theta=64))  # tau = 3
    assert O.tau(64) == 3
    n = 40000
    oips = np.random.default_rng(9).integers(0, 2**32, n, dtype=np.uint32)
    hits = sum(O.lsb(O.h1(p, int(o))) >= 3 for o in oips)
    mu, sd = n / 8, math.sqrt(n / 8 * 7 / 8)
    assert abs(hits - mu) < 4 * sd


def test_order_independence_and_idempotence():
    pairs = W.uniform_pairs(20000, seed=11, n_hosts=300)
    base = _sketch(pairs, **TINY, theta=16)
    perm = pairs[np.random.default_rng(1).permutation(len(pairs))]
    dup = np.concatenate([pairs, pairs[:7000]])
    for other in (perm, dup):
        s = _sketch(other, **TINY, theta=16)
        assert np.array_equal(s.seav, base.seav) and np.array_equal(s.ldca, base.ldca)


def test_merge_equals_concatenation():
    pairs = W.uniform_pairs(30000, seed=12, n_hosts=500)
    whole = _sketch(pairs, **TINY, theta=16)
    parts = np.array_split(pairs, 5)
    merged = _sketch(parts[0], **TINY, theta=16)
    for part in parts[1:]:
        merged.merge(_sketch(part, **TINY, theta=16))
    assert np.array_equal(merged.seav, whole.seav)
    assert np.array_equal(merged.ldca, whole.ldca)


# ----------------------------------------------------------------- restore --
def _popc8(x):
    return bin(int(x)).count("1")


def _brute_force_sea(p: O.Params, s: O.Sketch, threshold: int, rp_: int):
    """Forward enumeration of every LP of one SEA against the definition of a
    super point candidate (every chosen SE has weight >= 3 and their AND has
    weight >= 3, Sec. 3.2), then the LDCA union test (Sec. 3.3).  Idx is
    computed here bit by bit from Eq. 2; no inverse (Eq. 3) is used."""
    L = 32 - p.r
    sea_b = O.sea_bytes(p)
    offs = np.concatenate([[0], np.cumsum([1 << b for b in p.ibn])])
    lps = np.arange(1 << L, dtype=np.int64)
    popc = np.array([_popc8(x) for x in range(256)])
    zt = O.z_theta(p.k_log2, threshold)
    k = 1 << p.k_log2
    wpl = k // 32
    lcn = 1 << p.lc_log2
    sea = s.seav[rp_ * sea_b:(rp_ + 1) * sea_b]
    ok = np.ones(lps.size, bool)
    seu = np.full(lps.size, 0xFF, np.int64)
    for i in range(p.sr):
        v = np.zeros_like(lps)
        for j in range(p.ibn[i]):
            v |= ((lps >> ((p.isb[i] + j) % L)) & 1) << j
        se = sea[offs[i] + v]
        ok &= popc[se] >= 3
        seu &= se
    ok &= popc[seu] >= 3
    out = {}
    for lpv in lps[ok]:
        ip = (int(lpv) << p.r) | rp_
        u = np.full(wpl, 0xFFFFFFFF, np.uint32)
        for i in range(p.lr):
            col = O.lh(p, i, ip)
            u &= s.ldca[(i * lcn + col) * wpl:(i * lcn + col + 1) * wpl]
        z0 = k - int(np.unpackbits(u.view(np.uint8)).sum())
        if z0 <= zt:
            out[ip] = z0
    return out


def _rows_all_hot(p, s, rp_):
    sea_b = O.sea_bytes(p)
    sea = s.seav[rp_ * sea_b:(rp_ + 1) * sea_b]
    off = 0
    for b in p.ibn:
        row = sea[off:off + (1 << b)]
        if not any(_popc8(x) >= 3 for x in row):
            return False
        off += 1 << b
    return True


@pytest.mark.parametrize("seed", [21, 22])
def test_detect_matches_forward_brute_force(seed):
    p = O.Params(**TINY, theta=24, seed=seed)   # tau = 2
    rng = np.random.default_rng(seed)
    # hosts concentrated on 64 SEAs so that SEs are shared and noisy
    rps = rng.integers(0, 1 << p.r, 64)
    L = 32 - p.r
    heavy = [(int(rng.integers(0, 1 << L)) << p.r) | int(rps[i % 64]) for i in range(12)]
    rows = []
    for h in heavy:
        d = int(rng.integers(30, 200))
        rows.append(np.stack([np.full(d, h, np.uint32), rng.integers(0, 2**32, d, dtype=np.uint32)], 1))
    bg_hosts = (rng.integers(0, 1 << L, 3000) << p.r) | rps[rng.integers(0, 64, 3000)]
    bg = np.stack([bg_hosts[rng.integers(0, 3000, 20000)].astype(np.uint32),
                   rng.integers(0, 2**32, 20000, dtype=np.uint32)], 1)
    s = O.Sketch(p).update(np.concatenate(rows + [bg]))
    got, n, over = s.detect(threshold=24)
    assert not over and n == len(got)
    expect = {}
    # an SEA with an empty HSE(i) yields no candidate by definition, so the
    # brute force only needs the SEAs whose every row holds a hot SE
    hot = [rp_ for rp_ in range(1 << p.r) if _rows_all_hot(p, s, rp_)]
    assert 0 < len(hot) <= 64
    for rp_ in hot:
        expect.update(_brute_force_sea(p, s, 24, rp_))
    assert {int(c["ip"]): int(c["z0"]) for c in got} == expect
    assert list(got["ip"]) == sorted(got["ip"])
    assert len(set(heavy) & set(expect)) >= 6


def test_threshold_boundary_is_inclusive():
    """Def. 2 and Eq. 4 (reading 11: Est >= theta as z0 <= Z_theta): one host
    alone in the stream has a ULDC of exactly k - |H3(peers)| zeros (no other
    host shares its LDCs).  With Z_theta = floor(k exp(-theta / k)) zeros it
    is reported; with one zero more it is not."""
    theta, k = 64, 256
    p = O.Params(**dict(TINY, theta=theta, seed=77))
    zt = math.floor(k * math.exp(-theta / k))       # 199
    host = 0x0A0B0C0D

    def peers_with_distinct_h3(d):
        seen, peers, o = set(), [], 1
        while len(seen) < d:
            h = O.h3(p, o)
            if h not in seen:
                seen.add(h)
                peers.append(o)
            o += 1
        # enough sampled peers with distinct H2 for a hot SE in every row,
        # taken among peers whose H3 is already present (z0 unchanged)
        bits = {O.h1(p, x) >> 29 for x in peers if O.lsb(O.h1(p, x)) >= O.tau(theta)}
        while len(bits) < 3:
            h1 = O.h1(p, o)
            if O.h3(p, o) in seen and O.lsb(h1) >= O.tau(theta) and (h1 >> 29) not in bits:
                bits.add(h1 >> 29)
                peers.append(o)
            o += 1
        return np.stack([np.full(len(peers), host, np.uint32), np.array(peers, np.uint32)], 1)

    got, n, _ = O.Sketch(p).update(peers_with_distinct_h3(k - zt)).detect(theta)
    assert n == 1 and int(got["ip"][0]) == host and int(got["z0"][0]) == zt
    got, n, _ = O.Sketch(p).update(peers_with_distinct_h3(k - zt - 1)).detect(theta)
    assert n == 0


def test_detect_reports_est_and_saturation():
    # one host with far more peers than k ln k saturates its LDC union
    p = O.Params(**dict(TINY, theta=8, k_log2=5))
    rng = np.random.default_rng(3)
    host = 0xABCDE123
    pairs = np.stack([np.full(4000, host, np.uint32), rng.integers(0, 2**32, 4000, dtype=np.uint32)], 1)
    got, n, _ = O.Sketch(p).update(pairs).detect(8)
    assert n == 1 and int(got["ip"][0]) == host
    assert int(got["z0"][0]) == 0 and int(got["flags"][0]) == O.FLAG_SATURATED
    assert got["est"][0] == 32 * math.log(32)


def test_detect_cap_truncates_and_flags():
    pairs, planted = W.single_window(seed=1, n=1 << 16, n_background=4096, n_planted=6,
                                     planted_degree=3000)
    s = O.Sketch(O.Params()).update(pairs)
    full, n, over = s.detect()
    assert not over and n >= 6
    part, n2, over2 = s.detect(cap=3)
    assert over2 and n2 == n and np.array_equal(part, full[:3])


# ------------------------------------------ ground truth, Def. 1 and Def. 2 --
def test_exact_counts_brute_force():
    pairs = W.uniform_pairs(3000, seed=4, n_hosts=40)
    pairs = np.concatenate([pairs, pairs[:500]])  # duplicates do not count twice
    hosts, counts = O.exact_opposite_counts(pairs)
    ref = {}
    for h, o in pairs.tolist():
        ref.setdefault(h, set()).add(o)
    assert dict(zip(hosts.tolist(), counts.tolist())) == {h: len(v) for h, v in ref.items()}


def test_no_false_negative_invariant():
    """Every host whose own sampled SE has weight >= 3 becomes a candidate
    (sharing only adds bits), and passes the LDCA test when its own LDC
    already has at most Z_theta zeros (the AND union only adds noise ones)."""
    p = O.Params(r=10, isb=(0, 6, 12, 17), ibn=(8, 8, 8, 7), theta=256, lc_log2=12)
    assert O.check_params(p) == 0
    pairs, planted = W.single_window(seed=7, n=1 << 17, n_background=8192, n_planted=12,
                                     planted_degree=1200)
    s = O.Sketch(p).update(pairs)
    got, n, _ = s.detect()
    found = set(int(x) for x in got["ip"])
    tau = O.tau(p.theta)
    zt = O.z_theta(p.k_log2, p.theta)
    k = 1 << p.k_log2
    by_host = {}
    for h, o in np.unique(pairs, axis=0).tolist():
        by_host.setdefault(h, []).append(o)
    must = 0
    for h, peers in by_host.items():
        if len(peers) < 100:
            continue
        bits = set()
        h3s = set()
        for o in peers:
            v = O.h1(p, o)
            if O.lsb(v) >= tau:
                bits.add(v >> 29)
            h3s.add(O.h3(p, o))
        if len(bits) >= 3 and k - len(h3s) <= zt:
            must += 1
            assert h in found, hex(h)
    assert must >= 10


def test_single_window_finds_all_planted():
    pairs, planted = W.single_window(seed=1)
    assert pairs.shape == (1 << 20, 2)
    truth = O.exact_super_points(pairs, 1024)
    assert set(planted.tolist()) <= set(truth.tolist())
    got, n, over = O.Sketch(O.Params(seed=1)).update(pairs).detect(1024)
    assert not over
    assert set(planted.tolist()) <= set(int(x) for x in got["ip"])


# ------------------------------------------------ Eq. 4 and Lemma 1, stats --
def test_ldc_zero_count_expectation():
    """Linear counting (Whang et al.): with n distinct items hashed into k
    bits, E[z0] = k (1 - 1/k)^n, Var from the occupancy distribution."""
    k_log2, n, trials = 8, 300, 300
    k = 1 << k_log2
    zs = []
    rng = np.random.default_rng(31)
    for t in range(trials):
        p = O.Params(**dict(TINY, k_log2=k_log2, lr=1, seed=1000 + t))
        peers = np.unique(rng.integers(0, 2**32, n + 10, dtype=np.uint32))[:n]
        s = O.Sketch(p).update(np.stack([np.full(n, 77, np.uint32), peers], 1))
        zs.append(k - int(np.unpackbits(s.ldca.view(np.uint8)).sum()))
    q1, q2 = (1 - 1 / k) ** n, (1 - 2 / k) ** n
    mean = k * q1
    var = k * (k - 1) * q2 + k * q1 - (k * q1) ** 2
    assert abs(np.mean(zs) - mean) < 4 * math.sqrt(var / trials)


def test_lemma1_psu_monte_carlo():
    """Lemma 1: a bit of a fresh host's ULDC is set with probability
    Psu = (1 - (1 - 1/k)^(N / LC))^LR."""
    k_log2, lr, lc_log2, N = 6, 3, 4, 1200
    k, lc = 1 << k_log2, 1 << lc_log2
    p = O.Params(**dict(TINY, k_log2=k_log2, lr=lr, lc_log2=lc_log2, seed=99))
    pairs = W.uniform_pairs(N, seed=17)
    s = O.Sketch(p).update(pairs)
    probes = np.random.default_rng(18).integers(0, 2**32, 3000, dtype=np.uint32)
    ones = 0
    for h in probes:
        u = np.full(k // 32, 0xFFFFFFFF, np.uint32)
        for i in range(lr):
            c = O.lh(p, i, int(h))
            u &= s.ldca[(i * lc + c) * (k // 32):(i * lc + c + 1) * (k // 32)]
        ones += int(np.unpackbits(u.view(np.uint8)).sum())
    psu = (1 - (1 - 1 / k) ** (N / lc)) ** lr
    # probes share LDCs (only LR * LC of them), so use the LDC-level spread
    # as the error scale: each row's LDC fill varies by ~binomial(N/LC)
    got = ones / (len(probes) * k)
    assert abs(got - psu) < 0.25 * psu


# ------------------------------------------------- Sec. 5.1 sliding window --
def test_sliding_boundary_worked_example():
    """The Sec. 5.1 example, by exact counts (Def. 1, Def. 2)."""
    spec = {ln[0]: ln[1:] for ln in _golden_lines("sliding_boundary_example.txt")}
    theta, k = int(spec["theta"][0]), int(spec["slices_per_window"][0])
    per = [int(x) for x in spec["peers_per_slice"]]
    rng = np.random.default_rng(245)
    aip = 0xC0A80042
    slices = []
    for n in per:
        bg = W.uniform_pairs(3000, seed=int(rng.integers(1 << 30)), n_hosts=500)
        own = np.stack([np.full(n, aip, np.uint32), rng.integers(0, 2**32, n, dtype=np.uint32)], 1)
        slices.append(np.concatenate([bg, own]))
    dw1 = O.window_pairs(slices, k - 1, k)
    dw2 = O.window_pairs(slices, 2 * k - 1, k)
    tw = O.window_pairs(slices, k + 1, k)
    for pairs, want in ((dw1, spec["expect_dw1"]), (dw2, spec["expect_dw2"]), (tw, spec["expect_tw"])):
        assert (aip in set(O.exact_super_points(pairs, theta).tolist())) == bool(int(want[0]))


def test_window_pairs_definition():
    slices = [np.full((i + 1, 2), i, np.uint32) for i in range(6)]
    assert O.window_pairs(slices, 0, 3).shape == (1, 2)
    w = O.window_pairs(slices, 4, 3)
    assert sorted(set(w[:, 0].tolist())) == [2, 3, 4] and w.shape[0] == 3 + 4 + 5


def test_theorem1_is_the_argmin_of_lemma1():
    """Theorem 1's closed form equals a numeric minimisation (golden-section
    search) of Lemma 1's Psu over LR with LR * LC = V fixed."""
    for n, k_log2, v in [(1 << 26, 10, 1 << 18), (1 << 20, 8, 1 << 12), (5e6, 12, 3e5)]:
        f = lambda lr: O.psu(n, k_log2, lr, v / lr)   # noqa: E731
        lo, hi = 0.05, 200.0
        g = (math.sqrt(5) - 1) / 2
        for _ in range(200):
            a, b = hi - g * (hi - lo), lo + g * (hi - lo)
            if f(a) <= f(b):          # ties (the flat Psu = 1 tail) move inward
                hi = b
            else:
                lo = a
        assert abs((lo + hi) / 2 - O.lr_star(n, k_log2, v)) < 1e-4 * O.lr_star(n, k_log2, v)
    # at the optimum half the bits of one LDC are set: (1 - 1/k)^(N LR / V) = 1/2
    n, k_log2, v = 1 << 24, 10, 1 << 16
    lr = O.lr_star(n, k_log2, v)
    assert abs((1 - 2.0 ** -k_log2) ** (n * lr / v) - 0.5) < 1e-12
