"""Seeded synthetic IP-pair streams shaped like core-link captures.

This module draws inputs only: it holds none of the detection scheme's
arithmetic (no hashing, no sketch), so both the CUDA path and the CPU oracle
can be fed from it.  Every stream is a C-contiguous ``uint32`` array of shape
``(n, 2)`` holding ``(hip, oip)`` = (src IP, dst IP) pairs; the monitored
host is the source (Sec. 3, "<hip, oip>").

Generators use numpy's PCG64 ``default_rng(seed)``, whose integer streams are
identical on x86-64 and aarch64.  Ground truth is always recomputed from the
emitted stream, never taken from a generator's intent.

Workloads (the paper measured CAIDA OC192 traces, which these stand in for):
  * ``single_window``     -- 2^20 pairs, 65,536 background sources with
    Zipf(1.2) out-degree on [1, 200], 20 planted super points x 3,000 peers,
    shuffled and cut to exactly n pairs.
  * ``core_link``         -- 2^26 pairs, ~4M sources with Zipf(1.1) degrees
    (cap fitted so distinct pairs = 0.9 n), 500 planted super points with
    log-uniform degree in [1,500, 50,000], 10% duplicate pairs, shuffled.
  * ``distributed``       -- 16 routers x 2^24 pairs from an overlapping host
    population (30% shared sources); 1,000 global super points whose peers
    are split evenly so that no single router sees theta of them.
  * ``sliding_stream``    -- time slices of lognormal size, super points
    switching on and off per slice, background hosts one per 64 pairs of the
    stream (for the sliding-window extension).
  * ``uniform_pairs``     -- i.i.d. uniform pairs for small tests.
"""
from __future__ import annotations

import numpy as np


def uniform_pairs(n: int, seed: int, n_hosts: int | None = None) -> np.ndarray:
    """n i.i.d. pairs; hips drawn from ``n_hosts`` random hosts if given."""
    rng = np.random.default_rng(seed)
    out = np.empty((n, 2), np.uint32)
    if n_hosts is None:
        out[:, 0] = rng.integers(0, 2**32, n, dtype=np.uint32)
    else:
        hosts = rng.integers(0, 2**32, n_hosts, dtype=np.uint32)
        out[:, 0] = hosts[rng.integers(0, n_hosts, n)]
    out[:, 1] = rng.integers(0, 2**32, n, dtype=np.uint32)
    return out


def _distinct_hosts(rng, n: int, exclude: np.ndarray | None = None) -> np.ndarray:
    """n distinct uniform uint32 host addresses, none in ``exclude``."""
    got = np.empty(0, np.uint32)
    while got.size < n:
        draw = rng.integers(0, 2**32, int((n - got.size) * 1.05) + 16, dtype=np.uint32)
        got = np.unique(np.concatenate([got, draw]))
        if exclude is not None and exclude.size:
            got = got[~np.isin(got, exclude)]
    # random subset of the required size, in random order
    return rng.permutation(got)[:n]


def _zipf_degrees(rng, n: int, s: float, cap: int) -> np.ndarray:
    """n draws of a Zipf(s) law truncated to [1, cap] (inverse-CDF)."""
    k = np.arange(1, cap + 1, dtype=np.float64)
    cdf = np.cumsum(k ** (-s))
    cdf /= cdf[-1]
    u = rng.random(n)
    return np.minimum(np.searchsorted(cdf, u, side="right") + 1, cap).astype(np.int64)


def _zipf_mean(s: float, cap: int) -> float:
    k = np.arange(1, cap + 1, dtype=np.float64)
    w = k ** (-s)
    return float((k * w).sum() / w.sum())


def _expand(rng, hosts: np.ndarray, degrees: np.ndarray) -> np.ndarray:
    """Pairs (host, uniform random peer), each host repeated degree times."""
    hip = np.repeat(hosts.astype(np.uint32), degrees)
    oip = rng.integers(0, 2**32, hip.size, dtype=np.uint32)
    return np.stack([hip, oip], axis=1)


def _distinct_peers(rng, d: int) -> np.ndarray:
    peers = np.unique(rng.integers(0, 2**32, d + d // 8 + 16, dtype=np.uint32))
    while peers.size < d:
        peers = np.unique(np.concatenate([peers, rng.integers(0, 2**32, d, dtype=np.uint32)]))
    return rng.permutation(peers)[:d]


def _rows(pairs: np.ndarray, idx: np.ndarray) -> np.ndarray:
    """pairs[idx] for an (n, 2) uint32 array, gathered as 64-bit rows (the
    same values as 2-D fancy indexing, about three times faster)."""
    flat = np.ascontiguousarray(pairs, np.uint32).view(np.uint64).reshape(-1)
    return flat[idx].view(np.uint32).reshape(-1, 2)


def _fit_to(rng, pairs: np.ndarray, n: int) -> np.ndarray:
    """Shuffle, then truncate to n pairs or pad with duplicates of emitted pairs."""
    pairs = _rows(pairs, rng.permutation(pairs.shape[0]))
    if pairs.shape[0] >= n:
        return np.ascontiguousarray(pairs[:n])
    extra = _rows(pairs, rng.integers(0, pairs.shape[0], n - pairs.shape[0]))
    out = np.concatenate([pairs, extra])
    return _rows(out, rng.permutation(n))


def single_window(seed: int = 1, n: int = 1 << 20, n_background: int = 65536,
                  n_planted: int = 20, planted_degree: int = 3000):
    """Single router, one window.  Returns (pairs, planted hosts)."""
    rng = np.random.default_rng(seed)
    background = _distinct_hosts(rng, n_background)
    planted = _distinct_hosts(rng, n_planted, exclude=background)
    bg = _expand(rng, background, _zipf_degrees(rng, n_background, 1.2, 200))
    sp = np.concatenate([
        np.stack([np.full(planted_degree, h, np.uint32), _distinct_peers(rng, planted_degree)], 1)
        for h in planted
    ]) if n_planted else np.empty((0, 2), np.uint32)
    pairs = _fit_to(rng, np.concatenate([bg, sp]), n)
    return pairs, np.sort(planted)


def core_link(seed: int = 2, n: int = 1 << 26, n_sources: int | None = None,
              n_planted: int | None = None, dup_frac: float = 0.10,
              planted_range=(1500, 50000)):
    """Single router shaped like a core-link capture.  Returns (pairs, planted)."""
    rng = np.random.default_rng(seed)
    scale = n / float(1 << 26)
    n_sources = int(round(4_000_000 * scale)) if n_sources is None else n_sources
    n_planted = max(1, int(round(500 * scale))) if n_planted is None else n_planted
    n_distinct = int(round(n * (1.0 - dup_frac)))
    lo, hi = planted_range
    planted_deg = np.exp(rng.uniform(np.log(lo), np.log(hi), n_planted)).astype(np.int64)
    bg_total = max(n_distinct - int(planted_deg.sum()), n_sources)
    # fit the Zipf cap so that the expected background degree sum matches
    target = bg_total / n_sources
    cap_lo, cap_hi = 1, 1 << 20
    while cap_lo < cap_hi:
        mid = (cap_lo + cap_hi) // 2
        if _zipf_mean(1.1, mid) < target:
            cap_lo = mid + 1
        else:
            cap_hi = mid
    sources = _distinct_hosts(rng, n_sources)
    planted = _distinct_hosts(rng, n_planted, exclude=sources)
    bg = _expand(rng, sources, _zipf_degrees(rng, n_sources, 1.1, cap_lo))
    bg = _rows(bg, rng.permutation(bg.shape[0]))[: max(0, n_distinct - int(planted_deg.sum()))]
    sp = np.concatenate([
        np.stack([np.full(d, h, np.uint32), _distinct_peers(rng, int(d))], 1)
        for h, d in zip(planted, planted_deg)
    ])
    distinct = np.concatenate([bg, sp])
    dups = _rows(distinct, rng.integers(0, distinct.shape[0], n - distinct.shape[0]))
    pairs = np.concatenate([distinct, dups])
    pairs = _rows(pairs, rng.permutation(pairs.shape[0]))
    return pairs, np.sort(planted)


def distributed(seed: int = 3, n_routers: int = 16, n_per_router: int = 1 << 24,
                n_global_sp: int = 1000, shared_frac: float = 0.30,
                sp_range=(1500, 8000), theta: int = 1024):
    """Routers sharing a host population.  Returns (list of pair arrays, sp hosts)."""
    rng = np.random.default_rng(seed)
    scale = n_per_router / float(1 << 24)
    per_router_sources = max(16, int(round(1_000_000 * scale)))
    n_shared = int(per_router_sources * shared_frac)
    n_private = per_router_sources - n_shared
    shared = _distinct_hosts(rng, n_shared)
    sp_hosts = _distinct_hosts(rng, n_global_sp, exclude=shared)
    sp_deg = rng.integers(sp_range[0], sp_range[1] + 1, n_global_sp)
    # split every super point's peers evenly over the routers
    sp_parts = [[] for _ in range(n_routers)]
    for h, d in zip(sp_hosts, sp_deg):
        peers = _distinct_peers(rng, int(d))
        for r, chunk in enumerate(np.array_split(peers, n_routers)):
            assert chunk.size < theta
            sp_parts[r].append(np.stack([np.full(chunk.size, h, np.uint32), chunk], 1))
    routers = []
    for r in range(n_routers):
        private = _distinct_hosts(rng, n_private, exclude=sp_hosts)
        hosts = np.concatenate([shared, private])
        sp = np.concatenate(sp_parts[r]) if sp_parts[r] else np.empty((0, 2), np.uint32)
        room = n_per_router - sp.shape[0]
        cap = 1
        while _zipf_mean(1.1, cap) < room / hosts.size and cap < (1 << 20):
            cap += max(1, cap // 8)
        bg = _expand(rng, hosts, _zipf_degrees(rng, hosts.size, 1.1, cap))
        routers.append(_fit_to(rng, np.concatenate([bg[: max(0, room)], sp]), n_per_router))
    return routers, np.sort(sp_hosts)


def slice_sizes(seed: int, n_slices: int = 128, total: int = 1 << 28,
                lo: int = 1 << 19, hi: int = 1 << 22) -> np.ndarray:
    """Lognormal slice sizes clipped to [lo, hi], rescaled to sum to total."""
    rng = np.random.default_rng(seed)
    mean = total / n_slices
    raw = rng.lognormal(np.log(mean) - 0.5 * 0.6**2, 0.6, n_slices)
    sizes = np.clip(raw, lo, hi)
    for _ in range(64):
        sizes = np.clip(sizes * (total / sizes.sum()), lo, hi)
    sizes = np.floor(sizes).astype(np.int64)
    # put the rounding remainder where it still fits under hi
    rem = total - int(sizes.sum())
    i = 0
    while rem != 0 and i < 16 * n_slices:
        j = i % n_slices
        step = 1 if rem > 0 else -1
        if lo <= sizes[j] + step <= hi:
            sizes[j] += step
            rem -= step
        i += 1
    return sizes


def sliding_stream(seed: int = 4, sizes: np.ndarray | None = None, n_sp: int = 64,
                   sp_degree_per_slice=(64, 512), n_background: int | None = None):
    """Slices for the sliding-window extension (Sec. 5).

    Returns (list of per-slice pair arrays, schedule) where ``schedule`` is a
    bool array [n_sp, n_slices] telling when each planted host is active, and
    the planted hosts are ``schedule_hosts``.
    """
    rng = np.random.default_rng(seed)
    sizes = slice_sizes(seed) if sizes is None else np.asarray(sizes)
    n_slices = sizes.size
    # background hosts as dense as on the core link: one per 64 pairs of the
    # stream (4M at 2^28 pairs), so a 32-slice window of 2^26 pairs gives each
    # about 16 pairs
    n_background = n_background or max(1024, int(sizes.sum() // 64))
    hosts = _distinct_hosts(rng, n_background)
    sp_hosts = _distinct_hosts(rng, n_sp, exclude=hosts)
    schedule = np.zeros((n_sp, n_slices), bool)
    for s in range(n_sp):
        start = int(rng.integers(0, n_slices))
        length = int(rng.integers(1, max(2, n_slices // 2)))
        schedule[s, start:start + length] = True
    slices = []
    for t in range(n_slices):
        parts = []
        for s in np.nonzero(schedule[:, t])[0]:
            d = int(rng.integers(sp_degree_per_slice[0], sp_degree_per_slice[1] + 1))
            parts.append(np.stack([np.full(d, sp_hosts[s], np.uint32),
                                   rng.integers(0, 2**32, d, dtype=np.uint32)], 1))
        sp = np.concatenate(parts) if parts else np.empty((0, 2), np.uint32)
        room = int(sizes[t]) - sp.shape[0]
        bg = np.stack([hosts[rng.integers(0, hosts.size, room)],
                       rng.integers(0, 2**32, room, dtype=np.uint32)], 1)
        both = np.concatenate([bg, sp])
        slices.append(_rows(both, rng.permutation(both.shape[0])))
    return slices, sp_hosts, schedule
