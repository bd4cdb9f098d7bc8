"""GPU tests of the continuous-batching server: every window's global
detection equals the oracle on the window's requests; the batched engine
and the plain one-launch-per-request path give the same results (each result
is the same in the mix and alone); admission never exceeds the budget."""
import numpy as np
import pytest

import oracle as O
from paper_1901_07306_gb300 import workloads as W

pytestmark = pytest.mark.gpu

HEAVY = np.array([0x0A000001, 0x0A000102, 0xC0A80003, 0xAC100004, 0x08080805], np.uint32)


def _stream(router, n, seed):
    """Uniform background plus 20% of pairs from five heavy hosts."""
    rng = np.random.default_rng(seed)
    pairs = W.uniform_pairs(n, seed=seed, n_hosts=max(1, n // 4))
    k = n // 5
    pairs[:k, 0] = HEAVY[rng.integers(0, len(HEAVY), k)]
    return pairs


@pytest.fixture(scope="module")
def serving():
    from paper_1901_07306_gb300 import build
    build.build()
    from paper_1901_07306_gb300 import serving as mod
    return mod


def _requests(serving, seed=7, n=120, lo=8, hi=14, rate=5e8):
    return serving.poisson_requests(seed, n_routers=8, n_requests=n, rate_pairs_per_s=rate, lo_log2=lo, hi_log2=hi,
                                    streams=_stream)


def _clone(serving, reqs):
    return [serving.Request(router=r.router, pairs=r.pairs, arrival=r.arrival) for r in reqs]


def _oracle_window(reqs, windows, params):
    mine = [r.pairs.numpy().view(np.uint32).reshape(-1, 2) for r in reqs if r.window in windows]
    return O.Sketch(params).update(np.concatenate(mine)).detect()


PARAMS = dict(theta=64, seed=77)


def test_windows_match_oracle_and_plain_path(serving):
    reqs = _requests(serving)
    total = sum(r.n_pairs for r in reqs)
    srv = serving.SketchServer(8, PARAMS, budget_bytes=8 << 20, detect_every=total // 4 + 1)
    try:
        wins = srv.run(reqs)
    finally:
        srv.close()
    assert len(wins) >= 4 and all(np.isfinite(r.t_result) for r in reqs)
    op = O.Params(**PARAMS)
    for w in wins:
        want, n, _ = _oracle_window(reqs, {w.index}, op)
        assert w.n_found == n
        assert np.array_equal(w.records["ip"], want["ip"]) and np.array_equal(w.records["z0"], want["z0"])
        assert set(HEAVY.tolist()) <= set(w.records["ip"].tolist())
    plain_reqs = _clone(serving, reqs)
    srv = serving.SketchServer(8, PARAMS, budget_bytes=8 << 20, detect_every=total // 4 + 1, batched=False)
    try:
        plain = srv.run(plain_reqs)
    finally:
        srv.close()
    assert [r.window for r in plain_reqs] == [r.window for r in reqs]
    for a, b in zip(wins, plain):
        assert a.n_found == b.n_found and np.array_equal(a.records, b.records)


def test_budget_bounds_admission(serving):
    reqs = _requests(serving, seed=8, n=60, lo=10, hi=16, rate=1e12)   # everything arrives at once
    budget = 2 << 20
    srv = serving.SketchServer(8, PARAMS, budget_bytes=budget, detect_every=1 << 40)
    seen = []
    orig_take = srv.budget.take

    def take(nbytes):
        orig_take(nbytes)
        seen.append(srv.budget.in_use)
    assert len(seen) == 0
    srv.budget.take = take
    try:
        wins = srv.run(reqs)
    finally:
        srv.close()
    assert len(seen) == len(reqs) and max(seen) <= budget and len(wins) == 1
    want, n, _ = _oracle_window(reqs, {0}, O.Params(**PARAMS))
    assert wins[0].n_found == n and np.array_equal(wins[0].records["ip"], want["ip"])
    with pytest.raises(ValueError):
        srv2 = serving.SketchServer(2, PARAMS, budget_bytes=1024)
        try:
            srv2.run(_requests(serving, seed=9, n=2, lo=10, hi=11))
        finally:
            srv2.close()


def test_sliding_windows(serving):
    reqs = _requests(serving, seed=10, n=100)
    total = sum(r.n_pairs for r in reqs)
    srv = serving.SketchServer(8, PARAMS, budget_bytes=8 << 20, detect_every=total // 6 + 1, window_slices=3)
    try:
        wins = srv.run(reqs)
    finally:
        srv.close()
    op = O.Params(**PARAMS)
    for w in wins:
        want, n, _ = _oracle_window(reqs, {w.index - 2, w.index - 1, w.index}, op)
        assert w.n_found == n and np.array_equal(w.records["ip"], want["ip"])


def test_batched_engine_reads_requests_in_place(serving):
    """The batched engine scans each request where it lies: device tensors
    give the same windows as pinned host tensors, and a pageable host tensor
    (not guaranteed readable by the device) is refused before any launch."""
    reqs = _requests(serving, seed=11, n=40)
    total = sum(r.n_pairs for r in reqs)
    kw = dict(budget_bytes=8 << 20, detect_every=total // 3 + 1)
    srv = serving.SketchServer(8, PARAMS, **kw)
    try:
        host = srv.run(reqs)
        on_dev = [serving.Request(router=r.router, pairs=r.pairs.cuda(), arrival=r.arrival) for r in reqs]
        dev = srv.run(on_dev)
    finally:
        srv.close()
    assert len(host) == len(dev) >= 3
    for a, b in zip(host, dev):
        assert a.n_found == b.n_found and np.array_equal(a.records, b.records)
    pageable = [serving.Request(router=r.router, pairs=r.pairs.clone(), arrival=r.arrival) for r in reqs[:4]]
    assert not pageable[0].pairs.is_pinned()
    srv = serving.SketchServer(8, PARAMS, **kw)
    try:
        with pytest.raises(ValueError):
            srv.run(pageable)
    finally:
        srv.close()
