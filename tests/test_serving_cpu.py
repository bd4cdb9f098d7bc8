"""Host logic of the serving engine, driven by a stand-in for its device side
(no GPU): admission order and windows, the budget, and the failure detection
of its device waits -- a step's scan or a window's detection that never
completes makes ``run`` raise ``ServingTimeout`` once its bound has passed,
instead of waiting forever.  The stand-in's events are host objects, so
nothing here touches a GPU."""
import time

import numpy as np
import pytest
import torch

from paper_1901_07306_gb300 import serving as S


class FakeEvent:
    """Completes after `polls` queries; never when polls is None."""

    def __init__(self, polls):
        self.left = polls

    def query(self):
        if self.left is None:
            return False
        self.left -= 1
        return self.left < 0


class FakeOps:
    def __init__(self, hang_step=None, hang_window=None):
        self.hang_step, self.hang_window = hang_step, hang_window
        self.steps, self.windows = [], []

    def close(self):
        pass

    def synchronize(self):
        pass

    def issue_step(self, step):
        self.steps.append([id(r) for r in step])
        return FakeEvent(None if len(self.steps) - 1 == self.hang_step else 3)

    def close_window(self):
        i = len(self.windows)
        self.windows.append(i)
        return FakeEvent(None if i == self.hang_window else 2), i

    def read_window(self, handle):
        return handle + 100, np.zeros(0)


def _requests(n, size=64, gap=0.0):
    return [S.Request(router=i % 3, pairs=torch.zeros(2 * size, dtype=torch.int32), arrival=i * gap)
            for i in range(n)]


def test_windows_acks_and_budget_with_a_stand_in():
    reqs = _requests(40, size=64)
    budget = 64 * 8 * 5                                        # five requests in flight at most
    srv = S.SketchServer(3, budget_bytes=budget, detect_every=64 * 10, max_step_requests=4, ops=FakeOps())
    seen = []
    take = srv.budget.take
    srv.budget.take = lambda nb: (take(nb), seen.append(srv.budget.in_use))
    wins = srv.run(reqs)
    assert len(seen) == 40 and max(seen) <= budget
    assert [w.index for w in wins] == [0, 1, 2, 3] and [w.n_found for w in wins] == [100, 101, 102, 103]
    assert [r.window for r in reqs] == [i // 10 for i in range(40)]
    assert all(np.isfinite(r.t_ack) and np.isfinite(r.t_result) for r in reqs)
    # steps hold 1 to 4 requests and issue every request once, in arrival order
    assert all(1 <= len(st) <= 4 for st in srv.ops.steps)
    assert [x for st in srv.ops.steps for x in st] == [id(r) for r in reqs]


@pytest.mark.parametrize("hang", ["step", "window"])
def test_a_wait_that_never_completes_raises_after_its_bound(hang):
    ops = FakeOps(hang_step=2 if hang == "step" else None, hang_window=0 if hang == "window" else None)
    srv = S.SketchServer(3, budget_bytes=1 << 20, detect_every=64 * 6, max_step_requests=2, timeout_s=0.25,
                         ops=ops)
    t0 = time.perf_counter()
    with pytest.raises(S.ServingTimeout) as e:
        srv.run(_requests(12))
    dt = time.perf_counter() - t0
    assert 0.25 <= dt < 5.0
    assert ("scan of step 2" in str(e.value)) if hang == "step" else ("detection of window 0" in str(e.value))


def test_request_larger_than_the_budget_is_refused():
    srv = S.SketchServer(1, budget_bytes=64 * 8 - 4, ops=FakeOps())
    with pytest.raises(ValueError):
        srv.run(_requests(1, size=64))


class JitterOps(FakeOps):
    """Device events that complete after a random number of polls."""

    def __init__(self, seed):
        super().__init__()
        self.rng = np.random.default_rng(seed)

    def issue_step(self, step):
        self.steps.append([id(r) for r in step])
        return FakeEvent(int(self.rng.integers(0, 40)))

    def close_window(self):
        i = len(self.windows)
        self.windows.append(i)
        return FakeEvent(int(self.rng.integers(0, 40))), i


def test_windows_depend_only_on_arrival_order():
    """How fast the device completes steps changes how requests are grouped
    into steps, never which window a request belongs to or the windows'
    pair counts (a window closes after detect_every admitted pairs)."""
    sizes = np.random.default_rng(5).integers(16, 200, 60)
    runs = []
    for seed in range(4):
        reqs = [S.Request(router=i % 5, pairs=torch.zeros(2 * int(n), dtype=torch.int32), arrival=0.0)
                for i, n in enumerate(sizes)]
        srv = S.SketchServer(5, budget_bytes=8 * 400, detect_every=1000, max_step_requests=3,
                             ops=JitterOps(seed))
        wins = srv.run(reqs)
        runs.append(([r.window for r in reqs], [w.n_pairs for w in wins]))
    assert all(r == runs[0] for r in runs[1:])
    windows, pairs = runs[0]
    assert sum(pairs) == int(sizes.sum()) and all(p >= 1000 for p in pairs[:-1])
