"""The library's waits on its stream are bounded (sp_set_timeout): a detect
whose stream is held up returns SP_ERR_TIMEOUT from sp_results after the
bound, and the same detect is collected, bit-exact, once the stream moves.
The stream is held by a host function that waits on a flag set by the test
(at most 10 s): nothing runs or waits on the GPU meanwhile."""
import ctypes
import threading
import time

import numpy as np
import pytest

import oracle as O
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


def test_results_wait_is_bounded(sp, torch):
    libcuda = ctypes.CDLL("libcuda.so.1")
    hostfn = ctypes.CFUNCTYPE(None, ctypes.c_void_p)
    release = threading.Event()
    cb = hostfn(lambda _: release.wait(10.0))
    pairs, planted = W.single_window(seed=41, n=1 << 18, n_background=8192, n_planted=5, planted_degree=3000)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        flat = torch.from_numpy(pairs.reshape(-1).view(np.int32).copy()).cuda()
    with sp.SuperPoint(seed=41, stream=stream) as ctx:
        c = ctx.ctx
        sp.sp_update(c, 0, flat)
        assert libcuda.cuLaunchHostFunc(ctypes.c_void_p(stream.cuda_stream), cb, None) == 0
        sp.sp_detect_async(c, 0, 0)
        sp.sp_set_timeout(c, 200)
        t0 = time.perf_counter()
        try:
            with pytest.raises(sp.SPError) as e:
                sp.sp_results(c)
            dt = time.perf_counter() - t0
        finally:
            release.set()
        assert e.value.code == sp.SP_ERR_TIMEOUT and 0.2 <= dt < 5.0, (e.value.code, dt)
        sp.sp_set_timeout(c, 0)                               # unbounded again
        recs, n, rc = sp.sp_results(c)
        want, n_want, _ = O.Sketch(O.Params(seed=41)).update(pairs).detect()
        assert rc == sp.SP_OK and n == n_want
        assert np.array_equal(recs["ip"], want["ip"]) and np.array_equal(recs["z0"], want["z0"])
        assert set(planted.tolist()) <= set(recs["ip"].tolist())
    stream.synchronize()
