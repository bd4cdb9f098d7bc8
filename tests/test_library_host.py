"""Host-side checks of the C ABI library: it builds, loads, exports every
entry point include/superpoint.h declares, and its host logic (parameter
validation, Eq. 1, the integer form of Eq. 4, sizes) agrees with the
paper's closed forms.  No GPU compute is issued here."""
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def sp():
    from paper_1901_07306_gb300 import build
    build.build()
    from paper_1901_07306_gb300 import sp as mod
    return mod


def _declared():
    text = open(os.path.join(ROOT, "include", "superpoint.h")).read()
    return sorted(set(re.findall(r"^SP_API [\w\s\*]+?\b(sp_\w+)\(", text, flags=re.M)))


def test_exports_every_declared_symbol(sp):
    names = _declared()
    assert len(names) >= 20
    for name in names:
        assert hasattr(sp.lib, name), name
    assert set(names) == set(sp.EXPORTED)


def test_header_cites_the_paper():
    text = open(os.path.join(ROOT, "include", "superpoint.h")).read()
    for ref in ["Sec. 3.1", "Sec. 3.2", "Sec. 3.3", "Sec. 4.1", "Sec. 4.2", "Sec. 5", "Eq. 1", "Eq. 2",
                "Eq. 3", "Eq. 4"]:
        assert ref in text, ref


def test_version_and_strerror(sp):
    assert sp.lib.sp_version() >= 10000
    assert sp.lib.sp_strerror(sp.SP_ERR_CANDIDATE_OVERFLOW).decode().startswith("candidate")
    assert sp.lib.sp_strerror(12345).decode() == "unknown status"


def test_default_profile(sp):
    p = sp.sp_default_params()
    assert (p.r, p.sr, list(p.isb[:4]), list(p.ibn[:4])) == (14, 4, [0, 5, 10, 15], [7, 7, 7, 7])
    assert (p.k_log2, p.lr, p.lc_log2, p.theta, p.n_routers, p.window_slices) == (10, 4, 16, 1024, 1, 1)
    assert sp.sp_sketch_bytes(p) == (8 << 20, 32 << 20)
    assert sp.sp_check_params(p) == 0


def test_tau_and_z_theta(sp):
    for theta in list(range(1, 3000)) + [2**31, 2**32 - 1]:
        assert sp.sp_tau(theta) == max(0, (theta - 1).bit_length() - 3)
    assert sp.sp_z_theta(10, 1024) == 376
    for k_log2 in (5, 8, 10, 12, 16):
        k = 1 << k_log2
        for thr in (1, 7, 100, 1024, 4000, 10**5):
            b = k * math.exp(-thr / k)
            if abs(b - round(b)) > 1e-9:
                assert sp.sp_z_theta(k_log2, thr) == math.floor(b)


def test_param_validation_matches_oracle(sp):
    import oracle as O
    cases = [
        dict(),
        dict(r=12, isb=(0, 7, 14), ibn=(8, 8, 8), k_log2=8, lr=3, lc_log2=6),
        dict(isb=(0, 5, 10), ibn=(7, 7, 7)),            # LP bit 17 uncovered
        dict(isb=(0, 7, 10, 15)),                      # rows 0, 1 share nothing
        dict(r=0, isb=(0, 8, 16, 24), ibn=(9, 9, 9, 9)),
        dict(r=0, isb=(0, 8, 16, 24), ibn=(8, 8, 8, 8)),  # covered, no overlap
        dict(r=24, isb=(0, 4), ibn=(5, 5)),
        dict(r=25, isb=(0,), ibn=(7,)),
        dict(isb=(0,), ibn=(12,), r=20),               # SR = 1 covering all 12 LP bits
        dict(k_log2=4), dict(k_log2=17), dict(lr=0, ), dict(lr=9), dict(theta=0),
        dict(ibn=(13, 7, 7, 7)),
    ]
    for kw in cases:
        o = O.Params(**{k: v for k, v in kw.items()})
        if o.lr < 1 or o.lr > 8:
            want_ok = False
        else:
            want_ok = O.check_params(o) == 0
        p = sp.make_params(**kw)
        assert (sp.sp_check_params(p) == 0) == want_ok, kw


def test_library_limits(sp):
    # SEA of more than 4096 bytes is a library limit, not a paper constraint
    p = sp.make_params(r=8, isb=(0, 12), ibn=(12, 12))
    assert sp.sp_check_params(p) == sp.SP_ERR_PARAM
    p = sp.make_params(lr=8, lc_log2=24, k_log2=10)    # 2^37 bits > 2^32
    assert sp.sp_check_params(p) == sp.SP_ERR_PARAM
    p = sp.make_params(n_routers=0)
    assert sp.sp_check_params(p) == sp.SP_ERR_PARAM


def test_ldca_sizing_matches_lemma1_and_theorem1(sp):
    import oracle as O
    for n, k_log2, budget in [(1 << 26, 10, 1 << 18), (1 << 20, 8, 1 << 12), (1 << 28, 10, 1 << 20), (5000, 6, 64)]:
        for lr in (1, 3, 4, 8):
            for c in (4, 10, 16):
                a, b = sp.sp_psu(n, k_log2, lr, c), O.psu(n, k_log2, lr, 2 ** c)
                assert abs(a - b) <= 1e-12 * max(b, 1e-300)
        lr, c, psu, star = sp.sp_size_ldca(n, k_log2, budget)
        assert abs(star - O.lr_star(n, k_log2, budget)) < 1e-9 * star
        grid = [(O.psu(n, k_log2, r, 2 ** cc), r, cc) for r in range(1, 9) for cc in range(25)
                if r * 2 ** cc <= budget and r * 2 ** (cc + k_log2) <= 2 ** 32]
        best = min(grid)
        assert (lr, c) == (best[1], best[2]) and abs(psu - best[0]) < 1e-15
        assert lr * 2 ** c <= budget
    with pytest.raises(sp.SPError):
        sp.sp_size_ldca(0, 10, 1 << 16)


def test_bounds_probe_library_exports_its_header():
    """libspbounds.so (the hardware probes behind the roofline figures) loads
    without a GPU and exports exactly what include/sp_bounds.h declares."""
    import ctypes
    from paper_1901_07306_gb300 import build
    build.build()
    text = open(os.path.join(ROOT, "include", "sp_bounds.h")).read()
    names = sorted(set(re.findall(r"^SPB_API [\w\s\*]+?\b(sp_\w+)\(", text, flags=re.M)))
    assert names == ["sp_probe_l2_red", "sp_probe_smem_atomic", "sp_probe_stream_read"]
    lib = ctypes.CDLL(build.BOUNDS_LIB)
    for name in names:
        assert hasattr(lib, name), name


def test_param_validation_agrees_with_oracle_on_random_profiles(sp):
    """The library's and the oracle's checks of the Sec. 3.2 constraints
    (coverage, cyclic overlap of consecutive rows) are written independently;
    on random SEAV profiles inside the library's limits they accept and
    reject the same sets."""
    import numpy as np
    import oracle as O
    rng = np.random.default_rng(123)
    accepted = rejected = 0
    for _ in range(3000):
        r = int(rng.integers(0, 25))
        L = 32 - r
        sr = int(rng.integers(1, 9))
        ibn = tuple(int(x) for x in rng.integers(1, min(12, L) + 1, sr))
        isb = tuple(int(x) for x in rng.integers(0, L, sr))
        if sum(1 << b for b in ibn) > 4096:                 # a library limit, not a paper constraint
            continue
        want = O.check_params(O.Params(r=r, isb=isb, ibn=ibn)) == 0
        got = sp.sp_check_params(sp.make_params(r=r, isb=isb, ibn=ibn)) == 0
        assert got == want, (r, isb, ibn)
        accepted += want
        rejected += not want
    assert accepted > 100 and rejected > 100
