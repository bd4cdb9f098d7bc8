"""CPU oracle of the SLGA super point scheme (arXiv 1901.07306).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline legs of ``bench.py`` may import this package.  The product path
(``paper_1901_07306_gb300``) never imports it and shares no code with it.

The arithmetic lives in ``sp_oracle.c`` (plain single-threaded C, the paper's
steps in the paper's order); this module only loads it with ``ctypes`` and
marshals numpy arrays.  ``exact_opposite_counts`` is the problem's own
definition (Def. 1 and Def. 2, Sec. 3), written with numpy's sort-unique.

Parity status: every function is pinned by ``tests/test_oracle_*.py``
(closed forms, brute force on tiny inputs, structural invariants and
statistical checks of Eq. 4 and Lemma 1).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sp_oracle.c")
_LIB = os.path.join(_HERE, "_sp_oracle.so")

FLAG_SATURATED = 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, no target-specific flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [
        ("r", ctypes.c_uint32),
        ("sr", ctypes.c_uint32),
        ("isb", ctypes.c_uint32 * 8),
        ("ibn", ctypes.c_uint32 * 8),
        ("k_log2", ctypes.c_uint32),
        ("lr", ctypes.c_uint32),
        ("lc_log2", ctypes.c_uint32),
        ("theta", ctypes.c_uint32),
        ("seed", ctypes.c_uint64),
    ]


CANDIDATE_DTYPE = np.dtype(
    [("ip", "<u4"), ("z0", "<u4"), ("est", "<f8"), ("flags", "<u4"), ("pad", "<u4")]
)

_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        u32, u64, p = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_void_p
        PP = ctypes.POINTER(_Params)
        sigs = {
            "or_tau": (u32, [u32]),
            "or_lsb": (u32, [u32]),
            "or_popcount": (u32, [u64]),
            "or_splitmix64": (u64, [ctypes.POINTER(u64)]),
            "or_mas": (u32, [u64, u64, u32]),
            "or_hash_params": (None, [u64, u32, p, p]),
            "or_h1": (u32, [p, p, u32]),
            "or_h2": (u32, [u32]),
            "or_h3": (u32, [p, p, u32, u32]),
            "or_lh": (u32, [p, p, u32, u32, u32]),
            "or_rp": (u32, [u32, u32]),
            "or_lp": (u32, [u32, u32]),
            "or_idx": (u32, [PP, u32, u32]),
            "or_sea_bytes": (u64, [PP]),
            "or_seav_bytes": (u64, [PP]),
            "or_ldca_words": (u64, [PP]),
            "or_check_params": (ctypes.c_int, [PP]),
            "or_update": (None, [PP, p, p, p, u64]),
            "or_merge": (None, [p, p, u64]),
            "or_est": (ctypes.c_double, [u32, u32]),
            "or_z_theta": (u32, [u32, u32]),
            "or_detect": (ctypes.c_int, [PP, p, p, u32, p, u64, ctypes.POINTER(u64)]),
            "or_psu": (ctypes.c_double, [ctypes.c_double, u32, ctypes.c_double, ctypes.c_double]),
            "or_lr_star": (ctypes.c_double, [ctypes.c_double, u32, ctypes.c_double]),
        }
        for name, (res, args) in sigs.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


@dataclass
class Params:
    """SLGA parameters (Sec. 3.2 SEAV, Sec. 3.3 LDCA, Eq. 1 theta)."""

    r: int = 14
    isb: tuple = (0, 5, 10, 15)
    ibn: tuple = (7, 7, 7, 7)
    k_log2: int = 10
    lr: int = 4
    lc_log2: int = 16
    theta: int = 1024
    seed: int = 0x5EED

    @property
    def sr(self) -> int:
        return len(self.isb)

    def _c(self) -> _Params:
        c = _Params()
        c.r, c.sr = self.r, self.sr
        for i in range(self.sr):
            c.isb[i], c.ibn[i] = self.isb[i], self.ibn[i]
        c.k_log2, c.lr, c.lc_log2 = self.k_log2, self.lr, self.lc_log2
        c.theta, c.seed = self.theta, self.seed & (2**64 - 1)
        return c


def tau(theta: int) -> int:
    return _load().or_tau(theta)


def lsb(x: int) -> int:
    return _load().or_lsb(x)


def mas(a: int, b: int, x: int) -> int:
    return _load().or_mas(a, b, x)


def hash_params(seed: int, lr: int):
    a = np.zeros(2 + lr, np.uint64)
    b = np.zeros(2 + lr, np.uint64)
    _load().or_hash_params(seed & (2**64 - 1), lr, a.ctypes.data, b.ctypes.data)
    return a, b


def splitmix64_stream(seed: int, n: int):
    s = ctypes.c_uint64(seed & (2**64 - 1))
    return [_load().or_splitmix64(ctypes.byref(s)) for _ in range(n)]


def h1(p: Params, oip: int) -> int:
    a, b = hash_params(p.seed, p.lr)
    return _load().or_h1(a.ctypes.data, b.ctypes.data, oip)


def h3(p: Params, oip: int) -> int:
    a, b = hash_params(p.seed, p.lr)
    return _load().or_h3(a.ctypes.data, b.ctypes.data, p.k_log2, oip)


def lh(p: Params, i: int, hip: int) -> int:
    a, b = hash_params(p.seed, p.lr)
    return _load().or_lh(a.ctypes.data, b.ctypes.data, p.lc_log2, i, hip)


def rp(r: int, ip: int) -> int:
    return _load().or_rp(r, ip)


def lp(r: int, ip: int) -> int:
    return _load().or_lp(r, ip)


def idx(p: Params, i: int, lp_value: int) -> int:
    c = p._c()
    return _load().or_idx(ctypes.byref(c), i, lp_value)


def check_params(p: Params) -> int:
    c = p._c()
    return _load().or_check_params(ctypes.byref(c))


def seav_bytes(p: Params) -> int:
    c = p._c()
    return _load().or_seav_bytes(ctypes.byref(c))


def sea_bytes(p: Params) -> int:
    c = p._c()
    return _load().or_sea_bytes(ctypes.byref(c))


def ldca_words(p: Params) -> int:
    c = p._c()
    return _load().or_ldca_words(ctypes.byref(c))


def est(k_log2: int, z0: int) -> float:
    return _load().or_est(k_log2, z0)


def psu(n_pairs: float, k_log2: int, lr: float, lc: float) -> float:
    """Lemma 1."""
    return _load().or_psu(float(n_pairs), k_log2, float(lr), float(lc))


def lr_star(n_pairs: float, k_log2: int, v_ldcs: float) -> float:
    """Theorem 1."""
    return _load().or_lr_star(float(n_pairs), k_log2, float(v_ldcs))


def z_theta(k_log2: int, theta: int) -> int:
    return _load().or_z_theta(k_log2, theta)


@dataclass
class Sketch:
    """One watch point's SEAV (bytes, SEA-major) and LDCA (uint32 words)."""

    params: Params
    seav: np.ndarray = field(default=None)
    ldca: np.ndarray = field(default=None)

    def __post_init__(self):
        if check_params(self.params) != 0:
            raise ValueError(f"invalid parameters (code {check_params(self.params)})")
        if self.seav is None:
            self.seav = np.zeros(seav_bytes(self.params), np.uint8)
        if self.ldca is None:
            self.ldca = np.zeros(ldca_words(self.params), np.uint32)

    def update(self, pairs: np.ndarray) -> "Sketch":
        pairs = np.ascontiguousarray(pairs, dtype=np.uint32).reshape(-1)
        assert pairs.size % 2 == 0
        c = self.params._c()
        _load().or_update(ctypes.byref(c), self.seav.ctypes.data, self.ldca.ctypes.data,
                          pairs.ctypes.data, pairs.size // 2)
        return self

    def merge(self, other: "Sketch") -> "Sketch":
        _load().or_merge(self.seav.ctypes.data, other.seav.ctypes.data, self.seav.nbytes)
        _load().or_merge(self.ldca.ctypes.data, other.ldca.ctypes.data, self.ldca.nbytes)
        return self

    def copy(self) -> "Sketch":
        return Sketch(self.params, self.seav.copy(), self.ldca.copy())

    def detect(self, threshold: int | None = None, cap: int | None = None):
        """Returns (candidates sorted by IP, total count, overflowed)."""
        threshold = self.params.theta if threshold is None else threshold
        c = self.params._c()
        n_total = ctypes.c_uint64(0)
        _load().or_detect(ctypes.byref(c), self.seav.ctypes.data, self.ldca.ctypes.data,
                          threshold, None, 0, ctypes.byref(n_total))
        n = n_total.value
        out = np.zeros(max(n, 1), CANDIDATE_DTYPE)
        lim = n if cap is None else min(n, cap)
        rc = _load().or_detect(ctypes.byref(c), self.seav.ctypes.data, self.ldca.ctypes.data,
                               threshold, out.ctypes.data, lim, ctypes.byref(n_total))
        return out[:lim], n, rc != 0


def exact_opposite_counts(pairs: np.ndarray):
    """Def. 1: |OP(h)| for every hip h in the stream (hip = first of each pair).

    Returns (hosts ascending, counts) computed by sort-unique of the 64-bit
    keys hip << 32 | oip.
    """
    pairs = np.asarray(pairs, dtype=np.uint32).reshape(-1, 2)
    keys = (pairs[:, 0].astype(np.uint64) << np.uint64(32)) | pairs[:, 1].astype(np.uint64)
    keys = np.unique(keys)
    hips = (keys >> np.uint64(32)).astype(np.uint32)
    hosts, counts = np.unique(hips, return_counts=True)
    return hosts, counts


def exact_super_points(pairs: np.ndarray, theta: int) -> np.ndarray:
    """Def. 2: the hosts h with |OP(h)| >= theta, ascending."""
    hosts, counts = exact_opposite_counts(pairs)
    return hosts[counts >= theta]


def window_pairs(slices, t: int, k: int) -> np.ndarray:
    """Sec. 5.1: the sliding window W(t, k) holds the k successive slices
    ending at slice t (fewer at the start of the stream)."""
    part = [np.asarray(s, np.uint32).reshape(-1, 2) for s in slices[max(0, t - k + 1):t + 1]]
    return np.concatenate(part) if part else np.empty((0, 2), np.uint32)


def sliding_window_sketch(params: Params, slices, t: int, k: int) -> Sketch:
    """The sketch a sliding counter pool must expose at slice t (Sec. 5.2:
    an active counter reads as bit 1): the discrete sketch of W(t, k)."""
    return Sketch(params).update(window_pairs(slices, t, k))
