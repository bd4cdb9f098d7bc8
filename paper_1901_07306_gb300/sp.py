"""Thin ctypes binding of libsuperpoint (include/superpoint.h).

Argument marshalling only: every step of the scan, merge and detect runs in
the library's CUDA kernels.  The functions keep the C names (sp_create,
sp_update, ...); ``SuperPoint`` wraps one context for convenience.  PyTorch
supplies device memory (pair tensors) and streams.

The library must be built (``paper_1901_07306_gb300.build.build()``); if it
is missing or fails to load this module raises at import -- there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsuperpoint.so")

SP_OK = 0
SP_WARN_THETA_BELOW_INIT = 1
SP_ERR_PARAM = -1
SP_ERR_ROUTER = -2
SP_ERR_TRUNCATED = -3
SP_ERR_CANDIDATE_OVERFLOW = -4
SP_ERR_CUDA = -5
SP_ERR_TIMEOUT = -6
SP_ERR_CHECKSUM = -7
SP_ERR_NOMEM = -8
SP_ERR_STATE = -9
SP_FLAG_SATURATED = 1
SP_SCAN_AUTO, SP_SCAN_DIRECT, SP_SCAN_BINNED = 0, 1, 2
SP_NOALLOC_MAX_RESULTS = 65536
SP_NOALLOC_MAX_K_LOG2 = 12

EXPORTED = (
    "sp_version", "sp_strerror", "sp_default_params", "sp_check_params", "sp_sketch_bytes",
    "sp_tau", "sp_z_theta", "sp_create", "sp_destroy", "sp_set_stream", "sp_get_params",
    "sp_reset", "sp_update", "sp_update_host", "sp_update_batched", "sp_merge",
    "sp_detect_async", "sp_results", "sp_detect", "sp_results_device", "sp_slide",
    "sp_export", "sp_import", "sp_detect_noalloc", "sp_update_batched_device", "sp_autotune",
    "sp_results_async", "sp_psu", "sp_size_ldca", "sp_set_timeout", "sp_copy_sketch", "sp_merge_device",
    "sp_binned_shapes", "sp_set_binned_shape", "sp_get_binned_shape", "sp_autotune_binned",
    "sp_reset_range", "sp_update_batched_host", "sp_reserve",
)


class sp_params(ctypes.Structure):
    _fields_ = [
        ("r", ctypes.c_uint32), ("sr", ctypes.c_uint32),
        ("isb", ctypes.c_uint32 * 8), ("ibn", ctypes.c_uint32 * 8),
        ("k_log2", ctypes.c_uint32), ("lr", ctypes.c_uint32), ("lc_log2", ctypes.c_uint32),
        ("theta", ctypes.c_uint32), ("n_routers", ctypes.c_uint32),
        ("window_slices", ctypes.c_uint32), ("max_candidates", ctypes.c_uint32),
        ("scan_mode", ctypes.c_uint32), ("seed", ctypes.c_uint64), ("max_join", ctypes.c_uint64),
    ]


class sp_candidate(ctypes.Structure):
    _fields_ = [("ip", ctypes.c_uint32), ("z0", ctypes.c_uint32), ("est", ctypes.c_double),
                ("flags", ctypes.c_uint32), ("pad", ctypes.c_uint32)]


class sp_binned_shape(ctypes.Structure):
    _fields_ = [("index", ctypes.c_uint32), ("bin_threads", ctypes.c_uint32), ("bin_stage", ctypes.c_uint32),
                ("bin_tiles_per_round", ctypes.c_uint32), ("bin_blocks_per_sm", ctypes.c_uint32),
                ("apply_threads", ctypes.c_uint32)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class sp_batch(ctypes.Structure):
    _fields_ = [("pairs", ctypes.c_void_p), ("n_pairs", ctypes.c_uint64), ("router", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32)]


# the same layout as a numpy record, for batch tables built on the host and
# copied to device memory (sp_update_batched_device)
BATCH = np.dtype([("pairs", "<u8"), ("n_pairs", "<u8"), ("router", "<u4"), ("reserved", "<u4")])
assert BATCH.itemsize == ctypes.sizeof(sp_batch)

CANDIDATE = np.dtype([("ip", "<u4"), ("z0", "<u4"), ("est", "<f8"), ("flags", "<u4"), ("pad", "<u4")])
assert CANDIDATE.itemsize == ctypes.sizeof(sp_candidate)


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libsuperpoint is not built ({LIB_PATH} missing): run "
                          "paper_1901_07306_gb300.build.build() -- there is no CPU fallback")
    lib = ctypes.CDLL(LIB_PATH)
    u32, u64, vp, i32 = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_int
    P = ctypes.POINTER
    sig = {
        "sp_version": (i32, []),
        "sp_strerror": (ctypes.c_char_p, [i32]),
        "sp_default_params": (i32, [P(sp_params)]),
        "sp_check_params": (i32, [P(sp_params)]),
        "sp_sketch_bytes": (i32, [P(sp_params), P(u64), P(u64)]),
        "sp_tau": (u32, [u32]),
        "sp_z_theta": (u32, [u32, u32]),
        "sp_create": (i32, [P(sp_params), vp, P(vp)]),
        "sp_destroy": (None, [vp]),
        "sp_set_stream": (i32, [vp, vp]),
        "sp_set_timeout": (i32, [vp, u32]),
        "sp_reserve": (i32, [vp, u32, u32]),
        "sp_get_params": (i32, [vp, P(sp_params)]),
        "sp_reset": (i32, [vp, u32]),
        "sp_reset_range": (i32, [vp, u32, u32]),
        "sp_update": (i32, [vp, u32, vp, u64]),
        "sp_update_host": (i32, [vp, u32, vp, u64]),
        "sp_update_batched": (i32, [vp, u32, P(u32), P(vp), P(u64)]),
        "sp_update_batched_host": (i32, [vp, u32, P(u32), P(vp), P(u64), vp, u64, vp]),
        "sp_merge": (i32, [vp, P(u32), u32, u32]),
        "sp_copy_sketch": (i32, [vp, u32, vp, u64, P(u64)]),
        "sp_merge_device": (i32, [vp, P(vp), u32, u32]),
        "sp_binned_shapes": (i32, [P(sp_binned_shape), u32, P(u32)]),
        "sp_set_binned_shape": (i32, [vp, u32]),
        "sp_get_binned_shape": (i32, [vp, P(sp_binned_shape)]),
        "sp_autotune_binned": (i32, [vp, vp, u64, P(sp_binned_shape)]),
        "sp_detect_async": (i32, [vp, u32, u32]),
        "sp_results": (i32, [vp, vp, u64, P(u64)]),
        "sp_detect": (i32, [vp, u32, u32, vp, u64, P(u64)]),
        "sp_results_device": (i32, [vp, P(vp), P(vp)]),
        "sp_slide": (i32, [vp, u32]),
        "sp_export": (i32, [vp, u32, vp, u64, P(u64)]),
        "sp_import": (i32, [vp, u32, vp, u64]),
        "sp_detect_noalloc": (i32, [P(sp_params), vp, vp, u32, vp, u32, vp, vp]),
        "sp_update_batched_device": (i32, [vp, vp, u32]),
        "sp_autotune": (i32, [vp, vp, u64, P(u32), P(u32)]),
        "sp_results_async": (i32, [vp, vp, u64, vp]),
        "sp_psu": (ctypes.c_double, [u64, u32, u32, u32]),
        "sp_size_ldca": (i32, [u64, u32, u64, P(u32), P(u32), P(ctypes.c_double), P(ctypes.c_double)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype, fn.argtypes = res, args
    return lib


lib = _load()


class SPError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {lib.sp_strerror(code).decode()} ({code})")
        self.code = code


def _check(code: int, where: str, ok=(SP_OK,)) -> int:
    if code not in ok and code < 0:
        raise SPError(code, where)
    return code


# ---- the C names -----------------------------------------------------------
def sp_default_params() -> sp_params:
    p = sp_params()
    _check(lib.sp_default_params(ctypes.byref(p)), "sp_default_params")
    return p


def make_params(r=14, isb=(0, 5, 10, 15), ibn=(7, 7, 7, 7), k_log2=10, lr=4, lc_log2=16,
                theta=1024, n_routers=1, window_slices=1, max_candidates=0, seed=0x5EED,
                max_join=0, scan_mode=0) -> sp_params:
    p = sp_params()
    p.r, p.sr = r, len(isb)
    for i, (s, b) in enumerate(zip(isb, ibn)):
        p.isb[i], p.ibn[i] = s, b
    p.k_log2, p.lr, p.lc_log2, p.theta = k_log2, lr, lc_log2, theta
    p.n_routers, p.window_slices, p.max_candidates = n_routers, window_slices, max_candidates
    p.seed, p.max_join, p.scan_mode = seed & (2**64 - 1), max_join, scan_mode
    return p


def sp_psu(n_pairs: int, k_log2: int, lr: int, lc_log2: int) -> float:
    return lib.sp_psu(n_pairs, k_log2, lr, lc_log2)


def sp_size_ldca(n_pairs: int, k_log2: int, ldc_budget: int):
    """Returns (lr, lc_log2, psu, lr_star)."""
    lr, c = ctypes.c_uint32(), ctypes.c_uint32()
    psu, star = ctypes.c_double(), ctypes.c_double()
    _check(lib.sp_size_ldca(n_pairs, k_log2, ldc_budget, ctypes.byref(lr), ctypes.byref(c), ctypes.byref(psu),
                            ctypes.byref(star)), "sp_size_ldca")
    return lr.value, c.value, psu.value, star.value


def sp_check_params(p: sp_params) -> int:
    return lib.sp_check_params(ctypes.byref(p))


def sp_sketch_bytes(p: sp_params):
    a, b = ctypes.c_uint64(), ctypes.c_uint64()
    _check(lib.sp_sketch_bytes(ctypes.byref(p), ctypes.byref(a), ctypes.byref(b)), "sp_sketch_bytes")
    return a.value, b.value


def sp_tau(theta: int) -> int:
    return lib.sp_tau(theta)


def sp_z_theta(k_log2: int, threshold: int) -> int:
    return lib.sp_z_theta(k_log2, threshold)


def _stream_handle(stream) -> int:
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return int(getattr(stream, "cuda_stream", stream))


def sp_create(p: sp_params, stream=None) -> int:
    ctx = ctypes.c_void_p()
    _check(lib.sp_create(ctypes.byref(p), ctypes.c_void_p(_stream_handle(stream)), ctypes.byref(ctx)),
           "sp_create")
    return ctx.value


def sp_destroy(ctx: int) -> None:
    lib.sp_destroy(ctypes.c_void_p(ctx))


def sp_set_stream(ctx: int, stream) -> None:
    _check(lib.sp_set_stream(ctypes.c_void_p(ctx), ctypes.c_void_p(_stream_handle(stream))), "sp_set_stream")


def sp_set_timeout(ctx: int, timeout_ms: int) -> None:
    _check(lib.sp_set_timeout(ctypes.c_void_p(ctx), timeout_ms), "sp_set_timeout")


def sp_reserve(ctx: int, first: int = 0, count: int | None = None) -> None:
    """Allocates up front what updates of routers first .. first + count - 1
    would allocate on first use (default: every router)."""
    if count is None:
        count = sp_get_params(ctx).n_routers - first
    _check(lib.sp_reserve(ctypes.c_void_p(ctx), first, count), "sp_reserve")


def sp_get_params(ctx: int) -> sp_params:
    p = sp_params()
    _check(lib.sp_get_params(ctypes.c_void_p(ctx), ctypes.byref(p)), "sp_get_params")
    return p


def sp_reset(ctx: int, router: int = 0) -> None:
    _check(lib.sp_reset(ctypes.c_void_p(ctx), router), "sp_reset")


def sp_reset_range(ctx: int, first: int, count: int) -> None:
    _check(lib.sp_reset_range(ctypes.c_void_p(ctx), first, count), "sp_reset_range")


def _pairs_ptr(pairs):
    """(pointer, n_pairs) of a contiguous uint32/int32 tensor or array of pairs."""
    if hasattr(pairs, "data_ptr"):
        if not pairs.is_contiguous():
            raise ValueError("pairs must be contiguous")
        return pairs.data_ptr(), pairs.numel() // 2
    if not (isinstance(pairs, np.ndarray) and pairs.flags.c_contiguous and pairs.dtype.itemsize == 4):
        raise ValueError("host pairs must be a C-contiguous 4-byte integer array (the library borrows it)")
    return pairs.ctypes.data, pairs.size // 2


def sp_update(ctx: int, router: int, dev_pairs) -> None:
    """dev_pairs: contiguous CUDA tensor of 2n uint32/int32 values (hip, oip)."""
    ptr, n = _pairs_ptr(dev_pairs)
    _check(lib.sp_update(ctypes.c_void_p(ctx), router, ctypes.c_void_p(ptr), n), "sp_update")


def sp_update_host(ctx: int, router: int, host_pairs) -> None:
    """host_pairs: contiguous host tensor/array (pinned for overlapped copies);
    keep it alive until the stream has passed the update."""
    ptr, n = _pairs_ptr(host_pairs)
    _check(lib.sp_update_host(ctypes.c_void_p(ctx), router, ctypes.c_void_p(ptr), n), "sp_update_host")


def sp_update_batched(ctx: int, routers, batches) -> None:
    nb = len(batches)
    r = (ctypes.c_uint32 * nb)(*routers)
    ptrs = (ctypes.c_void_p * nb)()
    ns = (ctypes.c_uint64 * nb)()
    for i, b in enumerate(batches):
        ptrs[i], ns[i] = _pairs_ptr(b)
    _check(lib.sp_update_batched(ctypes.c_void_p(ctx), nb, r, ptrs, ns), "sp_update_batched")


def sp_update_batched_host(ctx: int, routers, host_batches, dev_arena, copy_stream) -> None:
    """host_batches: pinned host tensors/arrays of pairs; dev_arena: CUDA
    tensor the batches are copied into (packed at 16-byte boundaries);
    copy_stream: the stream the copies run on."""
    nb = len(host_batches)
    r = (ctypes.c_uint32 * nb)(*routers)
    ptrs = (ctypes.c_void_p * nb)()
    ns = (ctypes.c_uint64 * nb)()
    for i, b in enumerate(host_batches):
        ptrs[i], ns[i] = _pairs_ptr(b)
    _check(lib.sp_update_batched_host(ctypes.c_void_p(ctx), nb, r, ptrs, ns, ctypes.c_void_p(dev_arena.data_ptr()),
                                      dev_arena.numel() * dev_arena.element_size(),
                                      ctypes.c_void_p(_stream_handle(copy_stream))), "sp_update_batched_host")


def sp_update_batched_device(ctx: int, dev_table, n_batches: int) -> None:
    """dev_table: device memory (tensor) holding n_batches BATCH records."""
    ptr = dev_table.data_ptr() if hasattr(dev_table, "data_ptr") else int(dev_table)
    _check(lib.sp_update_batched_device(ctypes.c_void_p(ctx), ctypes.c_void_p(ptr), n_batches),
           "sp_update_batched_device")


def sp_autotune(ctx: int, dev_pairs):
    """Returns (threads, blocks per SM) chosen for the batched launch."""
    ptr, n = _pairs_ptr(dev_pairs)
    t, b = ctypes.c_uint32(), ctypes.c_uint32()
    _check(lib.sp_autotune(ctypes.c_void_p(ctx), ctypes.c_void_p(ptr), n, ctypes.byref(t), ctypes.byref(b)),
           "sp_autotune")
    return t.value, b.value


def sp_binned_shapes() -> list:
    n = ctypes.c_uint32()
    _check(lib.sp_binned_shapes(None, 0, ctypes.byref(n)), "sp_binned_shapes")
    out = (sp_binned_shape * n.value)()
    _check(lib.sp_binned_shapes(out, n.value, ctypes.byref(n)), "sp_binned_shapes")
    return [x.as_dict() for x in out]


def sp_set_binned_shape(ctx: int, index: int) -> None:
    _check(lib.sp_set_binned_shape(ctypes.c_void_p(ctx), index), "sp_set_binned_shape")


def sp_get_binned_shape(ctx: int) -> dict:
    out = sp_binned_shape()
    _check(lib.sp_get_binned_shape(ctypes.c_void_p(ctx), ctypes.byref(out)), "sp_get_binned_shape")
    return out.as_dict()


def sp_autotune_binned(ctx: int, dev_pairs) -> dict:
    """Times every compiled staging shape of the binned scan on the sample,
    keeps the fastest; returns its description."""
    ptr, n = _pairs_ptr(dev_pairs)
    out = sp_binned_shape()
    _check(lib.sp_autotune_binned(ctypes.c_void_p(ctx), ctypes.c_void_p(ptr), n, ctypes.byref(out)),
           "sp_autotune_binned")
    return out.as_dict()


def sp_merge(ctx: int, routers, dst_router: int) -> None:
    arr = (ctypes.c_uint32 * len(routers))(*routers)
    _check(lib.sp_merge(ctypes.c_void_p(ctx), arr, len(routers), dst_router), "sp_merge")


def sp_copy_sketch_bytes(ctx: int) -> int:
    n = ctypes.c_uint64()
    _check(lib.sp_copy_sketch(ctypes.c_void_p(ctx), 0, None, 0, ctypes.byref(n)), "sp_copy_sketch")
    return n.value


def sp_copy_sketch(ctx: int, router: int, dev_dst) -> None:
    """dev_dst: CUDA uint8 tensor of at least sp_copy_sketch_bytes(ctx) bytes."""
    n = ctypes.c_uint64()
    _check(lib.sp_copy_sketch(ctypes.c_void_p(ctx), router, ctypes.c_void_p(dev_dst.data_ptr()),
                              dev_dst.numel() * dev_dst.element_size(), ctypes.byref(n)), "sp_copy_sketch")


def sp_merge_device(ctx: int, dev_images, dst_router: int) -> None:
    """dev_images: CUDA tensors (or raw device addresses) of sp_copy_sketch images."""
    ptrs = [x.data_ptr() if hasattr(x, "data_ptr") else int(x) for x in dev_images]
    arr = (ctypes.c_void_p * max(1, len(ptrs)))(*ptrs)
    _check(lib.sp_merge_device(ctypes.c_void_p(ctx), arr, len(ptrs), dst_router), "sp_merge_device")


def sp_detect_async(ctx: int, router: int = 0, threshold: int = 0) -> int:
    return _check(lib.sp_detect_async(ctypes.c_void_p(ctx), router, threshold), "sp_detect_async")


def sp_results(ctx: int, cap: int | None = None):
    """Returns (records, n_total, status) for the last detect."""
    n = ctypes.c_uint64()
    if cap is None:
        rc = lib.sp_results(ctypes.c_void_p(ctx), None, 0, ctypes.byref(n))
        if rc not in (SP_OK, SP_ERR_TRUNCATED, SP_ERR_CANDIDATE_OVERFLOW):
            _check(rc, "sp_results")
        cap = n.value
    out = np.zeros(max(cap, 1), CANDIDATE)
    rc = lib.sp_results(ctypes.c_void_p(ctx), ctypes.c_void_p(out.ctypes.data), cap, ctypes.byref(n))
    _check(rc, "sp_results", ok=(SP_OK, SP_ERR_TRUNCATED, SP_ERR_CANDIDATE_OVERFLOW))
    written = min(cap, n.value, sp_get_params(ctx).max_candidates)
    return out[:written], n.value, rc


def _host_ptr(x) -> int:
    return x.data_ptr() if hasattr(x, "data_ptr") else x.ctypes.data


def sp_results_async(ctx: int, host_out, cap: int, host_status) -> None:
    """host_out: pinned host buffer of >= cap CANDIDATE records (tensor or
    array); host_status: pinned host buffer of 2 uint32/int32 words."""
    _check(lib.sp_results_async(ctypes.c_void_p(ctx), ctypes.c_void_p(_host_ptr(host_out)), cap,
                                ctypes.c_void_p(_host_ptr(host_status))), "sp_results_async")


def sp_detect(ctx: int, router: int = 0, threshold: int = 0, cap: int | None = None):
    w = sp_detect_async(ctx, router, threshold)
    recs, n, rc = sp_results(ctx, cap)
    return recs, n, (rc if rc != SP_OK else w)


def sp_results_device(ctx: int):
    recs, cnt = ctypes.c_void_p(), ctypes.c_void_p()
    _check(lib.sp_results_device(ctypes.c_void_p(ctx), ctypes.byref(recs), ctypes.byref(cnt)),
           "sp_results_device")
    return recs.value, cnt.value


def sp_slide(ctx: int, router: int = 0) -> None:
    _check(lib.sp_slide(ctypes.c_void_p(ctx), router), "sp_slide")


def sp_export(ctx: int, router: int = 0) -> bytes:
    n = ctypes.c_uint64()
    _check(lib.sp_export(ctypes.c_void_p(ctx), router, None, 0, ctypes.byref(n)), "sp_export")
    buf = (ctypes.c_uint8 * n.value)()
    _check(lib.sp_export(ctypes.c_void_p(ctx), router, buf, n.value, ctypes.byref(n)), "sp_export")
    return bytes(buf)


def sp_import(ctx: int, router: int, image: bytes) -> int:
    buf = (ctypes.c_uint8 * len(image)).from_buffer_copy(image)
    return lib.sp_import(ctypes.c_void_p(ctx), router, buf, len(image))


# ---- convenience wrapper ----------------------------------------------------
class SuperPoint:
    """One library context (one or more simulated watch points)."""

    def __init__(self, params: sp_params | None = None, stream=None, **kw):
        self.params = params if params is not None else make_params(**kw)
        self.ctx = sp_create(self.params, stream)

    def close(self):
        if self.ctx:
            sp_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sketch_image(self, router: int = 0):
        """(seav uint8 array, ldca uint32 array) in the logical layout."""
        img = sp_export(self.ctx, router)
        seav_b, ldca_b = sp_sketch_bytes(self.params)
        hdr = len(img) - seav_b - ldca_b - 8
        seav = np.frombuffer(img, np.uint8, seav_b, hdr).copy()
        ldca = np.frombuffer(img, np.uint32, ldca_b // 4, hdr + seav_b).copy()
        return seav, ldca

    def reset(self, router=0): sp_reset(self.ctx, router)
    def update(self, pairs, router=0): sp_update(self.ctx, router, pairs)
    def update_host(self, pairs, router=0): sp_update_host(self.ctx, router, pairs)
    def merge(self, routers, dst): sp_merge(self.ctx, routers, dst)
    def detect(self, router=0, threshold=0, cap=None): return sp_detect(self.ctx, router, threshold, cap)
    def slide(self, router=0): sp_slide(self.ctx, router)
