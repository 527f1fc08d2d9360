"""Thin ctypes binding of libbenelux (include/benelux.h), same names as the C ABI.

Argument marshalling only: every step of the search runs in the library's CUDA
kernels.  There is no CPU fallback -- if the library is missing or cannot be
loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

BNX_OK, BNX_E_ARG, BNX_E_TRUNCATED, BNX_E_NOMEM, BNX_E_CUDA = 0, 1, 2, 3, 4
BNX_E_TIMEOUT, BNX_E_BUSY, BNX_E_STATE, BNX_E_OVERFLOW, BNX_E_CANCELLED = 5, 6, 7, 8, 9
BNX_CKPT_ALL = (1 << 64) - 1
BNX_MAX_HI = 1 << 42

u64, u32, i32, sz, vp = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_size_t, ctypes.c_void_p


class bnx_pair(ctypes.Structure):
    _fields_ = [("m", u64), ("n", u64), ("kind", u32), ("iv", u32)]


class bnx_interval(ctypes.Structure):
    _fields_ = [("lo", u64), ("hi", u64), ("kinds", u32), ("id", u32)]


class bnx_tune(ctypes.Structure):
    _fields_ = [("tile_log2", u32), ("seg_tiles", u32), ("threads", u32), ("ctas_per_sm", u32),
                ("small_q_log2", u32), ("tile_kind", u32)]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


class bnx_stats(ctypes.Structure):
    _fields_ = [("integers", u64), ("segments", u64), ("bucket_hits", u64), ("survivors1", u64),
                ("survivors2", u64), ("candidates", u64), ("pairs", u64), ("hash_keys", u64),
                ("ms_total", ctypes.c_float), ("ms_sieve", ctypes.c_float), ("sieve_launches", u32),
                ("pad", u32)]

    def as_dict(self):
        return {f: (float(getattr(self, f)) if t is ctypes.c_float else int(getattr(self, f)))
                for f, t in self._fields_ if f != "pad"}


class bnx_server_cfg(ctypes.Structure):
    _fields_ = [("max_active", u32), ("pad", u32), ("slice", u64), ("mem_budget", u64)]


class bnx_server_stats(ctypes.Structure):
    _fields_ = [("submitted", u64), ("completed", u64), ("iterations", u64), ("deferred", u64),
                ("rejected", u64), ("budget_bytes", u64), ("ws_peak_bytes", u64), ("cancelled", u64)]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


class BnxError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"bnx error {code}: {msg}")
        self.code = code


_lib = None
_lock = threading.Lock()


def lib(auto_build: bool = True):
    """Load libbenelux.so (building it first when it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if auto_build and not _build.up_to_date():
            path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError("libbenelux.so is not built; run paper_2506_01099_gb300.build.build()")
        L = ctypes.CDLL(path)
        P = ctypes.POINTER
        sig = {
            "bnx_create": ([P(vp), i32, u64, ctypes.c_char_p, vp], i32),
            "bnx_destroy": ([vp], None),
            "bnx_tune_parse": ([ctypes.c_char_p, P(bnx_tune)], i32),
            "bnx_get_tune": ([vp, P(bnx_tune)], i32),
            "bnx_set_tune": ([vp, P(bnx_tune)], i32),
            "bnx_get_stats": ([vp, P(bnx_stats)], i32),
            "bnx_prime_count": ([vp, P(u64)], i32),
            "bnx_rad_segment": ([vp, u64, u64, vp, vp, vp], i32),
            "bnx_rad_segment_noalloc": ([u64, u64, vp, vp, vp], i32),
            "bnx_log_weight": ([u64, u32], u32),
            "bnx_log_weight54": ([u64], u32),
            "bnx_same_rad": ([P(u64), P(u64), sz, P(ctypes.c_uint8)], i32),
            "bnx_log_weights": ([vp, u32, P(u32), sz, P(sz)], i32),
            "bnx_search": ([vp, u64, u64, u32, P(bnx_pair), sz, P(sz)], i32),
            "bnx_search_segment": ([vp, u64, u32, u32, P(bnx_pair), sz, P(sz)], i32),
            "bnx_search_hash": ([vp, u64, u32, P(bnx_pair), sz, P(sz)], i32),
            "bnx_search_chunked": ([vp, u64, u32, u32, P(bnx_pair), sz, P(sz)], i32),
            "bnx_search_sorted": ([vp, u64, u32, P(bnx_pair), sz, P(sz)], i32),
            "bnx_batch": ([vp, P(bnx_interval), sz, P(bnx_pair), sz, P(sz), P(u64)], i32),
            "bnx_arm_lookback_timeout": ([vp, u32], i32),
            "bnx_server_start": ([vp, P(bnx_server_cfg)], i32),
            "bnx_server_submit": ([vp, P(bnx_interval), P(u64)], i32),
            "bnx_server_cancel": ([vp, u64], i32),
            "bnx_search_checkpointed": ([vp, u64, u64, u32, ctypes.c_char_p, u64, u64, P(bnx_pair), sz, P(sz),
                                         P(u64)], i32),
            "bnx_server_poll": ([vp, u64, P(bnx_pair), sz, P(sz), P(ctypes.c_double)], i32),
            "bnx_server_stop": ([vp], i32),
            "bnx_server_get_stats": ([vp, P(bnx_server_stats)], i32),
            "bnx_workspace_bytes": ([vp, P(bnx_interval), sz, P(u64)], i32),
            "bnx_autotune": ([vp, P(bnx_interval), sz, i32, ctypes.c_char_p, sz], i32),
            "bnx_strerror": ([i32], ctypes.c_char_p),
            "bnx_last_error": ([], ctypes.c_char_p),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes, f.restype = args, res
        _lib = L
        return L


def _check(rc: int):
    if rc != BNX_OK:
        L = lib()
        raise BnxError(rc, f"{L.bnx_strerror(rc).decode()}: {L.bnx_last_error().decode()}")


def _pairs(buf, n):
    return [(int(buf[i].m), int(buf[i].n), int(buf[i].kind)) for i in range(n)]


# ---------------------------------------------------------------- ABI names --

def bnx_strerror(code: int) -> str:
    return lib().bnx_strerror(code).decode()


def bnx_last_error() -> str:
    return lib().bnx_last_error().decode()


def bnx_create(device: int = 0, max_hi: int = 1 << 41, tune_json: str | None = None, stream: int | None = None):
    h = vp()
    _check(lib().bnx_create(ctypes.byref(h), device, max_hi,
                            tune_json.encode() if tune_json else None, stream or None))
    return h


def bnx_destroy(ctx) -> None:
    lib().bnx_destroy(ctx)


def bnx_tune_parse(json_text: str) -> bnx_tune:
    """The tuning a JSON object gives (defaults for absent fields); raises on a bad object."""
    t = bnx_tune()
    _check(lib().bnx_tune_parse(json_text.encode(), ctypes.byref(t)))
    return t


def bnx_get_tune(ctx) -> bnx_tune:
    t = bnx_tune()
    _check(lib().bnx_get_tune(ctx, ctypes.byref(t)))
    return t


def bnx_set_tune(ctx, tune: bnx_tune) -> None:
    _check(lib().bnx_set_tune(ctx, ctypes.byref(tune)))


def bnx_get_stats(ctx) -> bnx_stats:
    s = bnx_stats()
    _check(lib().bnx_get_stats(ctx, ctypes.byref(s)))
    return s


def bnx_prime_count(ctx) -> int:
    v = u64()
    _check(lib().bnx_prime_count(ctx, ctypes.byref(v)))
    return int(v.value)


def bnx_rad_segment(ctx, lo: int, length: int, rad_out_ptr: int, sq_out_ptr: int | None = None,
                    stream: int | None = None) -> None:
    """Device pointers: asynchronous on `stream`; host pointers: returns once written."""
    _check(lib().bnx_rad_segment(ctx, lo, length, rad_out_ptr, sq_out_ptr or None, stream or None))


BNX_NOALLOC_MAX_LEN, BNX_NOALLOC_MAX_HI = 1 << 18, 1 << 40


def bnx_rad_segment_noalloc(lo: int, length: int, rad_out_ptr: int, sq_out_ptr: int | None = None,
                            stream: int | None = None) -> None:
    """Like bnx_rad_segment, for callers that cannot allocate device memory: no
    context, no allocation, fixed limits (length <= 2^18, lo + length <= 2^40)."""
    _check(lib().bnx_rad_segment_noalloc(lo, length, rad_out_ptr, sq_out_ptr or None, stream or None))


def bnx_log_weight(p: int, frac_log2: int) -> int:
    """Smallest L with 2^L > p^(2^frac_log2), in integers (host only)."""
    return int(lib().bnx_log_weight(p, frac_log2))


def bnx_log_weight54(p: int) -> int:
    """The u8 tile's weight ceil(bitlen(p^5) / 4), units of 4/5 bit (host only)."""
    return int(lib().bnx_log_weight54(p))


def bnx_same_rad(x, y):
    """rad(x[i]) == rad(y[i]) per pair, on the device (the verification kernel's test)."""
    import numpy as np

    xa = np.ascontiguousarray(x, dtype=np.uint64)
    ya = np.ascontiguousarray(y, dtype=np.uint64)
    assert xa.shape == ya.shape
    out = np.zeros(xa.size, dtype=np.uint8)
    _check(lib().bnx_same_rad(xa.ctypes.data_as(ctypes.POINTER(u64)), ya.ctypes.data_as(ctypes.POINTER(u64)),
                              xa.size, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))))
    return out.astype(bool)


def bnx_log_weights(ctx, tile_kind: int = 3):
    """Per prime of the context's table: (p, in-tile, cached-bucket, global-bucket) weights
    of the log tile `tile_kind`, as the device computes them."""
    n = sz()
    rc = lib().bnx_log_weights(ctx, tile_kind, None, 0, ctypes.byref(n))
    if rc not in (BNX_OK, BNX_E_TRUNCATED):
        _check(rc)
    cap = int(n.value)
    buf = (u32 * (4 * max(cap, 1)))()
    _check(lib().bnx_log_weights(ctx, tile_kind, buf, cap, ctypes.byref(n)))
    import numpy as np

    return np.frombuffer(buf, dtype=np.uint32)[:4 * cap].reshape(cap, 4).copy()


def _grow_call(fn, cap=256):
    while True:
        buf = (bnx_pair * cap)()
        n = sz()
        rc = fn(buf, cap, ctypes.byref(n))
        if rc == BNX_E_TRUNCATED:
            cap = int(n.value) + 16
            continue
        _check(rc)
        return buf, int(n.value)


def bnx_search(ctx, lo: int, hi: int, kinds: int = 3):
    """Pairs (m, n, kind) with lo <= n < hi, sorted by (n, m, kind)."""
    buf, n = _grow_call(lambda b, c, pn: lib().bnx_search(ctx, lo, hi, kinds, b, c, pn))
    return _pairs(buf, n)


def bnx_search_segment(ctx, lo: int, length: int, kinds: int = 3):
    """Pairs (m, n, kind) with lo <= n < lo + length (length < 2^32), sorted by (n, m, kind)."""
    buf, n = _grow_call(lambda b, c, pn: lib().bnx_search_segment(ctx, lo, length, kinds, b, c, pn))
    return _pairs(buf, n)


def bnx_search_hash(ctx, S: int, kinds: int = 3):
    """Pairs (m, n, kind) with m < n < S by the device hash table."""
    buf, n = _grow_call(lambda b, c, pn: lib().bnx_search_hash(ctx, S, kinds, b, c, pn))
    return _pairs(buf, n)


def bnx_search_chunked(ctx, S: int, chunk_log2: int = 27, kinds: int = 3):
    """Pairs (m, n, kind) with m < n < S by Algorithm 3 (chunks of 2^chunk_log2)."""
    buf, n = _grow_call(lambda b, c, pn: lib().bnx_search_chunked(ctx, S, chunk_log2, kinds, b, c, pn))
    return _pairs(buf, n)


def bnx_search_sorted(ctx, S: int, kinds: int = 3):
    """Pairs (m, n, kind) with m < n < S by Algorithm 2 (device radix sort of the keys)."""
    buf, n = _grow_call(lambda b, c, pn: lib().bnx_search_sorted(ctx, S, kinds, b, c, pn))
    return _pairs(buf, n)


def bnx_arm_lookback_timeout(ctx, spin_limit: int) -> None:
    """Test hook: the next bnx_search_sorted call's look-back wait runs out (BNX_E_TIMEOUT)."""
    _check(lib().bnx_arm_lookback_timeout(ctx, spin_limit))


def make_intervals(intervals):
    """Sequence of (lo, hi, kinds[, id]) or objects with .lo/.hi/.kinds -> ctypes array."""
    arr = (bnx_interval * max(1, len(intervals)))()
    for i, iv in enumerate(intervals):
        if hasattr(iv, "lo"):
            arr[i].lo, arr[i].hi, arr[i].kinds, arr[i].id = iv.lo, iv.hi, iv.kinds, getattr(iv, "id", i)
        else:
            arr[i].lo, arr[i].hi, arr[i].kinds = iv[0], iv[1], iv[2]
            arr[i].id = iv[3] if len(iv) > 3 else i
    return arr


def bnx_batch(ctx, intervals, iv_array=None):
    """All intervals in one pipeline.  Returns (pairs, offsets): pairs as
    (interval index, m, n, kind) sorted by (interval, n, m, kind), offsets[i]..
    offsets[i+1] delimiting interval i."""
    k = len(intervals)
    arr = iv_array if iv_array is not None else make_intervals(intervals)
    offs = (u64 * (k + 1))()
    buf, n = _grow_call(lambda b, c, pn: lib().bnx_batch(ctx, arr, k, b, c, pn, offs))
    pairs = [(int(buf[i].iv), int(buf[i].m), int(buf[i].n), int(buf[i].kind)) for i in range(n)]
    return pairs, [int(offs[i]) for i in range(k + 1)]


def bnx_server_start(ctx, max_active: int = 64, slice_len: int = 1 << 28, mem_budget: int = 0) -> None:
    cfg = bnx_server_cfg(max_active, 0, slice_len, mem_budget)
    _check(lib().bnx_server_start(ctx, ctypes.byref(cfg)))


def bnx_server_submit(ctx, lo: int, hi: int, kinds: int = 3, ident: int = 0) -> int:
    iv = bnx_interval(lo, hi, kinds, ident)
    t = u64()
    _check(lib().bnx_server_submit(ctx, ctypes.byref(iv), ctypes.byref(t)))
    return int(t.value)


def bnx_server_poll(ctx, ticket: int):
    """None while the request runs; else (pairs, latency_s)."""
    cap = 64
    while True:
        buf = (bnx_pair * cap)()
        n, lat = sz(), ctypes.c_double()
        rc = lib().bnx_server_poll(ctx, ticket, buf, cap, ctypes.byref(n), ctypes.byref(lat))
        if rc == BNX_E_BUSY:
            return None
        if rc == BNX_E_TRUNCATED:
            cap = int(n.value) + 16
            continue
        _check(rc)
        return _pairs(buf, int(n.value)), float(lat.value)


def bnx_server_cancel(ctx, ticket: int) -> None:
    _check(lib().bnx_server_cancel(ctx, ticket))


def bnx_search_checkpointed(ctx, lo: int, hi: int, kinds: int, path: str, chunk: int, max_chunks: int = BNX_CKPT_ALL):
    """(pairs so far, next n to search, finished).  Runs at most max_chunks chunks of
    `chunk` integers, saving the progress to `path` after each; resumes from `path`."""
    p = os.fsencode(path)
    nxt = u64()
    cap = 256
    while True:
        buf = (bnx_pair * cap)()
        n = sz()
        rc = lib().bnx_search_checkpointed(ctx, lo, hi, kinds, p, chunk, max_chunks, buf, cap, ctypes.byref(n),
                                           ctypes.byref(nxt))
        if rc == BNX_E_TRUNCATED:  # the progress is saved: read the pairs back without searching
            cap, max_chunks = int(n.value) + 16, 0
            continue
        if rc not in (BNX_OK, BNX_E_BUSY):
            _check(rc)
        return _pairs(buf, int(n.value)), int(nxt.value), rc == BNX_OK


def bnx_server_stop(ctx) -> None:
    _check(lib().bnx_server_stop(ctx))


def bnx_server_get_stats(ctx) -> dict:
    st = bnx_server_stats()
    _check(lib().bnx_server_get_stats(ctx, ctypes.byref(st)))
    return st.as_dict()


def bnx_workspace_bytes(ctx, intervals) -> int:
    """Device workspace bytes one batched run over these intervals needs."""
    arr = make_intervals(intervals)
    v = u64()
    _check(lib().bnx_workspace_bytes(ctx, arr, len(intervals), ctypes.byref(v)))
    return int(v.value)


def bnx_autotune(ctx, intervals, rounds: int = 2) -> str:
    arr = make_intervals(intervals)
    out = ctypes.create_string_buffer(512)
    _check(lib().bnx_autotune(ctx, arr, len(intervals), rounds, out, 512))
    return out.value.decode()


class Context:
    """Owns one bnx_ctx; the methods forward to the functions above."""

    def __init__(self, device: int = 0, max_hi: int = 1 << 41, tune_json: str | None = None,
                 stream: int | None = None):
        self.h = bnx_create(device, max_hi, tune_json, stream)

    def close(self):
        if self.h:
            bnx_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def search(self, lo, hi, kinds=3):
        return bnx_search(self.h, lo, hi, kinds)

    def search_checkpointed(self, lo, hi, kinds, path, chunk, max_chunks=BNX_CKPT_ALL):
        return bnx_search_checkpointed(self.h, lo, hi, kinds, path, chunk, max_chunks)

    def search_segment(self, lo, length, kinds=3):
        return bnx_search_segment(self.h, lo, length, kinds)

    def search_hash(self, S, kinds=3):
        return bnx_search_hash(self.h, S, kinds)

    def search_chunked(self, S, chunk_log2=27, kinds=3):
        return bnx_search_chunked(self.h, S, chunk_log2, kinds)

    def search_sorted(self, S, kinds=3):
        return bnx_search_sorted(self.h, S, kinds)

    def batch(self, intervals):
        return bnx_batch(self.h, intervals)

    def rad_segment(self, lo, length, rad_ptr, sq_ptr=None, stream=None):
        return bnx_rad_segment(self.h, lo, length, rad_ptr, sq_ptr, stream)

    def stats(self):
        return bnx_get_stats(self.h).as_dict()

    def tune(self):
        return bnx_get_tune(self.h).as_dict()

    def set_tune(self, **kw):
        t = bnx_get_tune(self.h)
        for k, v in kw.items():
            setattr(t, k, v)
        bnx_set_tune(self.h, t)

    def prime_count(self):
        return bnx_prime_count(self.h)

    def log_weights(self, tile_kind=3):
        return bnx_log_weights(self.h, tile_kind)

    def autotune(self, intervals, rounds=2):
        return bnx_autotune(self.h, intervals, rounds)
