"""CPU oracle for the Benelux-pair search (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline leg may import this package.  The product library never does, and
this package imports nothing from the product.

The arithmetic lives in ``benelux_oracle.c`` (plain C, built here with gcc);
this module only compiles it and marshals arguments through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "benelux_oracle.c")
BUILD_DIR = os.path.join(HERE, "_build")

_lock = threading.Lock()
_loaded: dict = {}


class OrcPair(ctypes.Structure):
    _fields_ = [("m", ctypes.c_uint64), ("n", ctypes.c_uint64), ("kind", ctypes.c_uint32), ("pad", ctypes.c_uint32)]


def build(mutant: int = 0, out_dir: str | None = None) -> str:
    """Compile the oracle (optionally with one planted mistake) and return the .so path."""
    out_dir = out_dir or BUILD_DIR
    os.makedirs(out_dir, exist_ok=True)
    name = "liboracle.so" if mutant == 0 else f"liboracle_mut{mutant}.so"
    so = os.path.join(out_dir, name)
    if os.path.exists(so) and os.path.getmtime(so) >= os.path.getmtime(SRC):
        return so
    tmp = so + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC", f"-DORC_MUTANT={mutant}", SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, so)
    return so


class Oracle:
    """ctypes view of one build of the oracle library."""

    def __init__(self, so_path: str):
        lib = ctypes.CDLL(so_path)
        u64, u32, i32, sz = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_size_t
        lib.orc_init.argtypes, lib.orc_init.restype = [u64], i32
        lib.orc_rad_td.argtypes, lib.orc_rad_td.restype = [u64], u64
        lib.orc_sq_td.argtypes, lib.orc_sq_td.restype = [u64], u64
        lib.orc_nprimes_upto.argtypes, lib.orc_nprimes_upto.restype = [u64], u64
        lib.orc_rad_sieve.argtypes = [u64, u64, ctypes.POINTER(u64)]
        lib.orc_rad_sieve.restype = i32
        for f in ("orc_pairs_brute", "orc_pairs_sort", "orc_pairs_map"):
            getattr(lib, f).argtypes = [u64, u32, ctypes.POINTER(OrcPair), sz]
            getattr(lib, f).restype = sz
        lib.orc_pairs_brute_rad.argtypes = [ctypes.POINTER(u64), u64, u32, ctypes.POINTER(OrcPair), sz]
        lib.orc_pairs_brute_rad.restype = sz
        lib.orc_pairs_crt.argtypes = [u64, u64, u32, ctypes.POINTER(OrcPair), sz, i32]
        lib.orc_pairs_crt.restype = sz
        lib.orc_filter_counts.argtypes = [u64, u64, u32, ctypes.POINTER(u64), ctypes.POINTER(u64), i32]
        lib.orc_filter_counts.restype = i32
        lib.orc_hash_keys.argtypes, lib.orc_hash_keys.restype = [u64], u64
        self.lib = lib

    # -- radicals -----------------------------------------------------------
    def rad_td(self, x: int) -> int:
        """rad(x) by trial division (definition of Sec. 2.1)."""
        return int(self.lib.orc_rad_td(x))

    def sq_td(self, x: int) -> int:
        """x / rad(x)."""
        return int(self.lib.orc_sq_td(x))

    def rad_td_array(self, start: int, length: int):
        import numpy as np

        return np.array([self.lib.orc_rad_td(start + i) for i in range(length)], dtype=np.uint64)

    def rad_sieve(self, start: int, length: int):
        """Radicals of [start, start+length) by Algorithm 1."""
        import numpy as np

        out = np.zeros(length, dtype=np.uint64)
        rc = self.lib.orc_rad_sieve(start, length, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))
        if rc != 0:
            raise ValueError("orc_rad_sieve rejected its arguments")
        return out

    def nprimes_upto(self, lim: int) -> int:
        return int(self.lib.orc_nprimes_upto(lim))

    # -- pairs --------------------------------------------------------------
    @staticmethod
    def _collect(fn, *args, cap=4096):
        while True:
            buf = (OrcPair * cap)()
            cnt = fn(*args, buf, cap)
            if cnt == ctypes.c_size_t(-1).value:
                raise MemoryError("oracle ran out of memory")
            if cnt <= cap:
                return [(int(buf[i].m), int(buf[i].n), int(buf[i].kind)) for i in range(cnt)]
            cap = int(cnt)

    def pairs_brute(self, N: int, kinds: int = 3):
        """All pairs with m < n < N (N <= 2^14), by comparing every m < n."""
        return self._collect(self.lib.orc_pairs_brute, N, kinds)

    def pairs_brute_rad(self, r, N: int, kinds: int = 3):
        """The definitions of Sec. 1 applied to a given radical array r[0 .. N+1] (r[0]
        unused; any values), every m < n < N (N <= 2^14)."""
        import numpy as np

        arr = np.ascontiguousarray(r, dtype=np.uint64)
        assert arr.size >= N + 2
        ptr = arr.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))
        return self._collect(lambda N_, k_, buf, cap: self.lib.orc_pairs_brute_rad(ptr, N_, k_, buf, cap), N, kinds)

    def pairs_sort(self, S: int, kinds: int = 3):
        """All pairs with m < n < S (S <= 2^26), by Algorithm 2 with group-wise pairing."""
        return self._collect(self.lib.orc_pairs_sort, S, kinds)

    def pairs_map(self, S: int, kinds: int = 3):
        """All pairs with m < n < S (S <= 2^26), by a hash table of the 2-sets (Algorithm 3's collision search)."""
        return self._collect(self.lib.orc_pairs_map, S, kinds)

    def pairs_crt(self, lo: int, hi: int, kinds: int = 3, nthreads: int = 0):
        """All pairs with lo <= n < hi and any m < n, by CRT candidate enumeration."""
        fn = lambda lo_, hi_, k_, buf, cap: self.lib.orc_pairs_crt(lo_, hi_, k_, buf, cap, nthreads)
        return self._collect(fn, lo, hi, kinds)

    def filter_counts(self, lo: int, hi: int, kinds: int = 3, nthreads: int = 0):
        """(first-kind, second-kind) counts of n in [lo, hi) passing the necessary conditions."""
        c1, c2 = ctypes.c_uint64(0), ctypes.c_uint64(0)
        if self.lib.orc_filter_counts(lo, hi, kinds, ctypes.byref(c1), ctypes.byref(c2), nthreads) != 0:
            raise MemoryError("oracle ran out of memory")
        return int(c1.value), int(c2.value)

    def hash_keys(self, S: int) -> int:
        """Number of x in [1, S) with rad(x) rad(x+1) <= 2S."""
        return int(self.lib.orc_hash_keys(S))


def load(mutant: int = 0, out_dir: str | None = None) -> Oracle:
    """Build (if needed) and load the oracle library."""
    with _lock:
        key = (mutant, out_dir)
        if key not in _loaded:
            _loaded[key] = Oracle(build(mutant, out_dir))
        return _loaded[key]
