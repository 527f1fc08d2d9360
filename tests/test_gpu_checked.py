"""The bounds-checked build (compute-sanitizer is closed on the GPUs this runs on).

build.build_checked() compiles the library with -DBNX_CHECK_BOUNDS: every tile index
of the sieve and radical kernels and every bucket index of the fill and the sieves is
checked; one outside its buffer skips the access, sets an error bit, and the call then
fails with BNX_E_OVERFLOW -- nothing traps.  A subprocess loads that library and runs
each path that touches tiles and buckets (searches under several tunings, radical
segments into host buffers -- a blocking call that reports the flags -- a batch, the
hash search, Algorithms 2 and 3) on cases whose results are known: every call must
finish without an error and give the exact results.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
pytestmark = pytest.mark.gpu

SCRIPT = r'''
import os, sys
ROOT = sys.argv[1]
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "tests"))
import numpy as np
from paper_2506_01099_gb300 import benelux as B, build as Bd, workloads as W
B._build.LIB = Bd.CHECKED_LIB
B.lib(auto_build=False)
from paper_pins import theorem1_pairs
import oracle
orc = oracle.load()
MAX_HI = (1 << 41) + (1 << 31)
TUNES = [dict(), dict(tile_kind=3, tile_log2=16, seg_tiles=2, threads=512),
         dict(tile_kind=3, tile_log2=12, seg_tiles=8, threads=1024, small_q_log2=8),
         dict(tile_kind=2, tile_log2=15, seg_tiles=32), dict(tile_kind=0, tile_log2=15, threads=1024),
         dict(tile_kind=1)]
for tune in TUNES:
    with B.Context(0, max_hi=MAX_HI) as c:
        if tune:
            c.set_tune(**tune)
        assert c.search(1, 1 << 22) == theorem1_pairs(1, 1 << 22), tune
        lo, hi = 2**40 - 2**22, 2**40 + 2**22
        assert c.search(lo, hi) == theorem1_pairs(lo, hi), tune
        for cc in (3**25, 7**14):
            assert c.search(cc - 20000, cc + 20000) == orc.pairs_crt(cc - 20000, cc + 20000), (tune, cc)
        for rlo, n in ((2**40 - 2**13, 2**14 + 3), (3**25 - 3001, 6001)):
            rad = np.zeros(n, dtype=np.uint64)
            sq = np.zeros(n, dtype=np.uint64)
            c.rad_segment(rlo, n, rad.ctypes.data, sq.ctypes.data, None)
            assert np.array_equal(rad, orc.rad_td_array(rlo, n)), (tune, rlo)
with B.Context(0, max_hi=MAX_HI) as c:
    ivs = W.batch_intervals(64, seed=7)
    pairs, offs = B.bnx_batch(c.h, ivs, B.make_intervals(ivs))
    for i, iv in enumerate(ivs):
        got = [(m, n, k) for (_, m, n, k) in pairs[offs[i]:offs[i + 1]]]
        assert got == c.search(iv.lo, iv.hi, iv.kinds), i
    assert c.search_hash(1 << 20) == orc.pairs_sort(1 << 20)
    assert c.search_sorted(1 << 22) == theorem1_pairs(1, 1 << 22)
    assert c.search_chunked(1 << 20, chunk_log2=18) == orc.pairs_sort(1 << 20)
print("checked ok")
'''


def test_bounds_checked_build_runs_clean():
    from paper_2506_01099_gb300 import build as Bd

    Bd.build_checked()
    r = subprocess.run([sys.executable, "-c", SCRIPT, ROOT], capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0 and "checked ok" in r.stdout, (r.stdout[-2000:], r.stderr[-4000:])
