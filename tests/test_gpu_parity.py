"""CUDA path vs the oracle, element by element, through the C ABI (GPU only).

Radicals are compared bit-exactly on segments that span several tiles and
queue segments with a ragged tail; pair sets are compared exactly (they are
integer results, unique once sorted by (n, m, kind)); the survivor counts of
the per-kind necessary conditions are compared exactly with the oracle's.
"""
import math

import numpy as np
import pytest

from paper_pins import theorem1_pairs

pytestmark = pytest.mark.gpu

MAX_HI = (1 << 41) + (1 << 31)


@pytest.fixture(scope="module")
def B():
    from paper_2506_01099_gb300 import benelux

    return benelux


@pytest.fixture(scope="module")
def ctx(B):
    c = B.Context(0, max_hi=MAX_HI)
    yield c
    c.close()


def gpu_rad(ctx, lo, length):
    import torch

    rad = torch.empty(length, dtype=torch.int64, device="cuda")
    sq = torch.empty(length, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    ctx.rad_segment(lo, length, rad.data_ptr(), sq.data_ptr(), stream)
    torch.cuda.synchronize()
    return rad.cpu().numpy().view(np.uint64), sq.cpu().numpy().view(np.uint64)


def test_prime_count(ctx, orc):
    assert ctx.prime_count() == orc.nprimes_upto(math.isqrt(MAX_HI))


RAD_CASES = [
    (1, 70_000),                      # start at 1, several tiles, ragged tail
    (2, 1),                           # a single value
    (9, 100),                         # starts on a prime square
    (2**32 - 40_000, 90_001),         # across 2^32, several queue segments
    (1048573**2 - 5000, 10_001),      # around a large prime square
    (3**25 - 3000, 6000),             # around a high prime power
    (2**40 - 2**13, 2**14 + 3),       # across 2^40
    (1_400_000_000_000 - 4096, 8193),
]


@pytest.mark.parametrize("lo,length", RAD_CASES)
def test_rad_segment_bit_exact(ctx, orc, lo, length):
    rad, sq = gpu_rad(ctx, lo, length)
    want = orc.rad_td_array(lo, length)
    assert np.array_equal(rad, want), int(np.nonzero(rad != want)[0][0])
    xs = np.arange(lo, lo + length, dtype=np.uint64)
    assert np.array_equal(sq * rad, xs)


def test_rad_segment_unaligned_outputs(ctx, orc):
    """The kernel writes two values per 16-byte store when both output pointers are 16-byte
    aligned, and one value at a time otherwise: output pointers 8 bytes past a 16-byte
    boundary (one or both, and the radical alone) give the same values as aligned ones,
    which equal the oracle's trial-division radicals."""
    import torch

    stream = torch.cuda.current_stream().cuda_stream
    for lo, length in ((2**40 - 2**13, 2**14 + 3), (3**25 - 3001, 6001), (1, 70_000)):
        want = orc.rad_td_array(lo, length)
        rad_a, sq_a = gpu_rad(ctx, lo, length)
        assert np.array_equal(rad_a, want)
        for shift_rad, shift_sq in ((1, 1), (0, 1), (1, 0)):
            rb = torch.zeros(length + 2, dtype=torch.int64, device="cuda")
            qb = torch.zeros(length + 2, dtype=torch.int64, device="cuda")
            ctx.rad_segment(lo, length, rb.data_ptr() + 8 * shift_rad, qb.data_ptr() + 8 * shift_sq, stream)
            torch.cuda.synchronize()
            r = rb.cpu().numpy().view(np.uint64)
            q = qb.cpu().numpy().view(np.uint64)
            assert np.array_equal(r[shift_rad:shift_rad + length], want), (lo, shift_rad, shift_sq)
            assert np.array_equal(q[shift_sq:shift_sq + length], sq_a), (lo, shift_rad, shift_sq)
            # nothing written outside the outputs
            assert r[length + shift_rad:].sum() == 0 and r[:shift_rad].sum() == 0
            assert q[length + shift_sq:].sum() == 0 and q[:shift_sq].sum() == 0
        rb = torch.zeros(length + 1, dtype=torch.int64, device="cuda")
        ctx.rad_segment(lo, length, rb.data_ptr() + 8, None, stream)
        torch.cuda.synchronize()
        assert np.array_equal(rb.cpu().numpy().view(np.uint64)[1:], want), lo


def test_rad_segment_large_sampled(ctx, orc):
    """A 2^27-value segment at 2^40 (many queue segments): sampled windows vs trial division."""
    lo, length = 2**40 + 12345, 1 << 27
    rad, _ = gpu_rad(ctx, lo, length)
    rng = np.random.default_rng(5)
    for off in list(rng.integers(0, length - 512, 12)) + [0, length - 512]:
        off = int(off)
        assert np.array_equal(rad[off:off + 512], orc.rad_td_array(lo + off, 512)), off


@pytest.mark.parametrize("tune", [dict(tile_log2=12, seg_tiles=1, small_q_log2=10),
                                  dict(tile_log2=14, seg_tiles=4, threads=1024, small_q_log2=16),
                                  dict(tile_log2=11, seg_tiles=16, threads=256, small_q_log2=8),
                                  dict(tile_kind=1),
                                  dict(tile_kind=1, tile_log2=12, threads=256, small_q_log2=12),
                                  dict(tile_kind=2),
                                  dict(tile_kind=2, tile_log2=13, threads=128, small_q_log2=16),
                                  dict(tile_kind=2, tile_log2=14, threads=512, seg_tiles=2, small_q_log2=10),
                                  dict(tile_kind=1, tile_log2=15, seg_tiles=2),
                                  dict(tile_kind=0, tile_log2=15, threads=1024),
                                  # 2^19-value segments (the packed bucket cache at its offset limit) with
                                  # Q = 2^8: far more entries than the 1024 cached ones
                                  dict(tile_kind=2, tile_log2=15, seg_tiles=16, small_q_log2=8),
                                  # 2^20-value segments: the cache is off, every entry read from HBM
                                  dict(tile_kind=2, tile_log2=15, seg_tiles=32),
                                  dict(tile_kind=0, tile_log2=14, seg_tiles=64, small_q_log2=9),
                                  dict(tile_kind=3),
                                  dict(tile_kind=3, tile_log2=13, threads=128, small_q_log2=16),
                                  dict(tile_kind=3, tile_log2=16, seg_tiles=2, threads=512),
                                  dict(tile_kind=3, tile_log2=12, seg_tiles=8, threads=1024, small_q_log2=8),
                                  dict(tile_kind=3, tile_log2=15, seg_tiles=32),
                                  dict(tile_kind=2, tile_log2=16, seg_tiles=4)])
def test_tunings_agree(B, orc, tune):
    with B.Context(0, max_hi=1 << 41) as c:
        c.set_tune(**tune)
        for lo, length in [(1, 50_000), (2**40 - 20_000, 40_001)]:
            rad, _ = gpu_rad(c, lo, length)
            assert np.array_equal(rad, orc.rad_td_array(lo, length))
        assert c.search(1, 1 << 20) == theorem1_pairs(1, 1 << 20)
        st = c.stats()
        assert (st["survivors1"], st["survivors2"]) == orc.filter_counts(1, 1 << 20)
        assert c.search(2**40 - 2**21 - 8, 2**40 + 2**21 + 8) == theorem1_pairs(2**40 - 2**21 - 8, 2**40 + 2**21 + 8)
        assert c.search_hash(1 << 20) == orc.pairs_sort(1 << 20)
        assert c.stats()["hash_keys"] == orc.hash_keys(1 << 20)


@pytest.mark.parametrize("tune", [dict(tile_kind=3), dict(tile_kind=3, tile_log2=16, seg_tiles=2, threads=512),
                                  dict(tile_kind=2, tile_log2=15, seg_tiles=32), dict(tile_kind=1)])
def test_neighbours_of_2p16_multiples_at_tile_edges(B, orc, tune):
    """n next to a multiple of 2^16 are always candidates (their power of 2 can exceed the
    log bound's 2^14).  n = 2^40 - 1 (rad(n) rad(n+1) ~ 2^41/5) survives the filters of both
    kinds and sits on a tile edge here: a tile of 2^16 values starting at a multiple of 2^16
    holds two multiples, and its last value is such an n.  Survivor counts and pairs equal
    the oracle's."""
    windows = [(2**40 - 2**16, 2**40 + 2**16), (2**40 - 2**17 + 1, 2**40 + 1), (2**40 - 1, 2**40 + 1),
               (2**40 - 2**16, 2**40), (2**40, 2**40 + 3)]
    with B.Context(0, max_hi=1 << 41) as c:
        c.set_tune(**tune)
        for lo, hi in windows:
            assert c.search(lo, hi) == orc.pairs_crt(lo, hi), (lo, hi)
            st = c.stats()
            assert (st["survivors1"], st["survivors2"]) == orc.filter_counts(lo, hi), (lo, hi)
    assert orc.filter_counts(2**40 - 1, 2**40) == (1, 1) and orc.filter_counts(2**40, 2**40 + 1) == (0, 0)


def test_search_c1_full(ctx, orc):
    """All n < 2^24, both kinds: equals the oracle and Theorem 1 (25 pairs)."""
    got = ctx.search(1, 1 << 24)
    assert got == orc.pairs_crt(1, 1 << 24)
    assert got == theorem1_pairs(1, 1 << 24)
    assert len(got) == 25
    st = ctx.stats()
    assert (st["survivors1"], st["survivors2"]) == orc.filter_counts(1, 1 << 24)


@pytest.mark.parametrize("kinds", [1, 2])
def test_search_single_kind(ctx, orc, kinds):
    got = ctx.search(1, 1 << 22, kinds)
    assert got == orc.pairs_crt(1, 1 << 22, kinds)
    st = ctx.stats()
    c1, c2 = orc.filter_counts(1, 1 << 22, kinds)
    assert (st["survivors1"], st["survivors2"]) == (c1, c2)


def test_filter_counts_high_window(ctx, orc):
    lo, hi = 2**40 - 2**23, 2**40 + 2**23
    got = ctx.search(lo, hi)
    assert got == orc.pairs_crt(lo, hi)
    st = ctx.stats()
    assert (st["survivors1"], st["survivors2"]) == orc.filter_counts(lo, hi)


@pytest.mark.parametrize("tile_kind", [0, 2, 3])
def test_log_tiles_at_large_square_parts(B, orc, tile_kind):
    """Windows around the n below 2^42 with the largest odd square parts (3^26, 5^17, 7^14,
    2 * 3^25), where the log-domain tile values and pair sums are largest: pairs and
    survivor counts equal the oracle's for every tile width."""
    with B.Context(0, max_hi=1 << 42) as c:
        c.set_tune(tile_kind=tile_kind)
        for center in (3**26, 5**17, 7**14, 2 * 3**25):
            lo, hi = center - 12_000, center + 12_000
            assert c.search(lo, hi) == orc.pairs_crt(lo, hi), center
            st = c.stats()
            assert (st["survivors1"], st["survivors2"]) == orc.filter_counts(lo, hi), center


def test_search_edges(ctx, orc):
    # intervals whose ends sit exactly on pair members
    for m, n, kind in theorem1_pairs(1, 1 << 40):
        for lo, hi in ((n, n + 1), (n - 1, n), (n + 1, n + 2), (max(1, n - 3), n + 3)):
            assert ctx.search(lo, hi) == theorem1_pairs(lo, hi), (lo, hi)
    assert ctx.search(1, 2) == []
    assert ctx.search(2, 4) == [(2, 3, 2)]
    assert ctx.search(MAX_HI - 1000, MAX_HI) == orc.pairs_crt(MAX_HI - 1000, MAX_HI)


def test_search_c2_full_range(ctx):
    """All n < 2^32 (configured with 2^16-integer segments): the 33 pairs of Theorem 1."""
    ctx.set_tune(tile_log2=13, seg_tiles=8)
    got = ctx.search(1, 1 << 32)
    assert got == theorem1_pairs(1, 1 << 32)
    assert len(got) == 33


def test_hash_search(ctx, orc):
    assert ctx.search_hash(1 << 20) == orc.pairs_sort(1 << 20)
    assert ctx.stats()["hash_keys"] == orc.hash_keys(1 << 20)
    assert ctx.search_hash(1 << 24) == theorem1_pairs(1, 1 << 24)
    assert ctx.search_hash(1 << 24, 2) == theorem1_pairs(1, 1 << 24, 2)


def test_hash_search_c2(ctx):
    assert ctx.search_hash(1 << 32) == theorem1_pairs(1, 1 << 32)


def test_large_window_sample(ctx):
    """The first 2^30 integers of [2^40, 2^40 + 2^37): exactly one second-kind pair."""
    lo = 1 << 40
    assert ctx.search(lo, lo + (1 << 30)) == [(1048577, 1099513724928, 2)]
    hi = 1_400_000_000_000
    assert ctx.search(hi - (1 << 28), hi) == []


def test_batch_ragged_vs_oracle(ctx, orc):
    ivs = [(1, 2, 3), (2, 4, 3), (5, 1000, 1), (1000, 70_000, 2), (1, 1 << 16, 3), (2**33 + 1, 2**33 + 77_777, 3),
           (17179607040 - 100, 17179607040 + 1, 1), (17180131328, 17180131329, 2), (2**40 - 2**21, 2**40 - 2**21 + 1, 3),
           (2**40 + 2**21 - 5, 2**40 + 2**21 + 5, 3)]
    pairs, offs = ctx.batch(ivs)
    assert len(offs) == len(ivs) + 1
    for i, (lo, hi, k) in enumerate(ivs):
        mine = [(m, n, kd) for (v, m, n, kd) in pairs[offs[i]:offs[i + 1]]]
        assert all(v == i for (v, _, _, _) in pairs[offs[i]:offs[i + 1]])
        assert mine == orc.pairs_crt(lo, hi, k), (lo, hi, k)


def test_batch_equals_plain(ctx):
    from paper_2506_01099_gb300 import workloads as W

    ivs = [iv for iv in W.batch_intervals(256) if iv.length <= (1 << 24)][:64]
    pairs, offs = ctx.batch(ivs)
    for i, iv in enumerate(ivs):
        mine = [(m, n, kd) for (_, m, n, kd) in pairs[offs[i]:offs[i + 1]]]
        assert mine == ctx.search(iv.lo, iv.hi, iv.kinds)
        assert mine == theorem1_pairs(iv.lo, iv.hi, iv.kinds)


def test_batch_family_members(ctx):
    """Intervals of the batched workload's shape placed on every family member above 2^32."""
    ivs = []
    for m, n, kind in theorem1_pairs(1 << 32):
        ivs.append((n - (1 << 16), n + (1 << 16), kind))
        ivs.append((n - (1 << 20) + 7, n + 1, 3 - kind))  # the other kind: nothing
    pairs, offs = ctx.batch(ivs)
    for i, (lo, hi, k) in enumerate(ivs):
        mine = [(m, n, kd) for (_, m, n, kd) in pairs[offs[i]:offs[i + 1]]]
        assert mine == theorem1_pairs(lo, hi, k)


def test_batched_workload_full_size(B, orc):
    """The benchmark's own step at full size and in its launch configuration (the default
    tuning): 4096 seeded intervals in [2^32, 2^40), 4.6e11 integers.  Every interval's
    pairs are its Theorem 1 family members (the theorem is complete below 1.4e12), and
    sampled intervals, and sampled windows of long ones, equal the oracle's."""
    from paper_2506_01099_gb300 import workloads as W

    ivs = W.batch_intervals(4096)
    with B.Context(0, max_hi=MAX_HI) as c:
        pairs, offs = c.batch(ivs)
        assert len(offs) == len(ivs) + 1
        for i, iv in enumerate(ivs):
            mine = [(m, n, kd) for (_, m, n, kd) in pairs[offs[i]:offs[i + 1]]]
            assert mine == theorem1_pairs(iv.lo, iv.hi, iv.kinds), i
        rng = np.random.default_rng(11)
        short = [i for i, iv in enumerate(ivs) if iv.hi - iv.lo <= (1 << 20)]
        for i in rng.choice(short, 12, replace=False):
            iv = ivs[int(i)]
            mine = [(m, n, kd) for (_, m, n, kd) in pairs[offs[i]:offs[i + 1]]]
            assert mine == orc.pairs_crt(iv.lo, iv.hi, iv.kinds), iv
        # windows of long intervals searched alone with the same tuning, against the oracle
        # (pairs and the survivor counts of the per-kind conditions)
        long_ = [iv for iv in ivs if iv.hi - iv.lo >= (1 << 26)]
        for k in rng.choice(len(long_), 4, replace=False):
            iv = long_[int(k)]
            lo = iv.lo + int(rng.integers(0, iv.hi - iv.lo - (1 << 21)))
            assert c.search(lo, lo + (1 << 21), iv.kinds) == orc.pairs_crt(lo, lo + (1 << 21), iv.kinds)
            st = c.stats()
            assert (st["survivors1"], st["survivors2"]) == orc.filter_counts(lo, lo + (1 << 21), iv.kinds)


def test_large_windows_full(ctx):
    """The two large windows whole: [2^40, 2^40 + 2^37) holds exactly Theorem 1's
    second-kind member (2^20 + 1, 2^40 + 2^21), [1.3e12, 1.4e12) nothing; the plain call
    and the batch of 2^30-integer pieces agree."""
    from paper_2506_01099_gb300 import workloads as W

    for which in (0, 1):
        lo, hi = W.LARGE_WINDOWS[which]
        want = theorem1_pairs(lo, hi)
        assert ctx.search(lo, hi) == want
        pairs, _ = ctx.batch(W.large_window_intervals(which))
        assert sorted((m, n, kd) for (_, m, n, kd) in pairs) == want
    assert theorem1_pairs(*W.LARGE_WINDOWS[0]) == [(1048577, 1099513724928, 2)]
    assert theorem1_pairs(*W.LARGE_WINDOWS[1]) == []


def test_bad_arguments(B, ctx):
    for args in ((0, 10, 3), (10, 10, 3), (5, 4, 3), (1, MAX_HI + 1, 3), (1, 10, 0), (1, 10, 8)):
        with pytest.raises(B.BnxError) as e:
            ctx.search(*args)
        assert e.value.code == B.BNX_E_ARG


def test_server_alone_vs_mix(B, ctx):
    """Requests served concurrently return what each returns alone."""
    reqs = [(2**40 - 2**23, 2**40 + 2**23, 3), (1, 1 << 22, 3), (2**36 - 5, 2**36 + 2**25, 2),
            (17179607040 - 2**24, 17179607040 + 2**20, 1), (1_300_000_000_000, 1_300_000_000_000 + 2**26, 3)]
    alone = [ctx.search(*r) for r in reqs]
    B.bnx_server_start(ctx.h, max_active=3, slice_len=1 << 22)
    try:
        tickets = [B.bnx_server_submit(ctx.h, *r) for r in reqs]
        got = {}
        import time

        t0 = time.time()
        while len(got) < len(tickets) and time.time() - t0 < 120:
            for t in tickets:
                if t not in got:
                    r = B.bnx_server_poll(ctx.h, t)
                    if r is not None:
                        got[t] = r
            time.sleep(0.005)
    finally:
        B.bnx_server_stop(ctx.h)
    assert len(got) == len(tickets)
    for t, want in zip(tickets, alone):
        pairs, lat = got[t]
        assert pairs == want
        assert lat > 0


def test_theorem1_full_range(B):
    """The paper's whole computation (Theorem 1): every pair of either kind with
    n < 1.4e12 is one of the listed families or exceptional pairs."""
    from paper_pins import THEOREM1_BOUND

    with B.Context(0, max_hi=THEOREM1_BOUND) as c:
        got = c.search(1, THEOREM1_BOUND, 7)  # both kinds and the three-term question
        st = c.stats()
    assert got == theorem1_pairs(1, THEOREM1_BOUND)  # in particular, no three-term pair
    assert len(got) == 42  # 20 of the first kind, 22 of the second
    assert st["integers"] == THEOREM1_BOUND - 1


def test_three_term_kind(ctx, orc):
    """Bit 4 (Erdos's three-term question) reports nothing where the oracle does not."""
    assert ctx.search(1, 1 << 22, 4) == orc.pairs_crt(1, 1 << 22, 4) == []
    assert ctx.search(1, 1 << 32, 5) == theorem1_pairs(1, 1 << 32, 1)
    lo = 2**40 - 2**22
    assert ctx.search(lo, lo + 2**23, 6) == orc.pairs_crt(lo, lo + 2**23, 6)


def test_algorithm3_chunked(ctx, orc):
    """The paper's Algorithm 3 (all earlier chunks re-sieved and probed) finds the
    same pairs as the oracle, with S not a multiple of the chunk."""
    S = (1 << 20) + 12345
    got = ctx.search_chunked(S, 16)
    assert got == orc.pairs_sort(S)
    assert ctx.search_chunked(1 << 22, 18, 2) == theorem1_pairs(1, 1 << 22, 2)
    assert ctx.search_chunked(1 << 22, 18, 1) == theorem1_pairs(1, 1 << 22, 1)


@pytest.mark.parametrize("S", [3, 4, 5, 100, 7169, 7168 * 3 + 17, 8192 * 3 + 17, (1 << 20) + 12345])
def test_algorithm2_sorted(ctx, orc, S):
    """The paper's Algorithm 2 by a device radix sort: the same pairs as the
    oracle's sort-based search, with ragged last sort tiles and tiny S."""
    assert ctx.search_sorted(S) == orc.pairs_sort(S)


def test_algorithm2_sorted_kinds_and_scale(ctx, orc):
    """Single kinds, and S = 2^30 (radix sort of 2^30 records over 149797 tiles)
    against the pairs of Theorem 1."""
    S = (1 << 22) + 3
    both = orc.pairs_sort(S)
    assert ctx.search_sorted(S, 1) == [p for p in both if p[2] == 1]
    assert ctx.search_sorted(S, 2) == [p for p in both if p[2] == 2]
    assert ctx.search_sorted(1 << 30) == theorem1_pairs(1, 1 << 30, 3)


def test_algorithm2_sorted_bad_arguments(B, ctx):
    for S, kinds in [(2, 3), ((1 << 32) + 1, 3), (1 << 20, 4), (1 << 20, 0)]:
        with pytest.raises(B.BnxError) as e:
            ctx.search_sorted(S, kinds)
        assert e.value.code == B.BNX_E_ARG


SEGMENT_CASES = [
    (1, 1 << 20),                         # from 1: the small pairs, (2, 3) first
    (2**32 - 2**19 - 17, 2**20 + 33),     # across 2^32, ragged
    (2**40 - 2**21, 2**21),               # ends at 2^40
    (2**40, 2**21 + 1),                   # starts at 2^40: holds (2^20 + 1, 2^40 + 2^21)
    (MAX_HI - 2**20, 2**20),              # ends at the context's max_hi
]


@pytest.mark.parametrize("lo,length", SEGMENT_CASES)
def test_search_segment_vs_oracle(ctx, orc, lo, length):
    """bnx_search_segment (Algorithm 3's output for one chunk) equals the oracle."""
    got = ctx.search_segment(lo, length)
    assert got == orc.pairs_crt(lo, lo + length)
    st = ctx.stats()
    assert (st["survivors1"], st["survivors2"]) == orc.filter_counts(lo, lo + length)


def test_search_segment_straddles_family_members(ctx):
    """Segments that start, end or sit on every pair member of Theorem 1 below 2^40."""
    for m, n, kind in theorem1_pairs(1, 1 << 40):
        for lo, length in ((n, 1), (max(1, n - 999), 1000), (max(1, n - 500), 1001), (n + 1, 4096)):
            assert ctx.search_segment(lo, length) == theorem1_pairs(lo, lo + length), (lo, length)
        assert ctx.search_segment(n, 1, 3 - kind) == theorem1_pairs(n, n + 1, 3 - kind)  # n = 8 has both kinds


def test_segment_loop_equals_search(ctx):
    """A caller's own loop of consecutive segments concatenates to bnx_search's result."""
    lo, hi = 2**40 - 2**22 - 5, 2**40 + 2**22 + 12345
    step = (1 << 20) + 7
    got = []
    for a in range(lo, hi, step):
        got += ctx.search_segment(a, min(step, hi - a))
    assert got == ctx.search(lo, hi) == theorem1_pairs(lo, hi)


def test_search_segment_bad_arguments(B, ctx):
    import ctypes

    L = B.lib()
    n = ctypes.c_size_t()
    for lo, length, kinds in ((0, 10, 3), (1, 0, 3), (MAX_HI - 9, 10, 3), (2**64 - 1, 2, 3), (2**64 - 5, 10, 3),
                              (1, 10, 0), (1, 10, 8)):
        assert L.bnx_search_segment(ctx.h, lo, length, kinds, None, 0, ctypes.byref(n)) == B.BNX_E_ARG, (lo, length)
    assert L.bnx_search_segment(ctx.h, MAX_HI - 10, 10, 3, None, 0, ctypes.byref(n)) == B.BNX_OK
    with B.Context(0, max_hi=1 << 20) as small:  # len beyond max_hi must not wrap the check
        assert L.bnx_search_segment(small.h, 1, 1 << 30, 3, None, 0, ctypes.byref(n)) == B.BNX_E_ARG


def test_rad_segment_host_buffers(ctx, orc):
    """bnx_rad_segment into HOST buffers (pageable numpy arrays): the same values as into
    device buffers, and the oracle's trial-division radicals."""
    for lo, length in ((2**40 - 2**13, 2**14 + 3), (1, 70_000)):
        rad = np.zeros(length, dtype=np.uint64)
        sq = np.zeros(length, dtype=np.uint64)
        ctx.rad_segment(lo, length, rad.ctypes.data, sq.ctypes.data, None)
        drad, dsq = gpu_rad(ctx, lo, length)
        assert np.array_equal(rad, drad) and np.array_equal(sq, dsq)
        assert np.array_equal(rad, orc.rad_td_array(lo, length))
        rad_only = np.zeros(length, dtype=np.uint64)
        ctx.rad_segment(lo, length, rad_only.ctypes.data, None, None)
        assert np.array_equal(rad_only, rad)


def test_rad_segment_bad_arguments(B, ctx):
    import ctypes

    import torch

    L = B.lib()
    dev = torch.empty(16, dtype=torch.int64, device="cuda")
    host = np.zeros(16, dtype=np.uint64)
    for lo, length in ((0, 4), (1, 0), (2**64 - 1, 2), (2**64 - 8, 16), (MAX_HI - 3, 4), (1, (1 << 31) + 1)):
        assert L.bnx_rad_segment(ctx.h, lo, length, dev.data_ptr(), None, None) == B.BNX_E_ARG, (lo, length)
    # rad and sq must both be host or both device buffers
    assert L.bnx_rad_segment(ctx.h, 5, 16, dev.data_ptr(), host.ctypes.data, None) == B.BNX_E_ARG
    assert L.bnx_rad_segment(ctx.h, 5, 16, None, None, None) == B.BNX_E_ARG
    torch.cuda.synchronize()


def test_algorithm2_lookback_wait_runs_out(B, ctx, orc):
    """The radix sort's bounded look-back wait: with the test hook, tile 0 of the first
    pass withholds its counts, the waits on it give up after 1024 polls, and the call
    fails with BNX_E_TIMEOUT instead of stalling; the next call is clean."""
    import ctypes

    L = B.lib()
    assert L.bnx_arm_lookback_timeout(ctx.h, 0) == B.BNX_E_ARG
    assert L.bnx_arm_lookback_timeout(ctx.h, (1 << 22) + 1) == B.BNX_E_ARG
    S = 1 << 16  # 10 sort tiles
    B.bnx_arm_lookback_timeout(ctx.h, 1024)
    n = ctypes.c_size_t(12345)
    assert L.bnx_search_sorted(ctx.h, S, 3, None, 0, ctypes.byref(n)) == B.BNX_E_TIMEOUT
    assert "look-back" in B.bnx_last_error()
    assert ctx.search_sorted(S) == orc.pairs_sort(S)  # disarmed
    assert ctx.search(1, 1 << 20) == theorem1_pairs(1, 1 << 20)


def test_server_admission_by_memory(B, orc):
    """A workspace budget that holds one request's slice but not two: the second and
    third requests wait for memory (first come, first served), the workspace never
    exceeds the budget, and every request's pairs equal its result alone, Theorem 1 and
    the oracle."""
    import time

    sl = 1 << 30
    base = 1 << 40
    reqs = [(base + i * 2 * sl, base + (i + 1) * 2 * sl, 3) for i in range(3)]
    with B.Context(0, max_hi=MAX_HI) as c:
        one = B.bnx_workspace_bytes(c.h, [(reqs[0][0], reqs[0][0] + sl, 3)])
        two = B.bnx_workspace_bytes(c.h, [(r[0], r[0] + sl, 3) for r in reqs[:2]])
        assert two > one > 0
        budget = (one + two) // 2
        alone = [c.search(*r) for r in reqs]
        B.bnx_server_start(c.h, max_active=4, slice_len=sl, mem_budget=budget)
        try:
            tickets = [B.bnx_server_submit(c.h, *r) for r in reqs]
            got = {}
            t0 = time.time()
            while len(got) < len(tickets) and time.time() - t0 < 300:
                for t in tickets:
                    if t not in got:
                        r = B.bnx_server_poll(c.h, t)
                        if r is not None:
                            got[t] = r
                time.sleep(0.002)
        finally:
            B.bnx_server_stop(c.h)
        st = B.bnx_server_get_stats(c.h)
    assert len(got) == 3
    assert st["submitted"] == 3 and st["completed"] == 3 and st["rejected"] == 0
    assert st["deferred"] == 2, st  # the second and the third request waited for memory
    assert st["budget_bytes"] == budget and 0 < st["ws_peak_bytes"] <= budget, st
    assert st["iterations"] >= 6  # slices shortened to fit: 2^30 integers per iteration
    lat = [got[t][1] for t in tickets]
    assert lat[0] < lat[1] < lat[2]  # one after the other
    for t, r, want in zip(tickets, reqs, alone):
        assert got[t][0] == want == theorem1_pairs(r[0], r[1]) == orc.pairs_crt(r[0], r[1])
    assert alone[0] == [(1048577, 1099513724928, 2)]


def test_search_checkpointed_resumes(B, ctx, orc, tmp_path):
    """A long search run in chunks stops after a few (its progress in the checkpoint
    file), is read back without searching, resumes in a new context (as after a restart)
    and ends with exactly the pairs of one uninterrupted search; the file refuses another
    search and a corrupt file is refused."""
    lo, hi = 2**40 - 2**22, 2**40 + 2**22 + 12345  # both kinds' family members near 2^40
    want = theorem1_pairs(lo, hi)
    assert len(want) == 2 and want == orc.pairs_crt(lo, hi)
    path, chunk = str(tmp_path / "search.ckpt"), 1 << 20
    got, nxt, fin = ctx.search_checkpointed(lo, hi, 3, path, chunk, max_chunks=3)
    assert not fin and nxt == lo + 3 * chunk and got == [p for p in want if p[1] < nxt]
    assert ctx.search_checkpointed(lo, hi, 3, path, chunk, max_chunks=0) == (got, nxt, False)
    with B.Context(0, max_hi=MAX_HI) as c2:
        got2, nxt2, fin2 = c2.search_checkpointed(lo, hi, 3, path, chunk)
    assert fin2 and nxt2 == hi and got2 == want == ctx.search(lo, hi)
    assert ctx.search_checkpointed(lo, hi, 3, path, chunk) == (want, hi, True)  # finished: no search
    with pytest.raises(B.BnxError) as e:
        ctx.search_checkpointed(lo, hi + 1, 3, path, chunk)
    assert e.value.code == B.BNX_E_STATE
    with open(path, "rb") as f:
        good = f.read()
    for bad in (b"NOTACKPT" + good[8:], good[:-10], good + b"x"):  # a corrupt header, cut or padded
        with open(path, "wb") as f:
            f.write(bad)
        with pytest.raises(B.BnxError) as e:
            ctx.search_checkpointed(lo, hi, 3, path, chunk)
        assert e.value.code == B.BNX_E_ARG


def test_server_cancel(B):
    """A waiting request cancelled is dropped at once, an active one is retired at the end
    of its iteration; both poll as BNX_E_CANCELLED, the counters record them, and the
    request behind them still gets exactly its pairs."""
    import time

    with B.Context(0, max_hi=MAX_HI) as c:
        B.bnx_server_start(c.h, max_active=1, slice_len=1 << 26)  # one slot: the others wait
        try:
            big = B.bnx_server_submit(c.h, 2**40, 2**40 + 2**38)  # about four thousand iterations
            small = B.bnx_server_submit(c.h, 1, 1 << 20)
            lo, hi = 2**40 - 2**22, 2**40 + 2**22
            last = B.bnx_server_submit(c.h, lo, hi)
            B.bnx_server_cancel(c.h, small)
            time.sleep(0.05)
            assert B.bnx_server_poll(c.h, big) is None  # still running
            B.bnx_server_cancel(c.h, big)
            B.bnx_server_cancel(c.h, big)  # a second cancel changes nothing
            with pytest.raises(B.BnxError) as e:
                B.bnx_server_cancel(c.h, 10**9)
            assert e.value.code == B.BNX_E_ARG
            codes = {}
            got = None
            t0 = time.time()
            while (len(codes) < 2 or got is None) and time.time() - t0 < 120:
                for t in (big, small):
                    if t not in codes:
                        try:
                            if B.bnx_server_poll(c.h, t) is not None:
                                codes[t] = B.BNX_OK
                        except B.BnxError as err:
                            codes[t] = err.code
                if got is None:
                    got = B.bnx_server_poll(c.h, last)
                time.sleep(0.002)
            st = B.bnx_server_get_stats(c.h)
        finally:
            B.bnx_server_stop(c.h)
    assert codes == {big: B.BNX_E_CANCELLED, small: B.BNX_E_CANCELLED}
    assert got is not None and got[0] == theorem1_pairs(lo, hi)
    assert st["cancelled"] == 2 and st["completed"] == 3 and st["submitted"] == 3, st


def test_server_rejects_a_request_that_never_fits(B):
    """A budget below one slice's workspace: the request finishes at once with BNX_E_NOMEM."""
    import time

    with B.Context(0, max_hi=MAX_HI) as c:
        need = B.bnx_workspace_bytes(c.h, [(1 << 40, (1 << 40) + (1 << 26), 3)])
        B.bnx_server_start(c.h, max_active=2, slice_len=1 << 26, mem_budget=need // 2)
        try:
            t = B.bnx_server_submit(c.h, 1 << 40, (1 << 40) + (1 << 26), 3)
            t0 = time.time()
            while time.time() - t0 < 60:
                try:
                    r = B.bnx_server_poll(c.h, t)
                except B.BnxError as e:
                    assert e.code == B.BNX_E_NOMEM
                    break
                assert r is None
                time.sleep(0.002)
            else:
                raise AssertionError("no answer")
        finally:
            B.bnx_server_stop(c.h)
        st = B.bnx_server_get_stats(c.h)
    assert st["rejected"] == 1 and st["iterations"] == 0


def test_autotune_picks_a_sound_tuning(B, orc):
    """bnx_autotune over 64 intervals of the batched workload (one timed round per
    candidate): the JSON it returns parses, every field lies in its search space, the
    context keeps that tuning, and searches with it equal Theorem 1 and the oracle
    (pairs and survivor counts)."""
    import json

    from paper_2506_01099_gb300 import workloads as W

    ivs = [iv for iv in W.batch_intervals(4096) if iv.length <= (1 << 26)][:64]
    with B.Context(0, max_hi=MAX_HI) as c:
        text = c.autotune(ivs, rounds=1)
        d = json.loads(text)
        assert set(d) == {"tile_log2", "seg_tiles", "threads", "ctas_per_sm", "small_q_log2", "tile_kind", "ms"}
        assert d["tile_log2"] in (13, 14, 15, 16) and d["seg_tiles"] in (2, 4, 8, 16, 32)
        assert d["threads"] in (128, 256, 512, 1024) and d["small_q_log2"] in (12, 13, 14, 15, 16)
        assert d["ctas_per_sm"] in (0, 1, 2) and d["tile_kind"] in (0, 2, 3) and d["ms"] > 0
        tuned = c.tune()
        assert tuned == {k: v for k, v in d.items() if k != "ms"}
        assert B.bnx_tune_parse(text).as_dict() == tuned
        assert c.search(1, 1 << 20) == theorem1_pairs(1, 1 << 20)
        lo = 1 << 40
        assert c.search(lo, lo + (1 << 21)) == orc.pairs_crt(lo, lo + (1 << 21))
        st = c.stats()
        assert (st["survivors1"], st["survivors2"]) == orc.filter_counts(lo, lo + (1 << 21))
        pairs, offs = c.batch(ivs)
        for i, iv in enumerate(ivs):
            assert [(m, n, kd) for (_, m, n, kd) in pairs[offs[i]:offs[i + 1]]] == theorem1_pairs(iv.lo, iv.hi, iv.kinds)


def test_same_rad_on_constructed_pairs(B, orc):
    """The gcd strips behind the three-term test (rad(m+2) = rad(n+2), Sec. 1) on pairs
    built from chosen factorisations -- equal prime supports with different exponents,
    one prime swapped, edge values -- and on random pairs against the oracle's radicals."""
    import math

    rng = np.random.default_rng(7)
    small = [2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37, 41, 43, 47, 53, 59, 61, 67, 71, 73, 79, 83, 89, 97]
    big = [1000003, 2147483647, 4294967291]
    xs, ys, want = [], [], []

    def add(x, y, w):
        xs.append(x)
        ys.append(y)
        want.append(w)

    for _ in range(3000):
        k = int(rng.integers(1, 5))
        supp = [int(p) for p in rng.choice(small, k, replace=False)]
        if rng.random() < 0.3:
            supp[0] = int(rng.choice(big))
        x = y = 1
        for p in supp:
            x *= p ** int(rng.integers(1, 4))
            y *= p ** int(rng.integers(1, 4))
        if x >= 1 << 63 or y >= 1 << 63:
            continue
        if rng.random() < 0.5:
            add(x, y, True)
        else:  # swap one prime of y's support for one outside it
            p = supp[int(rng.integers(0, k))]
            q = next(int(v) for v in rng.permutation(small) if int(v) not in supp)
            y2 = y
            while y2 % p == 0:
                y2 //= p
            y2 *= q
            if y2 < 1 << 63:
                add(x, y2, False)
    for x, y, w in ((1, 1, True), (1, 2, False), (2, 1, False), (2**62, 2, True), (3**39, 3, True), (3 * 2**40, 6, True),
                    (6, 10, False), (2147483647 * 3, 2147483647, False), (2147483647**2, 2147483647, True),
                    (1000003 * 65537, 1000003**2 * 65537, True), (77, 1217, False)):
        add(x, y, w)
    for x, y in rng.integers(1, 1 << 40, size=(500, 2)):
        add(int(x), int(y), orc.rad_td(int(x)) == orc.rad_td(int(y)))
    for m, n, _ in theorem1_pairs(1, 1 << 40, 1):  # the families fail the three-term question (Sec. 1)
        add(m + 2, n + 2, orc.rad_td(m + 2) == orc.rad_td(n + 2))
    got = B.bnx_same_rad(xs, ys)
    bad = [(xs[i], ys[i], want[i]) for i in range(len(xs)) if bool(got[i]) != want[i]]
    assert not bad, bad[:5]
    assert sum(want) > 1000 and len(want) - sum(want) > 1000


def test_rad_segment_square_parts_past_2p32(ctx, orc):
    """Values whose odd square part passes 2^32 (the radical tile's 32-bit products give
    way to an exact recomputation): windows around odd prime powers with exponent large
    enough, and multiples of 3^21, against the oracle's trial division, rad and square
    part both."""
    centres = [3**22, 2 * 3**22, 4 * 3**23, 3**25, 7**13, 5**16, 11**11, 13**10, 17**9, 3**20 * 5**3,
               25 * 3**21, 49 * 3**21, 121 * 3**21]
    seen = 0
    for c in centres:
        lo = c - 700
        rad, sq = gpu_rad(ctx, lo, 1401)
        want = orc.rad_td_array(lo, 1401)
        assert np.array_equal(rad, want), (c, int(np.nonzero(rad != want)[0][0]))
        xs = np.arange(lo, lo + 1401, dtype=np.uint64)
        assert np.array_equal(sq * rad, xs), c
        odd_sq = [int(v) >> (int(v) & -int(v)).bit_length() - 1 if v else 0 for v in sq]
        seen += sum(1 for v in odd_sq if v >= 1 << 32)
    assert seen >= len(centres)  # every window holds at least its centre (odd square part > 2^32)
