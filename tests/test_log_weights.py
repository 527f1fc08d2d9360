"""The log-domain filter's per-prime weights are exact integers.

The log tiles reject n when a sum of per-prime weights -- an upper bound of
F log2 of the odd square part of n(n+1), F units per bit -- cannot meet the
per-kind necessary condition.  That rejection loses no pair only if every
weight w(p) is at least F log2 p, i.e. 2^w(p) > p^F.  The library computes the
weights in integers (bnx_log_weight: repeated squaring with upward rounding,
F = 2^f, for the u16 and u32 tiles; bnx_log_weight54: ceil(bitlen(p^5) / 4),
F = 5/4, for the u8 tile); these tests compare them with Python's exact
big-integer bit lengths, (p**F).bit_length() = floor(F log2 p) + 1:

* CPU: the host build of both weight functions for every prime below 2^21 (all
  primes a context up to 2^42 holds), bnx_log_weight at F = 2, 128 and 256 and
  at F = 2^16 for the primes below 2^8 (the only ones struck inside a tile:
  q = p^2 <= 2^16); and the bound that keeps the u8 tile's pair sums below 2^7;
* GPU: the weights the device kernels themselves use, per tile kind, read back
  along the kernels' code paths (bnx_log_weights).
"""
import math

import numpy as np
import pytest

PRIME_LIMIT = 1 << 21  # sqrt(2^42): the largest prime table a context holds


def primes_below(n):
    s = np.ones(n, dtype=bool)
    s[:2] = False
    for i in range(2, int(n ** 0.5) + 1):
        if s[i]:
            s[i * i::i] = False
    return np.nonzero(s)[0]


@pytest.fixture(scope="module")
def primes():
    return primes_below(PRIME_LIMIT)


@pytest.fixture(scope="module")
def exact(primes):
    """Exact bit lengths of p^F for every prime, F = 2, 128, 256 (Python big integers)."""
    ps = primes.tolist()
    return {F: np.array([(p ** F).bit_length() for p in ps], dtype=np.int64) for F in (2, 128, 256)}


@pytest.fixture(scope="module")
def exact54(primes):
    """ceil(bitlen(p^5) / 4) for every prime (Python big integers): the smallest integer
    number of 4/5-bit units whose 2^(4w/5) exceeds p, rounded up from bit lengths."""
    return np.array([-(-(p ** 5).bit_length() // 4) for p in primes.tolist()], dtype=np.int64)


def _lw():
    from paper_2506_01099_gb300 import benelux as B

    return B.bnx_log_weight


def test_log_weight_small_cases():
    lw = _lw()
    assert lw(3, 1) == 4           # 3^2 = 9 = 0b1001
    assert lw(3, 0) == 2           # 3 = 0b11
    assert lw(2, 1) == 3 and lw(2, 16) == 65537  # p = 2: F log2 2 = F, bit length F + 1
    assert lw(5, 3) == (5 ** 8).bit_length() == 19
    for p in (2**31 - 1, 4294967291):  # primes at the top of the domain (the latter is the largest below 2^32)
        assert lw(p, 7) == (p ** 128).bit_length() and lw(p, 10) == (p ** 1024).bit_length(), p
    assert lw(1, 4) == 0 and lw(0, 4) == 0 and lw(1 << 32, 4) == 0 and lw(3, 17) == 0  # outside the domain


@pytest.mark.parametrize("F", [2, 128, 256])
def test_log_weight_is_the_exact_bit_length(primes, exact, F):
    lw = _lw()
    f = F.bit_length() - 1
    got = np.array([lw(p, f) for p in primes.tolist()], dtype=np.int64)
    bad = np.nonzero(got != exact[F])[0]
    assert bad.size == 0, [(int(primes[i]), int(got[i]), int(exact[F][i])) for i in bad[:5]]


def test_log_weight54_small_cases():
    from paper_2506_01099_gb300 import benelux as B

    w = B.bnx_log_weight54
    assert w(3) == 2 and 4 * 2 > 5 * math.log2(3)   # 3^5 = 243: 8 bits
    assert w(17) == 6 and w(5) == 3 and w(7) == 4  # bit lengths 21, 12, 15
    q = (1 << 25) - 39                               # the largest prime below 2^25
    assert w(q) == -(-(q ** 5).bit_length() // 4)
    assert w(1) == 0 and w(0) == 0 and w(1 << 25) == 0  # outside the domain


def test_log_weight54_is_exact(primes, exact54):
    from paper_2506_01099_gb300 import benelux as B

    got = np.array([B.bnx_log_weight54(p) for p in primes.tolist()], dtype=np.int64)
    bad = np.nonzero(got != exact54)[0]
    assert bad.size == 0, [(int(primes[i]), int(got[i]), int(exact54[i])) for i in bad[:5]]
    # every weight over-estimates (5/4) log2 p: 2^(4 w) > p^5 in integers
    assert all((1 << (4 * int(w))) > p ** 5 for p, w in zip(primes.tolist(), exact54.tolist()))


def test_u8_pair_sums_stay_below_2p7(primes, exact54):
    """The u8 tile's flag test adds pair sum and threshold in one byte add; that is
    exact only if a pair sum L(n) + L(n+1) never reaches 2^7.  L(x) <= r log2 s_odd(x)
    with r the largest weight per bit of p, and s_odd(n) s_odd(n+1) <= n(n+1)/9 when
    both exceed 1 (else one factor is 1 and the bound is smaller still)."""
    odd = primes[primes > 2]
    r = (exact54[primes > 2] / np.log2(odd.astype(np.float64))).max()
    assert abs(r - 6 / math.log2(17)) < 1e-12  # p = 17 is the worst
    assert r * (84 - math.log2(9)) < 127
    # brute force on the extreme values below 2^42: odd prime powers and their neighbours
    w = dict(zip(primes.tolist(), exact54.tolist()))
    def L(x):
        tot, p = 0, 3
        while p * p <= x:
            if x % p == 0:
                e = 0
                while x % p == 0:
                    x //= p
                    e += 1
                tot += (e - 1) * w[p]
            p += 2
        return tot
    worst = 0
    for p in (3, 5, 7, 11, 13, 17, 19, 23):
        k = int(math.log(1 << 42, p))
        for n in (p ** k - 1, p ** k, 2 * p ** (k - 1) - 1, 2 * p ** (k - 1)):
            if 1 <= n < (1 << 42):
                worst = max(worst, L(n) + L(n + 1))
    assert 40 <= worst < 128


def test_log_weight_in_tile_scale():
    """F = 2^16 (the u32 tile's units) for every prime struck inside a tile."""
    lw = _lw()
    for p in primes_below(1 << 8).tolist():
        assert lw(p, 16) == (p ** 65536).bit_length(), p


@pytest.mark.gpu
@pytest.mark.parametrize("tile_kind", [3, 2, 0])
def test_device_weights_over_estimate_for_every_prime(primes, exact, tile_kind):
    """The device tables and kernels of a context up to 2^42 (all primes below 2^21)
    use, for every prime, the exact weights: in-tile, cached bucket and global bucket."""
    from paper_2506_01099_gb300 import benelux as B

    with B.Context(0, max_hi=1 << 42) as ctx:
        w = ctx.log_weights(tile_kind).astype(np.int64)
    assert np.array_equal(w[:, 0], primes)
    tile, cached, glob = w[:, 1], w[:, 2], w[:, 3]
    if tile_kind == 3:  # units of 4/5 bit: every weight is ceil(bitlen(p^5) / 4)
        e54 = np.array([-(-(int(p) ** 5).bit_length() // 4) for p in primes], dtype=np.int64)
        assert np.array_equal(tile, e54)
        assert np.array_equal(cached, e54) and np.array_equal(glob, e54)
    elif tile_kind == 2:  # units of 2^-8: in-tile bit length of p^256; buckets 2 x that of p^128
        assert np.array_equal(tile, exact[256])
        assert np.array_equal(cached, 2 * exact[128]) and np.array_equal(glob, 2 * exact[128])
        assert np.all(cached >= exact[256])  # 2 bitlen(p^128) > 256 log2 p
    else:  # units of 2^-16: in-tile bit length of p^65536 (p < 2^8); buckets 2^9 x that of p^128
        small = primes < (1 << 8)
        want = np.array([(int(p) ** 65536).bit_length() for p in primes[small]], dtype=np.int64)
        assert np.array_equal(tile[small], want)
        assert np.array_equal(cached, 512 * exact[128]) and np.array_equal(glob, 512 * exact[128])
