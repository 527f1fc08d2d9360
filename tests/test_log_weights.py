"""The log-domain filter's per-prime weights are exact integers.

The log tiles reject n when a sum of per-prime weights -- an upper bound of
F log2 of the odd square part of n(n+1), F units per bit -- cannot meet the
per-kind necessary condition.  That rejection loses no pair only if every
weight w(p) is at least F log2 p, i.e. 2^w(p) > p^F.  The library computes the
weights in integers (bnx_log_weight: repeated squaring with upward rounding);
these tests compare them with Python's exact big-integer bit lengths,
(p**F).bit_length() = floor(F log2 p) + 1, the smallest such integer:

* CPU: the host build of the weight function for every prime below 2^21 (all
  primes a context up to 2^42 holds) at F = 2, 128 and 256, and at F = 2^16 for
  the primes below 2^8 (the only ones struck inside a tile: q = p^2 <= 2^16);
* GPU: the weights the device kernels themselves use, per tile kind, read back
  along the kernels' code paths (bnx_log_weights).
"""
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
    if tile_kind == 3:  # half-bit units: every weight is the bit length of p^2
        assert np.array_equal(tile, exact[2])
        assert np.array_equal(cached, exact[2]) and np.array_equal(glob, exact[2])
    elif tile_kind == 2:  # units of 2^-8: in-tile bit length of p^256; buckets 2 x that of p^128
        assert np.array_equal(tile, exact[256])
        assert np.array_equal(cached, 2 * exact[128]) and np.array_equal(glob, 2 * exact[128])
        assert np.all(cached >= exact[256])  # 2 bitlen(p^128) > 256 log2 p
    else:  # units of 2^-16: in-tile bit length of p^65536 (p < 2^8); buckets 2^9 x that of p^128
        small = primes < (1 << 8)
        want = np.array([(int(p) ** 65536).bit_length() for p in primes[small]], dtype=np.int64)
        assert np.array_equal(tile[small], want)
        assert np.array_equal(cached, 512 * exact[128]) and np.array_equal(glob, 512 * exact[128])
