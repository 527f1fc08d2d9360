"""Seeded synthetic workloads (integer ranges) shared by the tests, the
benchmark and the CPU baseline.

This module holds random-number generation and interval bookkeeping only:
none of the search's arithmetic.  The generator is splitmix64 (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014), seeded
with ``config_index ^ 0x250601099``.

Workloads (all n-ranges are half-open [lo, hi) and a search reports pairs
(m, n) with n in the range and any m < n):

* full ranges ``[1, 2^24)`` and ``[1, 2^32)``;
* ``batch_intervals``: 4096 intervals, length floor(2^(16 + 14u)) (log-uniform in
  [2^16, 2^30]), start uniform in [2^32, 2^40), kind 1 or 2 with probability 1/2;
* ``serving_requests``: a Poisson stream of requests, length log-uniform in
  [2^20, 2^34], start uniform in [1, 1.4e12], kinds in {1, 2, 3};
* ``large_windows``: [2^40, 2^40 + 2^37) and [1.3e12, 1.4e12), each also split
  into 2^30-integer intervals for the batched path.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

MASK64 = (1 << 64) - 1
SEED_SALT = 0x250601099


class SplitMix64:
    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def below(self, bound: int) -> int:
        """Integer in [0, bound) (bound <= 2^64), by 128-bit multiply-shift."""
        return (self.next_u64() * bound) >> 64


@dataclass(frozen=True)
class Interval:
    lo: int
    hi: int
    kinds: int
    id: int = 0

    @property
    def length(self) -> int:
        return self.hi - self.lo


def full_range(hi: int, kinds: int = 3):
    return [Interval(1, hi, kinds, 0)]


def batch_intervals(count: int = 4096, seed: int = 3 ^ SEED_SALT):
    """The batched workload: uneven intervals with starts in [2^32, 2^40)."""
    rng = SplitMix64(seed)
    out = []
    for i in range(count):
        u = rng.uniform()
        length = int(math.floor(2.0 ** (16 + 14 * u)))
        lo = (1 << 32) + rng.below((1 << 40) - (1 << 32))
        kind = 1 + (rng.next_u64() >> 63)
        out.append(Interval(lo, lo + length, kind, i))
    return out


@dataclass(frozen=True)
class Request:
    arrival_s: float
    interval: Interval


def serving_requests(count: int = 1024, rate_per_s: float = 1.0, seed: int = 4 ^ SEED_SALT,
                     len_log2=(20, 34), lo_max: int = 1_400_000_000_000):
    """A Poisson stream: exponential gaps with the given rate; lengths
    log-uniform in [2^len_log2[0], 2^len_log2[1]]; kinds drawn from {1, 2, 3}."""
    rng = SplitMix64(seed)
    t = 0.0
    out = []
    a, b = len_log2
    for i in range(count):
        t += -math.log(1.0 - rng.uniform()) / rate_per_s
        length = int(math.floor(2.0 ** (a + (b - a) * rng.uniform())))
        lo = 1 + rng.below(lo_max)
        kinds = 1 + rng.below(3)
        out.append(Request(t, Interval(lo, lo + length, kinds, i)))
    return out


def mean_serving_length(len_log2=(20, 34)) -> float:
    """E[floor(2^(a + (b-a)u))] ~ (2^b - 2^a) / ((b-a) ln 2)."""
    a, b = len_log2
    return (2.0**b - 2.0**a) / ((b - a) * math.log(2.0))


LARGE_WINDOWS = ((1 << 40, (1 << 40) + (1 << 37)), (1_300_000_000_000, 1_400_000_000_000))


def split(lo: int, hi: int, piece: int, kinds: int = 3, first_id: int = 0):
    """[lo, hi) cut into consecutive intervals of at most `piece` integers."""
    out = []
    i = first_id
    x = lo
    while x < hi:
        y = min(hi, x + piece)
        out.append(Interval(x, y, kinds, i))
        i += 1
        x = y
    return out


def large_window_intervals(which: int = 0, piece: int = 1 << 30, kinds: int = 3):
    lo, hi = LARGE_WINDOWS[which]
    return split(lo, hi, piece, kinds)


def total_integers(intervals) -> int:
    return sum(iv.hi - iv.lo for iv in intervals)
