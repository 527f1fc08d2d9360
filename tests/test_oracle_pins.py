"""The oracle pinned to what the paper and the mathematics fix (CPU only).

Pins, each independent of the oracle's own code:
  * radicals of the integers printed in Tables 1 and 2, from their factorisations;
  * radicals from sympy's factoriser (a library routine) on random and adversarial x;
  * structural invariants of rad (squarefree, divides x, same prime support);
  * Algorithm 1's sieve agrees with the trial-division definition on segments
    whose edges sit on prime powers;
  * pair sets equal Theorem 1's closed forms (brute force, Algorithm 2, CRT);
  * Algorithm 2 and the CRT enumeration, two different methods, agree;
  * every Theorem 1 pair passes the per-kind necessary conditions.
A planted-mistake test builds the oracle with each ORC_MUTANT hook and checks
that these pins catch every one of them.
"""
import math
import random

import numpy as np
import pytest

from paper_pins import THEOREM1_BOUND, table_rows, theorem1_pairs


def _rad_from_fact(fd):
    return math.prod(fd.keys())


# ---------------------------------------------------------------------------
# pins as functions returning a list of failures (reused by the mutant test)
# ---------------------------------------------------------------------------

def pin_tables(o):
    bad = []
    for kind, m, n, facts in table_rows():
        for x, fd in facts.items():
            if math.prod(p**e for p, e in fd.items()) != x:
                bad.append(f"table factorisation of {x} does not multiply out")
            if o.rad_td(x) != _rad_from_fact(fd):
                bad.append(f"rad_td({x}) = {o.rad_td(x)} != {_rad_from_fact(fd)}")
    return bad


def pin_sieve_edges(o):
    bad = []
    cases = [(1, 9), (1, 5000), (9, 100), (2**32 - 3000, 6000), (2**40 - 2**12, 2**13),
             (1048573**2 - 100, 101), (1048573**2, 64), (3**25 - 7, 50), (65537**2 - 1, 3),
             (1_400_000_000_000 - 4096, 4096)]
    for start, length in cases:
        got = o.rad_sieve(start, length)
        want = o.rad_td_array(start, length)
        if not np.array_equal(got, want):
            i = int(np.nonzero(got != want)[0][0])
            bad.append(f"sieve({start},{length})[{i}] = {got[i]} != {want[i]}")
    return bad


def pin_brute(o):
    got = o.pairs_brute(1 << 12)
    want = theorem1_pairs(1, 1 << 12)
    return [] if got == want else [f"brute(2^12) {got} != {want}"]


def pin_sort(o):
    got = o.pairs_sort(1 << 20)
    want = theorem1_pairs(1, 1 << 20)
    return [] if got == want else [f"sort(2^20) {got} != {want}"]


def pin_crt(o):
    bad = []
    windows = [(1, 1 << 20), (2**40 - 2**21 - 2**19, 2**40 + 2**21 + 2**19),
               (17179607040 - 5000, 17180131328 + 5000)]
    for lo, hi in windows:
        for kinds in (1, 2, 3):
            got = o.pairs_crt(lo, hi, kinds)
            want = theorem1_pairs(lo, hi, kinds)
            if got != want:
                bad.append(f"crt[{lo},{hi}) kinds={kinds}: {got} != {want}")
    return bad


def pin_pairs_on_planted_radicals(o):
    """The definitions of Sec. 1 on a fabricated radical array (no real radicals give a
    three-term pair): distinct values everywhere, then collisions planted for a
    three-term pair (5, 20) -- which makes (6, 21) a first-kind pair too, since
    r[6] = r[21] and r[7] = r[22] -- a first-kind pair without the third term
    (10, 25), and a second-kind pair (30, 35)."""
    import numpy as np

    N = 40
    r = np.arange(1000, 1000 + N + 2, dtype=np.uint64)
    r[0] = 0
    r[20], r[21], r[22] = r[5], r[6], r[7]      # rad(m + i) = rad(n + i), i = 0, 1, 2
    r[25], r[26] = r[10], r[11]                 # first kind only: r[12] != r[27]
    r[36], r[35] = r[30], r[31]                 # second kind: r[30] = r[36], r[31] = r[35]
    first = [(5, 20, 1), (6, 21, 1), (10, 25, 1)]
    key = lambda p: (p[1], p[0], p[2])
    bad = []
    for kinds, exp in ((1, first), (2, [(30, 35, 2)]), (4, [(5, 20, 4)]),
                       (7, sorted(first + [(30, 35, 2), (5, 20, 4)], key=key))):
        got = o.pairs_brute_rad(r, N, kinds)
        if got != exp:
            bad.append(f"planted radicals, kinds {kinds}: {got} != {exp}")
    return bad


ALL_PINS = [pin_tables, pin_sieve_edges, pin_brute, pin_pairs_on_planted_radicals, pin_sort, pin_crt]


# ---------------------------------------------------------------------------
# the tests
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("pin", ALL_PINS, ids=lambda f: f.__name__)
def test_pin(orc, pin):
    assert pin(orc) == []


def test_theorem1_matches_tables():
    """The closed forms of Theorem 1 list exactly the rows of Tables 1 and 2."""
    rows = sorted(((m, n, kind) for kind, m, n, _ in table_rows()), key=lambda p: (p[1], p[0], p[2]))
    assert rows == theorem1_pairs()


def test_table_rows_are_pairs(orc):
    for kind, m, n, _ in table_rows():
        a, b, c, d = orc.rad_td(m), orc.rad_td(m + 1), orc.rad_td(n), orc.rad_td(n + 1)
        if kind == 1:
            assert (a, b) == (c, d)
        else:
            assert (a, b) == (d, c)


def test_rad_td_vs_sympy(orc):
    sympy = pytest.importorskip("sympy")
    rng = random.Random(2506_01099)
    xs = [1, 2, 3, 4, 8, 9, 2**40, 2**41 + 1, 3**26, 1048573**2, 1048573 * 1048571, 999983**2 * 4]
    xs += [2**k + d for k in range(2, 42) for d in (-1, 1)]
    xs += [rng.randrange(1, 2**42) for _ in range(300)]
    xs += [rng.randrange(1, 2**20) ** 2 for _ in range(50)]
    for x in xs:
        assert orc.rad_td(x) == math.prod(sympy.primefactors(x)), x


def test_rad_invariants(orc):
    rng = random.Random(7)
    for _ in range(2000):
        x = rng.randrange(1, 2**42)
        r = orc.rad_td(x)
        assert x % r == 0
        # same prime support: x divides rad(x)^e for e = log2(x)
        assert pow(r, 42, x) == 0 or x == 1
        # squarefree: no prime square below 2^11 divides it, and rad is idempotent
        assert all(r % (p * p) for p in (2, 3, 5, 7, 11, 13, 1009, 2039))
        assert orc.rad_td(r) == r
        assert orc.sq_td(x) * r == x
    assert orc.rad_td(1) == 1


def test_sort_equals_crt(orc):
    """Algorithm 2 (sorting all 2-sets) and the CRT enumeration agree on [1, 2^22)."""
    assert orc.pairs_sort(1 << 22) == orc.pairs_crt(1, 1 << 22)


def test_hash_map_search(orc):
    """The hash-table key search finds Theorem 1's pairs below 2^20 and agrees with the
    sort-based search and the CRT enumeration on [1, 2^22), per kind."""
    assert orc.pairs_map(1 << 20) == theorem1_pairs(1, 1 << 20)
    for kinds in (1, 2, 3):
        got = orc.pairs_map(1 << 22, kinds)
        assert got == orc.pairs_sort(1 << 22, kinds) == orc.pairs_crt(1, 1 << 22, kinds)
    # a group of three equal keys ({2, 3} is the key of 2, 3 and 8): every pair, not only neighbours
    assert orc.pairs_map(9) == [(2, 3, 2), (2, 8, 1), (3, 8, 2)]


def test_crt_window_at_2p40(orc):
    """[2^40, 2^40 + 2^30) holds exactly one pair, of the second kind."""
    lo = 2**40
    got = orc.pairs_crt(lo, lo + (1 << 30))
    assert got == [(1048577, 1099513724928, 2)]
    assert got == theorem1_pairs(lo, lo + (1 << 30))


def test_crt_empty_window_below_bound(orc):
    assert orc.pairs_crt(THEOREM1_BOUND - (1 << 26), THEOREM1_BOUND) == []


def test_necessary_conditions_hold_for_every_pair(orc):
    """Each Theorem 1 pair passes its kind's filter; counts are monotone in the window."""
    for m, n, kind in theorem1_pairs(1, 1 << 40):
        c1, c2 = orc.filter_counts(n, n + 1, kind)
        assert (c1 if kind == 1 else c2) == 1, (m, n, kind)
    a1, a2 = orc.filter_counts(1, 1 << 20)
    b1, b2 = orc.filter_counts(1, 1 << 21)
    assert b1 >= a1 and b2 >= a2 and a2 >= 0


def test_hash_keys_cover_pair_members(orc):
    """Every member of a pair with n < S has rad(x)rad(x+1) <= 2S (the hash insert rule)."""
    S = 1 << 16
    assert orc.hash_keys(S) >= len({x for m, n, _ in theorem1_pairs(1, S) for x in (m, n)})
    for m, n, _ in theorem1_pairs(1, S):
        for x in (m, n):
            assert orc.rad_td(x) * orc.rad_td(x + 1) <= 2 * S


def test_nprimes(orc):
    """pi(x) at a few textbook values."""
    assert orc.nprimes_upto(100) == 25
    assert orc.nprimes_upto(2**12) == 564
    assert orc.nprimes_upto(2**16) == 6542
    assert orc.nprimes_upto(10**6) == 78498


MUTANTS = {1: "rad_td drops the last prime cofactor", 2: "Alg. 1 misses the multiple at start",
           3: "Alg. 1 starts at exponent 1", 4: "Alg. 2 kind rule inverted",
           5: "CRT second kind m = j*ab - n", 6: "first-kind inequality used for the second kind",
           7: "Alg. 1 sieves primes p < sqrt(S) only", 8: "brute force transposes an operand",
           9: "three-term rule compares m + 2 with n + 1"}


@pytest.mark.parametrize("k", sorted(MUTANTS), ids=lambda k: f"mutant{k}")
def test_planted_mistake_is_caught(k, tmp_path):
    import oracle

    mut = oracle.Oracle(oracle.build(mutant=k, out_dir=str(tmp_path)))
    failures = []
    for pin in ALL_PINS:  # cheapest first; stop at the first pin that fails
        try:
            failures += pin(mut)
        except Exception as e:  # a mutant may also crash a pin
            failures.append(repr(e))
        if failures:
            break
    assert failures, f"no pin caught mutant {k}: {MUTANTS[k]}"


def test_three_term_question(orc):
    """Erdos's original question (Sec. 1): rad(m+i) = rad(n+i) for i = 0, 1, 2.
    Sec. 1 shows why the families fail it (m+2 = 2^(k+1) while n+2 = 2 mod 4)
    and that (75, 1215) fails it (77 = 7*11, 1217 prime); no solution is known."""
    for m, n, kind in theorem1_pairs(1, 1 << 40, 1):
        assert orc.rad_td(m + 2) != orc.rad_td(n + 2), (m, n)
    assert orc.rad_td(77) == 77 and orc.rad_td(1217) == 1217
    assert orc.pairs_brute(1 << 12, 4) == []
    assert orc.pairs_crt(1, 1 << 22, 4) == []
    # bit 4 adds nothing to bit 1, and the brute force agrees with the CRT path
    assert orc.pairs_crt(1, 1 << 22, 5) == theorem1_pairs(1, 1 << 22, 1)
    assert orc.pairs_brute(1 << 12, 7) == theorem1_pairs(1, 1 << 12, 3)


def _rad_sympy(x: int) -> int:
    from sympy import primefactors

    r = 1
    for p in primefactors(x):
        r *= p
    return r


def _conditions_brute(lo: int, hi: int):
    """The per-kind necessary conditions counted from their definitions, with radicals
    from sympy: first kind rad(n) rad(n+1) <= n - 1; second kind some multiple of
    rad(n) rad(n+1) in [n + 2, 2n]."""
    c1 = c2 = 0
    rads = {x: _rad_sympy(x) for x in range(lo, hi + 1)}
    for n in range(lo, hi):
        ab = rads[n] * rads[n + 1]
        if ab <= n - 1:
            c1 += 1
        if ab <= 2 * n and -(-(n + 2) // ab) <= (2 * n) // ab:
            c2 += 1
    return c1, c2


def test_filter_counts_brute_force(orc):
    """orc_filter_counts equals the conditions evaluated one by one (brute force, sympy
    radicals) on [1, 2^14) and on a window at 2^40."""
    pytest.importorskip("sympy")
    assert orc.filter_counts(1, 1 << 14) == _conditions_brute(1, 1 << 14)
    lo = (1 << 40) - 300
    assert orc.filter_counts(lo, lo + 1024) == _conditions_brute(lo, lo + 1024)


def test_hash_keys_brute_force(orc):
    """orc_hash_keys(S) is the number of x in [1, S) with rad(x) rad(x+1) <= 2S (brute force)."""
    pytest.importorskip("sympy")
    for S in (2, 3, 100, 1 << 13):
        want = sum(1 for x in range(1, S) if _rad_sympy(x) * _rad_sympy(x + 1) <= 2 * S)
        assert orc.hash_keys(S) == want, S
