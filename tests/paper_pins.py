"""What the paper fixes, restated independently of the oracle.

* Theorem 1 (Sec. 3.2): for m < n < 1.4e12 the first-kind pairs are exactly
  (75, 1215) and m = 2^k - 2, n = 2^(2k) - 2^(k+1) for 2 <= k <= 20; the
  second-kind pairs are exactly (35, 4374) and m = 2^k + 1, n = 2^(2k) + 2^(k+1)
  for 0 <= k <= 20.
* Tables 1 and 2 (Sec. 3.2): every pair with the factorisations of m, n, m+1,
  n+1 (stored in golden/paper_tables.txt with their typesetting slips fixed).
"""
from __future__ import annotations

import os

THEOREM1_BOUND = 1_400_000_000_000
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def theorem1_pairs(lo: int = 1, hi: int = THEOREM1_BOUND, kinds: int = 3):
    """(m, n, kind) of Theorem 1 with lo <= n < hi, sorted by (n, m, kind)."""
    assert hi <= THEOREM1_BOUND, "Theorem 1 says nothing above 1.4e12"
    out = []
    if kinds & 1:
        out.append((75, 1215, 1))
        for k in range(2, 21):
            out.append((2**k - 2, 2 ** (2 * k) - 2 ** (k + 1), 1))
    if kinds & 2:
        out.append((35, 4374, 2))
        for k in range(0, 21):
            out.append((2**k + 1, 2 ** (2 * k) + 2 ** (k + 1), 2))
    out = [p for p in out if lo <= p[1] < hi]
    return sorted(out, key=lambda p: (p[1], p[0], p[2]))


def parse_factorisation(f: str):
    """'2^3*3' -> {2: 3, 3: 1}"""
    d = {}
    for t in f.strip().split("*"):
        if "^" in t:
            b, e = t.split("^")
            d[int(b)] = d.get(int(b), 0) + int(e)
        else:
            d[int(t)] = d.get(int(t), 0) + 1
    return d


def table_rows():
    """Rows of Tables 1 and 2: (kind, m, n, {x: factorisation dict} for x in m, n, m+1, n+1)."""
    rows = []
    with open(os.path.join(GOLDEN, "paper_tables.txt")) as fh:
        for line in fh:
            if not line.strip() or line.startswith("#"):
                continue
            parts = [p.strip() for p in line.split("|")]
            kind, m, n = (int(v) for v in parts[0].split())
            facts = {m: parse_factorisation(parts[1]), n: parse_factorisation(parts[2]),
                     m + 1: parse_factorisation(parts[3]), n + 1: parse_factorisation(parts[4])}
            rows.append((kind, m, n, facts))
    return rows
