"""The tuning JSON reader (bnx_tune_parse, the reader bnx_create applies): fields,
defaults, and every malformed or out-of-range input rejected with BNX_E_ARG (CPU only)."""
import ctypes
import json
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DEFAULTS = {"tile_log2": 15, "seg_tiles": 16, "threads": 256, "ctas_per_sm": 0, "small_q_log2": 16, "tile_kind": 3}


@pytest.fixture(scope="module")
def B():
    from paper_2506_01099_gb300 import benelux

    return benelux


def parse(B, text):
    return B.bnx_tune_parse(text).as_dict()


def test_defaults_and_fields(B):
    assert parse(B, "{}") == DEFAULTS
    assert parse(B, " \n{ }\t") == DEFAULTS
    got = parse(B, '{"tile_log2": 13, "seg_tiles": 4,\n "threads": 512, "ctas_per_sm": 2, "small_q_log2": 12, '
                   '"tile_kind": 1}')
    assert got == {"tile_log2": 13, "seg_tiles": 4, "threads": 512, "ctas_per_sm": 2, "small_q_log2": 12,
                   "tile_kind": 1}
    assert parse(B, '{"threads":128}') == dict(DEFAULTS, threads=128)


def test_autotune_output_round_trips(B):
    """bnx_autotune writes the six fields and "ms" (a timing, ignored on input)."""
    text = ('{"tile_log2": 14, "seg_tiles": 8, "threads": 256, "ctas_per_sm": 0, "small_q_log2": 15, '
            '"tile_kind": 2, "ms": 91.0437}')
    assert parse(B, text) == {"tile_log2": 14, "seg_tiles": 8, "threads": 256, "ctas_per_sm": 0,
                              "small_q_log2": 15, "tile_kind": 2}
    assert parse(B, '{"ms": 1e-3}') == DEFAULTS and parse(B, '{"ms": 7}') == DEFAULTS


def test_committed_tune_cache_parses(B):
    cache = json.load(open(os.path.join(ROOT, "paper_2506_01099_gb300", "tune_cache.json")))
    assert cache
    for key, t in cache.items():
        assert parse(B, json.dumps(t)) == dict(DEFAULTS, **t), key


BAD = [
    '{"tile_size": 15}',                        # unknown key
    '{"tile_log2": 15, "tile_log2": 14}',       # repeated key
    '{"threads": -256}',                        # negative
    '{"threads": 256.0}',                       # not an integer
    '{"threads": 2.56e2}',
    '{"threads": "256"}',                       # a string
    '{"seg_tiles": 4294967296}',                # beyond 32 bits
    '{"tile_log2": 9}', '{"tile_log2": 17}',    # out of range
    '{"seg_tiles": 3}', '{"seg_tiles": 128}', '{"seg_tiles": 0}',
    '{"threads": 100}', '{"threads": 2048}',
    '{"small_q_log2": 7}', '{"small_q_log2": 17}',
    '{"tile_kind": 4}', '{"ctas_per_sm": 33}',
    '', '   ', '[]', '{', '}', '{"threads" 256}', '{"threads": }', '{threads: 256}', '{"threads: 256}',
    '{"threads": 256,}', '{"threads": 256} x', '{"threads": 256}}', '{"threads": 256 "seg_tiles": 4}',
    '{"a": {"b": 1}}',
]


@pytest.mark.parametrize("text", BAD)
def test_bad_json_is_an_argument_error(B, text):
    L = B.lib()
    t = B.bnx_tune(1, 2, 3, 4, 5, 6)
    assert L.bnx_tune_parse(text.encode(), ctypes.byref(t)) == B.BNX_E_ARG
    assert t.as_dict() == {"tile_log2": 1, "seg_tiles": 2, "threads": 3, "ctas_per_sm": 4, "small_q_log2": 5,
                           "tile_kind": 6}  # left as it was
    assert "tune" in B.bnx_last_error() or "must" in B.bnx_last_error()


def test_null_arguments(B):
    L = B.lib()
    t = B.bnx_tune()
    assert L.bnx_tune_parse(None, ctypes.byref(t)) == B.BNX_E_ARG
    assert L.bnx_tune_parse(b"{}", None) == B.BNX_E_ARG
