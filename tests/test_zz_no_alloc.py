"""bnx_rad_segment_noalloc: the radicals entry point for callers that cannot
allocate device memory (no context, fixed static scratch inside the library).

The GPU test calls it through the C ABI twice in a row and checks each result
against bnx_rad_segment, the entry point that allocates its workspace (the
results are integers, so they must be identical), and against the oracle's
trial-division radicals on windows at both ends of each range.  It makes its own buffers and
context, so it passes alone in a fresh process as well as after other tests.
"""
import ctypes

import numpy as np
import pytest


def _lib():
    from paper_2506_01099_gb300 import benelux as B

    return B, B.lib()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    B, L = _lib()
    dummy = ctypes.c_void_p(16)  # never dereferenced: the limits are checked first
    assert L.bnx_rad_segment_noalloc(0, 10, dummy, None, None) == B.BNX_E_ARG
    assert L.bnx_rad_segment_noalloc(1, 0, dummy, None, None) == B.BNX_E_ARG
    assert L.bnx_rad_segment_noalloc(1, B.BNX_NOALLOC_MAX_LEN + 1, dummy, None, None) == B.BNX_E_ARG
    assert L.bnx_rad_segment_noalloc(B.BNX_NOALLOC_MAX_HI - 10, 11, dummy, None, None) == B.BNX_E_ARG
    assert L.bnx_rad_segment_noalloc(1, 10, None, None, None) == B.BNX_E_ARG
    # ranges whose end lo + len would wrap past 2^64 (the check must not overflow)
    assert L.bnx_rad_segment_noalloc(2**64 - 1, 2, dummy, None, None) == B.BNX_E_ARG
    assert L.bnx_rad_segment_noalloc(2**64 - 2**17, 2**17, dummy, None, None) == B.BNX_E_ARG
    assert L.bnx_rad_segment_noalloc(B.BNX_NOALLOC_MAX_HI - 10, 10, None, None, None) == B.BNX_E_ARG  # NULL first


@pytest.mark.gpu
def test_noalloc_matches_rad_segment_twice_in_a_row(orc):
    import torch

    B, L = _lib()
    stream = torch.cuda.current_stream().cuda_stream
    cases = [(B.BNX_NOALLOC_MAX_HI - B.BNX_NOALLOC_MAX_LEN, B.BNX_NOALLOC_MAX_LEN),  # the largest allowed
             (1, 70_001)]                                                           # from 1, ragged length
    with B.Context(0, max_hi=B.BNX_NOALLOC_MAX_HI + 1) as ctx:
        for lo, n in cases:
            rad = torch.empty(n, dtype=torch.int64, device="cuda")
            sq = torch.empty(n, dtype=torch.int64, device="cuda")
            rc = L.bnx_rad_segment_noalloc(lo, n, rad.data_ptr(), sq.data_ptr(), stream)
            assert rc == B.BNX_OK, B.bnx_last_error()
            want_rad = torch.empty(n, dtype=torch.int64, device="cuda")
            want_sq = torch.empty(n, dtype=torch.int64, device="cuda")
            ctx.rad_segment(lo, n, want_rad.data_ptr(), want_sq.data_ptr(), stream)
            torch.cuda.synchronize()
            assert torch.equal(rad, want_rad), (lo, n)
            assert torch.equal(sq, want_sq), (lo, n)
            xs = np.arange(lo, lo + n, dtype=np.uint64)
            r = rad.cpu().numpy().view(np.uint64)
            assert np.array_equal(r * sq.cpu().numpy().view(np.uint64), xs)
            # and against the oracle's trial-division radicals: both ends of each range
            # (the last window ends at the largest value allowed) and sampled windows
            rng = np.random.default_rng(lo % 1000)
            for off in [0, n - 512] + [int(v) for v in rng.integers(0, n - 512, 4)]:
                assert np.array_equal(r[off:off + 512], orc.rad_td_array(lo + off, 512)), (lo, off)
