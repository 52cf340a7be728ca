"""The frame-wise pass's index arithmetic, checked on the CPU (no GPU needed): the division-free
floor division by the magnification (a multiplier and a high-word product, as gen_fdiv in
csrc/misr_general.cuh computes it) over the whole argument range the kernels pass it, and the
adjoint's gather ranges, which must visit exactly the (LR row, tap) pairs of the forward."""
import numpy as np
import pytest

OFF = 1 << 21


def fdiv(a, f):
    """floor(a / f) as the kernels compute it: umulhi(a + f 2^21, ceil(2^32 / f)) - 2^21"""
    if f == 1:
        return a
    m = ((1 << 32) + f - 1) // f
    n = (a + f * OFF).astype(np.uint64)
    return ((n * np.uint64(m)) >> np.uint64(32)).astype(np.int64) - OFF


@pytest.mark.parametrize("f", range(1, 9))
def test_division_free_floor_division(f):
    a = np.arange(-(1 << 21), (1 << 22) + 1, dtype=np.int64)
    assert np.array_equal(fdiv(a, f), np.floor_divide(a, f))


@pytest.mark.parametrize("f", [1, 2, 3, 8])
def test_adjoint_gather_ranges_are_the_forward_transposed(f):
    """For every HR row u the LR rows i in [ceil((a - tw + 1) / f), floor(a / f)] (a = u - t + R,
    clamped to the frame) are exactly those whose forward taps f i + t - R + dy, dy < tw, reach u."""
    for h in (1, 3, 7):
        H = f * h
        for R in (0, 1, 2):
            for tw in {1 + 2 * R, f + 2 * R, f + 2 * R + 1}:
                for t in range(-2 * H - 3, 2 * H + 4):
                    fwd = {(f * i + t - R + dy, i) for i in range(h) for dy in range(tw)
                           if 0 <= f * i + t - R + dy < H}
                    adj = set()
                    for u in range(H):
                        a = u - t + R
                        lo = max(int(fdiv(np.array([a - tw + f]), f)[0]), 0)
                        hi = min(int(fdiv(np.array([a]), f)[0]), h - 1)
                        for i in range(lo, hi + 1):
                            assert 0 <= a - f * i < tw
                            adj.add((u, i))
                    assert fwd == adj, (f, h, R, tw, t)
