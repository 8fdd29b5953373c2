"""The exact-depth argument of the per-thread walk, checked on the CPU.

For a covered sample the walk estimates q = floor((w1 d1 + w2 d2) / A) in
float32 from k_i = fl(rA d_i), rA = 1/A to within 2 ulp (the fast reciprocal
the kernel uses), one product and one fused multiply-add, and then corrects
q against the exact remainder.  The kernel relies on two bounds:
- fast form (A < 2^27, |d1| + |d2| < 2^22): the estimate is within 3 of q,
  so the remainder lies in (-3A, 4A) and fits a wrapping 32-bit int;
- 64-bit form (A < 2^30, |d_i| < 2^24): the estimate is within 16 of q,
  well inside the fix-up loops' bound of 64 steps.
Both are checked here against exact integer arithmetic on adversarial and
random inputs, emulating each float32 rounding with numpy.
"""
import numpy as np

FIX_LIMIT = 64


def _ulp_shift(x: np.ndarray, k: int) -> np.ndarray:
    """x moved by k float32 ulps (x > 0)."""
    return (x.view(np.int32) + np.int32(k)).view(np.float32)


def _estimate(w1, w2, d1, d2, A, ulps):
    rA = _ulp_shift((np.float32(1.0) / A.astype(np.float32)).astype(np.float32), ulps)
    k1 = (rA * d1.astype(np.float32)).astype(np.float32)
    k2 = (rA * d2.astype(np.float32)).astype(np.float32)
    w1f = w1.astype(np.float32)
    w2f = w2.astype(np.float32)
    p2 = (w2f * k2).astype(np.float32)
    # fused multiply-add: the float32 product is exact in float64
    s = (w1f.astype(np.float64) * k1.astype(np.float64) + p2.astype(np.float64)).astype(np.float32)
    return np.floor(s.astype(np.float64)).astype(np.int64)


def _cases(rng, n, a_max_log2, d_sum_max, d_max):
    A = np.exp2(rng.uniform(0, a_max_log2, n)).astype(np.int64)
    A = np.clip(A, 1, (1 << a_max_log2) - 1)
    # depth differences: half at the extremes of the allowed range
    dmag = np.where(rng.random(n) < 0.5, d_sum_max - 1, rng.integers(0, d_sum_max, n))
    split = rng.random(n)
    d1 = np.minimum((dmag * split).astype(np.int64), d_max - 1)
    d2 = np.minimum(dmag - d1, d_max - 1)
    d1 *= rng.choice([-1, 1], n)
    d2 *= rng.choice([-1, 1], n)
    # barycentric numerators with w1 + w2 <= A, corners included
    u = rng.random(n)
    v = rng.random(n) * (1 - u)
    w1 = np.floor(u * A).astype(np.int64)
    w2 = np.floor(v * A).astype(np.int64)
    corner = rng.integers(0, 4, n)
    w1 = np.where(corner == 0, A, np.where(corner == 1, 0, w1))
    w2 = np.where(corner == 0, 0, np.where(corner == 1, A, w2))
    return w1, w2, d1, d2, A


def _check(w1, w2, d1, d2, A, bound):
    n = w1 * d1 + w2 * d2
    q = np.floor_divide(n, A)
    worst = 0
    for ulps in (-2, -1, 0, 1, 2):
        est = _estimate(w1, w2, d1, d2, A, ulps)
        worst = max(worst, int(np.abs(est - q).max()))
    assert worst <= bound, f"estimate off by {worst} > {bound}"
    return worst


def test_fast_form_estimate_within_3_and_remainder_fits_int32():
    rng = np.random.default_rng(20260317)
    w1, w2, d1, d2, A = _cases(rng, 400_000, 27, 1 << 22, 1 << 22)
    assert (np.abs(d1) + np.abs(d2) < (1 << 22)).all() and (A < (1 << 27)).all()
    _check(w1, w2, d1, d2, A, 3)
    # with the estimate within 3, |r| < 4A < 2^29: a wrapping int32 holds it
    n = w1 * d1 + w2 * d2
    for off in (-3, 3):
        q = np.floor_divide(n, A) + off
        r = n - q * A
        assert (np.abs(r) < (1 << 29)).all()
        wrapped = ((w1 * d1 + w2 * d2 - q * A) & 0xFFFFFFFF).astype(np.uint32).view(np.int32)
        assert np.array_equal(wrapped.astype(np.int64), r)


def test_64bit_form_estimate_within_fix_up_limit():
    rng = np.random.default_rng(20260318)
    w1, w2, d1, d2, A = _cases(rng, 400_000, 30, 1 << 25, 1 << 24)
    worst = _check(w1, w2, d1, d2, A, 16)
    assert worst < FIX_LIMIT


def test_extreme_corners():
    # the largest allowed magnitudes, every sign combination, w at the corners
    vals = []
    for A in (1, 2, 3, (1 << 27) - 1, (1 << 26) + 12345):
        for d1 in ((1 << 22) - 1, -((1 << 22) - 1), (1 << 21), 0, 1, -1):
            d2 = ((1 << 22) - 1 - abs(d1)) * (1 if d1 >= 0 else -1)
            for w1, w2 in ((A, 0), (0, A), (A // 2, A - A // 2), (0, 0), (1 % (A + 1), 0)):
                vals.append((w1, w2, d1, d2, A))
    w1, w2, d1, d2, A = (np.array(c, dtype=np.int64) for c in zip(*vals))
    assert (np.abs(d1) + np.abs(d2) < (1 << 22)).all()
    _check(w1, w2, d1, d2, A, 3)


# ---------------------------------------------------------------------------
# Compacted small boxes: a thread walks a box of at most 32 pixels for
# coverage only, shifting each sample's bit in from the top (mask = mask >> 1
# | covered << 31), then shifts the mask down by 32 - n; bit j is then the
# box's j-th pixel in row-major order.  The warp's fragment pass recovers the
# row of bit j as (j * M) >> 16 with M = floor(fl(65536 / bw)) + 1, the
# quotient taken with a fast division good to 2 ulp.


def test_small_box_mask_bit_order():
    rng = np.random.default_rng(20261204)
    for n in range(1, 33):
        for _ in range(50):
            cov = rng.random(n) < 0.5
            mask = 0
            for c in cov:
                mask = (mask >> 1) | (0x80000000 if c else 0)
            mask >>= 32 - n
            assert [(mask >> j) & 1 for j in range(n)] == [int(c) for c in cov]


def test_small_box_row_from_bit():
    for bw in range(1, 33):
        q = np.float32(65536.0) / np.float32(bw)
        for ulps in (-2, -1, 0, 1, 2):
            M = int(np.floor(np.float64(_ulp_shift(np.array([q], dtype=np.float32), ulps)[0]))) + 1
            assert 65536 / bw <= M < 65536 / bw + 2
            for j in range(32):
                assert (j * M) >> 16 == j // bw, (bw, j, M)
