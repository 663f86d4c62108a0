"""The integer reformulations the batched scan relies on, checked exhaustively
or on dense samples against plain integer arithmetic (host only):
  - a float32-reciprocal quotient, truncated and corrected once, is exact for
    numerators below 2^24 (the case-B draw units i = m Qn + q);
  - the number of pairs of projectile s in a cell with N_p < N_t,
    ceil((N_t - s) / N_p), equals q0 + [s < r0] with N_t = q0 N_p + r0;
  - a 16-bit high digit w >> 16 is at most k exactly when the whole word is at
    most 2^16 k + 0xFFFF (the quick reject tests the high digit this way)."""
import numpy as np


def f32_quotient(i, n):
    """floor(float32(i) * float32(1/n)) truncated toward zero, then corrected
    by at most one step, as the scan's division does."""
    inv = np.float32(1.0) / np.float32(n)
    q = np.floor((np.float32(i) * inv).astype(np.float64)).astype(np.int64)
    r = i - q * n
    q = np.where(r < 0, q - 1, q)
    r = np.where(r < 0, r + n, r)
    q = np.where(r >= n, q + 1, q)
    r = np.where(r >= n, r - n, r)
    return q, r


def test_float_reciprocal_division_is_exact_below_2_24():
    rng = np.random.default_rng(3)
    ns = np.unique(np.concatenate([np.arange(1, 4097), rng.integers(1, 1 << 16, 4000), [65535, 65536]]))
    for n in ns:
        i = np.concatenate([rng.integers(0, 1 << 24, 2000), np.arange(0, 3 * n + 3),
                            (1 << 24) - 1 - np.arange(0, 64), n * np.arange(1, 64), n * np.arange(1, 64) - 1])
        i = i[(i >= 0) & (i < (1 << 24))].astype(np.int64)
        q, r = f32_quotient(i, int(n))
        assert np.array_equal(q, i // n) and np.array_equal(r, i % n), n


def test_case_b_pair_counts():
    for Np in range(1, 120):
        for Nt in range(Np + 1, 700, 7):
            s = np.arange(Np)
            q0, r0 = divmod(Nt, Np)
            assert np.array_equal(-((s - Nt) // Np), q0 + (s < r0)), (Np, Nt)
            assert (q0 + (s < r0)).sum() == Nt        # every target in exactly one pair


def test_high_digit_on_the_whole_word():
    rng = np.random.default_rng(5)
    w = np.concatenate([rng.integers(0, 1 << 32, 200000, dtype=np.uint64),
                        np.array([0, 0xFFFF, 0x10000, 0xFFFFFFFF], dtype=np.uint64)])
    for k in (0, 1, 557, 0x7FFF, 0xFFFE, 0xFFFF):
        assert np.array_equal((w >> 16) <= k, w <= ((k << 16) | 0xFFFF))
