"""The digit-slice arithmetic that TEVO_OZAKI documents (include/tevo.h), worked
in exact integers on the CPU, against its stated properties:

* a row scaled by 2^-e (max |entry| < 2^e) and rounded to a fixed-point integer
  X of F = P + W (G - 1) fraction bits splits into G balanced base-2^W digits
  with |digit| <= 2^P, and the digits give X back exactly;
* a group of slice pairs (s + t = g) over a pass of at most 2048 / (g + 1)
  K-indices sums to an integer below 2^24 (exact in an fp32 accumulator);
* the product of the pairs s + t < G differs from the exact complex product
  by at most (G + 2) 2^(-W G) 2^(e_m + e_n) K per entry.

This checks the scheme, not the kernel: the GPU tests compare the kernel's
results with numpy.
"""
from fractions import Fraction

import numpy as np
import pytest

P, W = 6, 7


def row_exponent(row):
    """e with max(|Re|, |Im|) < 2^e over the row (0 for a zero row)."""
    mx = max(max(abs(z.real), abs(z.imag)) for z in row)
    if mx == 0.0:
        return 0
    return int(np.frexp(mx)[1])          # mx = m 2^E with 0.5 <= m < 1, so mx < 2^E


def to_fixed(x, e, F):
    """x 2^(F - e) rounded to the nearest integer, ties to even (exact)."""
    q = Fraction(x) * Fraction(2) ** (F - e)
    n = q.numerator // q.denominator
    r = q - n
    if r > Fraction(1, 2) or (r == Fraction(1, 2) and n % 2 == 1):
        n += 1
    return n


def digits(X, G):
    """Balanced base-2^W digits d_0..d_{G-1} of X: X = sum_s d_s 2^(W (G-1-s))."""
    out = []
    rem = X
    for s in range(G - 1, 0, -1):        # lowest digit first, each in [-2^(W-1), 2^(W-1))
        d = ((rem + (1 << (W - 1))) % (1 << W)) - (1 << (W - 1))
        out.append(d)
        rem = (rem - d) >> W
    out.append(rem)                      # the top digit takes what is left
    return out[::-1]


def slice_rows(M, G):
    F = P + W * (G - 1)
    exps = [row_exponent(r) for r in M]
    re = [[digits(to_fixed(z.real, e, F), G) for z in r] for r, e in zip(M, exps)]
    im = [[digits(to_fixed(z.imag, e, F), G) for z in r] for r, e in zip(M, exps)]
    return exps, re, im


def ozaki_product(A, B, G):
    """C[m][n] = sum_k A[m][k] B[n][k] from the pairs s + t < G, as exact Fractions."""
    ea, ar, ai = slice_rows(A, G)
    eb, br, bi = slice_rows(B, G)
    M, K = A.shape
    N = B.shape[0]
    C = [[None] * N for _ in range(M)]
    for m in range(M):
        for n in range(N):
            re_sum = 0
            im_sum = 0
            for g in range(G):
                gr = gi = 0                 # one group over all of K (K <= 2048 / (g + 1) here)
                for s in range(g + 1):
                    t = g - s
                    for k in range(K):
                        gr += ar[m][k][s] * br[n][k][t] - ai[m][k][s] * bi[n][k][t]
                        gi += ar[m][k][s] * bi[n][k][t] + ai[m][k][s] * br[n][k][t]
                # exact in fp32: |sum| <= 2 (g + 1) K 2^(2P) must stay below 2^24
                assert abs(gr) < 2 ** 24 and abs(gi) < 2 ** 24
                re_sum += Fraction(gr) * Fraction(2) ** (-W * g)
                im_sum += Fraction(gi) * Fraction(2) ** (-W * g)
            scale = Fraction(2) ** (ea[m] + eb[n] - 2 * P)
            C[m][n] = (re_sum * scale, im_sum * scale)
    return C, ea, eb


def _operands(seed, M, N, K):
    rng = np.random.default_rng(seed)
    A = (rng.standard_normal((M, K)) + 1j * rng.standard_normal((M, K))) * np.exp(rng.uniform(-8, 8, (M, 1)))
    B = (rng.standard_normal((N, K)) + 1j * rng.standard_normal((N, K))) * np.exp(rng.uniform(-8, 8, (N, 1)))
    A[0, 1] = 0.0                        # exact zeros and a tie-prone value
    B[-1, 0] = 0.5 + 0.25j
    return A, B


@pytest.mark.parametrize("G", [1, 2, 3, 5, 8])
def test_digits_are_bounded_and_exact(G):
    F = P + W * (G - 1)
    rng = np.random.default_rng(G)
    for _ in range(400):
        e = int(rng.integers(-30, 30))
        x = float(rng.uniform(-1, 1)) * 2.0 ** e * (1 - 2 ** -53)
        X = to_fixed(x, e, F)
        d = digits(X, G)
        assert len(d) == G
        assert all(abs(v) <= 2 ** P for v in d), d
        assert sum(v << (W * (G - 1 - s)) for s, v in enumerate(d)) == X


@pytest.mark.parametrize("G", [1, 2, 4, 8])
def test_product_error_within_stated_bound(G):
    M, N, K = 4, 3, 37
    A, B = _operands(100 + G, M, N, K)
    C, ea, eb = ozaki_product(A, B, G)
    for m in range(M):
        for n in range(N):
            exact_re = sum(Fraction(A[m, k].real) * Fraction(B[n, k].real) - Fraction(A[m, k].imag) *
                           Fraction(B[n, k].imag) for k in range(K))
            exact_im = sum(Fraction(A[m, k].real) * Fraction(B[n, k].imag) + Fraction(A[m, k].imag) *
                           Fraction(B[n, k].real) for k in range(K))
            bound = (G + 2) * Fraction(2) ** (-W * G) * Fraction(2) ** (ea[m] + eb[n]) * K
            assert abs(C[m][n][0] - exact_re) <= bound
            assert abs(C[m][n][1] - exact_im) <= bound


def test_eight_slices_reach_fp64_accuracy():
    """With the default 8 slices the scheme's error is below an fp64 rounding of
    the largest possible entry (|C| <= 2 K 2^(e_m + e_n))."""
    A, B = _operands(7, 3, 3, 20)
    C, ea, eb = ozaki_product(A, B, 8)
    for m in range(3):
        for n in range(3):
            exact = sum(Fraction(A[m, k].real) * Fraction(B[n, k].real) - Fraction(A[m, k].imag) *
                        Fraction(B[n, k].imag) for k in range(20))
            scale = 2 * 20 * Fraction(2) ** (ea[m] + eb[n])
            assert abs(C[m][n][0] - exact) <= scale * Fraction(2) ** -53
