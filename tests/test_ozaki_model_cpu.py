"""The bit-exact CPU model of the Ozaki-scheme GEMM (tests/ozaki_model.py), pinned
on the CPU: exact products of small integers, the documented error bound
against exact rational products, NaN rows, and the split-K planning."""
from fractions import Fraction

import numpy as np
import pytest

import ozaki_model as oz


def _exact(A, B):
    M, K = A.shape
    N = B.shape[0]
    out = np.empty((M, N), dtype=object)
    for m in range(M):
        for n in range(N):
            re = im = Fraction(0)
            for k in range(K):
                ar, ai = Fraction(A[m, k].real), Fraction(A[m, k].imag)
                br, bi = Fraction(B[n, k].real), Fraction(B[n, k].imag)
                re += ar * br - ai * bi
                im += ar * bi + ai * br
            out[m, n] = (re, im)
    return out


def test_plan_matches_the_kernel_rules():
    # K = 200: one chunk, no split; K = 300: two chunks over one tile, two splits
    assert oz.plan(4, 4, 200, 152) == (7, 1, 1, 1, 38)
    assert oz.plan(4, 4, 300, 152) == (10, 2, 1, 2, 38)
    # many chunks on one tile: at most 64 splits, chunks per split grow, S unit shrinks
    k_tiles, nchunks, cps, splits, base_shift = oz.plan(4, 4, 50000, 152)
    assert (k_tiles, nchunks, cps, splits, base_shift) == (1563, 196, 4, 49, 36)
    # enough tiles to fill the GPU: no split
    assert oz.plan(23808, 512, 256, 152)[3] == 1


@pytest.mark.parametrize("K", [5, 200, 300, 700])
def test_small_integers_give_exact_products(K):
    rng = np.random.default_rng(K)
    A = rng.integers(-9, 10, (3, K)) + 1j * rng.integers(-9, 10, (3, K))
    B = rng.integers(-9, 10, (5, K)) + 1j * rng.integers(-9, 10, (5, K))
    C = oz.gemm(A, B)
    assert np.array_equal(C, A @ B.T)


@pytest.mark.parametrize("G,K", [(8, 40), (8, 300), (5, 300), (3, 100)])
def test_error_within_the_documented_bound(G, K):
    rng = np.random.default_rng(1000 + K + G)
    M, N = 3, 4
    A = (rng.standard_normal((M, K)) + 1j * rng.standard_normal((M, K))) * np.exp(rng.uniform(-6, 6, (M, 1)))
    B = (rng.standard_normal((N, K)) + 1j * rng.standard_normal((N, K))) * np.exp(rng.uniform(-6, 6, (N, 1)))
    C = oz.gemm(A, B, G=G)
    ex = _exact(A, B)
    ea, eb = oz.row_exponents(A), oz.row_exponents(B)
    _, _, cps, splits, base_shift = oz.plan(M, N, K, 152)
    npass = sum(-(-cps * oz.CHUNK // (64 // (g + 1))) for g in range(G))
    for m in range(M):
        for n in range(N):
            unit = Fraction(2) ** (ea[m] + eb[n])
            # dropped digits and pairs, the floor of each shifted pass value, one
            # fp64 rounding per split partial and per fp64 addition of partials
            tol = ((G + 2) * Fraction(2) ** (-oz.W * G) * K * unit
                   + splits * npass * unit * Fraction(2) ** (-2 * oz.P - base_shift))
            for part, got in ((0, C[m, n].real), (1, C[m, n].imag)):
                e = ex[m, n][part]
                rounding = (2 * splits + 1) * Fraction(2) ** -53 * (abs(e) + tol)
                assert abs(Fraction(got) - e) <= tol + rounding, (G, K, m, n, part)


def test_nonfinite_rows_give_nan_in_their_row_and_column_only():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((3, 50)) + 1j * rng.standard_normal((3, 50))
    B = rng.standard_normal((4, 50)) + 1j * rng.standard_normal((4, 50))
    A[1, 7] = np.nan
    B[2, 0] = np.inf
    C = oz.gemm(A, B)
    bad = np.zeros((3, 4), bool)
    bad[1, :] = True
    bad[:, 2] = True
    assert np.all(np.isnan(C.real[bad])) and np.all(np.isnan(C.imag[bad]))
    assert np.all(np.isfinite(C[~bad]))
    with np.errstate(invalid="ignore"):
        ref = A @ B.T
    assert np.allclose(C[~bad], ref[~bad], rtol=1e-13, atol=0)


def test_digits_and_fixed_point_of_the_model():
    for G in (1, 4, 8):
        F = oz.P + oz.W * (G - 1)
        rng = np.random.default_rng(G)
        for _ in range(300):
            e = int(rng.integers(-40, 40))
            x = float(rng.uniform(-1, 1)) * 2.0 ** e
            X = oz.to_fixed(x, e, F)
            assert abs(Fraction(X) - Fraction(x) * Fraction(2) ** (F - e)) <= Fraction(1, 2)
            d = oz.digits(X, G)
            assert all(abs(v) <= 2 ** oz.P for v in d)
            assert sum(v << (oz.W * (G - 1 - s)) for s, v in enumerate(d)) == X
    # ties go to even
    assert oz.to_fixed(2.5, 3, 1) == 1
    assert oz.to_fixed(1.0, 2, 1) == 0                       # 0.5 -> 0 (even)
    assert oz.to_fixed(3.0, 2, 1) == 2                       # 1.5 -> 2 (even)
    assert oz.to_fixed(-3.0, 2, 1) == -2

