"""Bit-exact CPU model of the Ozaki-scheme complex GEMM of the library
(TEVO_OZAKI, C[m][n] = sum_k A[m][k] B[n][k]), as the header of csrc/k_oz.cu and
include/tevo.h describe its arithmetic. Test infrastructure: plain numpy and
Python integers, no code shared with the library.

Steps, per operand row r: the exponent e_r of its largest magnitude (from the
binary64 fields: max |Re|, |Im| < 2^e_r), the fixed-point integers
X = round(x 2^(F - e_r)) (ties to even, F = P + W (G - 1)) of the real and
imaginary parts, and their G balanced base-2^W digits. Per output tile the
K-range is cut as the kernel plans it (K-tiles of 32 in chunks of 8; split-K
over chunks when there are fewer tiles than SMs); per group g = s + t the
digit products are summed exactly over passes of at most 64 / (g + 1) K-tiles,
each pass value is shifted left by (base_shift + 28 h - W g) bits into the
64-bit fixed-point sum h = g // 4 (groups 0..3 and 4..7), both sums exact; the
entry is the exact value S0 2^28 + S1, rounded once to fp64. Split partials
are added in fp64 in split order, starting from 0.0.
"""
from __future__ import annotations

import math

import numpy as np

P, W = 6, 7
TM = TN = 128          # output tile of one CTA
KT = 32                # K-indices per K-tile
CHUNK = 8              # K-tiles per exact chunk
NONFINITE = None
HI_GROUPS = 4          # groups 0..3 in the first fixed-point sum, 4..7 in the second
LO_SHIFT = W * HI_GROUPS


def exp_bound(z):
    """e with max(|Re z|, |Im z|) < 2^e from the binary64 fields of the larger
    magnitude: biased exponent E -> E - 1022 (normal), -1022 (subnormal); None
    for zero, NONFINITE_E for a NaN or an infinity."""
    mag = max(abs(z.real), abs(z.imag))
    if mag == 0.0:
        return None
    if not math.isfinite(mag):
        return NONFINITE_E
    E = int(np.float64(mag).view(np.uint64)) >> 52
    return -1022 if E == 0 else E - 1022


NONFINITE_E = "nonfinite"


def row_exponents(X):
    """e_r: the largest exponent bound over row r; 0 for a zero row, None
    (NONFINITE) when the row holds a NaN or an infinity."""
    R, K = X.shape
    out = []
    for r in range(R):
        best, bad = None, False
        for k in range(K):
            e = exp_bound(X[r, k])
            if e is None:
                continue
            if e == NONFINITE_E:
                bad = True
                continue
            best = e if best is None else max(best, e)
        out.append(NONFINITE if bad else (0 if best is None else best))
    return out


def to_fixed(x, e, F):
    """round(x 2^(F - e)), ties to even, for |x| < 2^e (exact, via the binary64 fields)."""
    x = float(x)
    if x == 0.0:
        return 0
    m, ex = math.frexp(abs(x))              # |x| = m 2^ex, 0.5 <= m < 1
    mi = int(m * (1 << 53))                 # |x| = mi 2^(ex - 53), exact
    sh = ex - 53 - e + F
    if sh >= 0:
        X = mi << sh
    else:
        q = -sh
        X = mi >> q
        rem = mi - (X << q)
        half = 1 << (q - 1)
        if rem > half or (rem == half and X & 1):
            X += 1
    return -X if x < 0 else X


def digits(X, G):
    """Balanced base-2^W digits d_0..d_{G-1}, X = sum_s d_s 2^(W (G - 1 - s))."""
    out = []
    rem = X
    for _ in range(G - 1):
        d = ((rem + (1 << (W - 1))) % (1 << W)) - (1 << (W - 1))
        out.append(d)
        rem = (rem - d) >> W
    out.append(rem)
    return out[::-1]


def slices(X, G):
    """(exponents, re digits [G][R][K], im digits [G][R][K]) of the rows of X."""
    R, K = X.shape
    F = P + W * (G - 1)
    exps = row_exponents(X)
    dre = np.zeros((G, R, K), np.int64)
    dim = np.zeros((G, R, K), np.int64)
    for r in range(R):
        e = exps[r]
        if e is NONFINITE:
            continue                          # digits zero, outputs NaN
        for k in range(K):
            z = X[r, k]
            dre[:, r, k] = digits(to_fixed(z.real, e, F), G)
            dim[:, r, k] = digits(to_fixed(z.imag, e, F), G)
    return exps, dre, dim


def plan(M, N, K, num_sms):
    k_tiles = -(-K // KT)
    nchunks = -(-k_tiles // CHUNK)
    tiles = -(-M // TM) * -(-N // TN)
    splits = max(1, min(-(-num_sms // tiles), nchunks))
    splits = min(splits, 64)
    cps = -(-nchunks // splits)
    splits = -(-nchunks // cps)
    lg = 0
    while (1 << lg) < cps:
        lg += 1
    return k_tiles, nchunks, cps, splits, 38 - lg


def gemm(A, B, G=8, num_sms=152):
    """The library's TEVO_OZAKI_SLICES(G) product C = A B^T, bit for bit."""
    A = np.asarray(A, np.complex128)
    B = np.asarray(B, np.complex128)
    M, K = A.shape
    N = B.shape[0]
    k_tiles, nchunks, cps, splits, base_shift = plan(M, N, K, num_sms)
    Kp = k_tiles * KT
    pad = lambda X: np.pad(X, ((0, 0), (0, Kp - K)))
    ea, ar, ai = slices(pad(A), G)
    eb, br, bi = slices(pad(B), G)
    partials = []
    for z in range(splits):
        t0 = z * cps * CHUNK
        t1 = min(k_tiles, (z + 1) * cps * CHUNK)
        S_re = np.zeros((2, M, N), np.int64)
        S_im = np.zeros((2, M, N), np.int64)
        for g in range(G):
            plen = 64 // (g + 1)
            h = g // HI_GROUPS
            shift = base_shift + LO_SHIFT * h - W * g
            assert shift >= 0
            for p0 in range(t0, t1, plen):
                k0, k1 = p0 * KT, min(t1, p0 + plen) * KT
                v_re = np.zeros((M, N), np.int64)
                v_im = np.zeros((M, N), np.int64)
                for s in range(g + 1):
                    t = g - s
                    a_r, a_i = ar[s][:, k0:k1], ai[s][:, k0:k1]
                    b_r, b_i = br[t][:, k0:k1], bi[t][:, k0:k1]
                    v_re += a_r @ b_r.T - a_i @ b_i.T
                    v_im += a_r @ b_i.T + a_i @ b_r.T
                assert np.abs(v_re).max(initial=0) < 2 ** 24 and np.abs(v_im).max(initial=0) < 2 ** 24
                S_re[h] += v_re << shift
                S_im[h] += v_im << shift
                assert np.abs(S_re[h]).max(initial=0) < 2 ** 63 and np.abs(S_im[h]).max(initial=0) < 2 ** 63
        part = np.empty((M, N), np.complex128)
        for m in range(M):
            for n in range(N):
                if ea[m] is NONFINITE or eb[n] is NONFINITE:
                    part[m, n] = complex(math.nan, math.nan)
                    continue
                e2 = ea[m] + eb[n] - 2 * P - base_shift - LO_SHIFT
                tot_re = (int(S_re[0, m, n]) << LO_SHIFT) + int(S_re[1, m, n])
                tot_im = (int(S_im[0, m, n]) << LO_SHIFT) + int(S_im[1, m, n])
                part[m, n] = complex(_scaled(tot_re, e2), _scaled(tot_im, e2))
        partials.append(part)
    if splits == 1:
        return partials[0]
    out = np.zeros((M, N), np.complex128)
    for p in partials:                       # 0.0 + p_0 + p_1 + ..., per part
        out.real = out.real + p.real
        out.imag = out.imag + p.imag
    return out


def _scaled(s, e2):
    """s 2^e2 rounded to fp64 (s an integer; float() rounds it to nearest, ties
    to even)."""
    try:
        return math.ldexp(float(s), e2)
    except OverflowError:
        return math.copysign(math.inf, s)
