"""GPU tests of the Ozaki-scheme fp64 GEMM (tevo_gemm with TEVO_OZAKI, through the
C ABI) and of evolve_step with its fp64 contractions computed that way, against
numpy fp64 products and the fp64 oracle."""
import ctypes

import numpy as np
import pytest

import workloads as wl
from oracle import fit, mpo

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)
tv = pytest.importorskip("paper_2302_14181_gb300")


@pytest.fixture(scope="module")
def ctx():
    torch.cuda.set_device(0)
    return tv.Context()


def gemm(ctx, prec, A, B):
    M, K = A.shape
    N = B.shape[0]
    a = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    b = torch.from_numpy(np.ascontiguousarray(B)).cuda()
    c = torch.full((M, N), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
    rc = tv._lib.lib.tevo_gemm(ctx.handle, prec, M, N, K, ctypes.c_void_p(a.data_ptr()),
                               ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(c.data_ptr()))
    assert rc == 0, rc
    return c.cpu().numpy()


def bound(G, A, B):
    """Dropped part of the G-slice product: about (G + 2) 2^(-7G) max|A| max|B| K per
    entry (digits carry 7 bits; pairs with s + t >= G are left out)."""
    K = A.shape[1]
    return (G + 2) * 2.0 ** (-7 * G) * np.abs(A).max() * np.abs(B).max() * K


def test_integer_operands_give_the_exact_product(ctx):
    """Integers below 2^20 are cut into three exact digit slices; every retained
    product and every pass sum is exact, so C equals the integer product."""
    rng = np.random.default_rng(3)
    A = rng.integers(-2**20, 2**20, (300, 512)) + 1j * rng.integers(-2**20, 2**20, (300, 512))
    B = rng.integers(-2**20, 2**20, (200, 512)) + 1j * rng.integers(-2**20, 2**20, (200, 512))
    ref = A @ B.T  # integer-valued, |.| < 2^50: exact in fp64
    for G in (5, 7, 8):
        assert np.array_equal(gemm(ctx, tv.OZAKI_SLICES(G), A, B), ref), G


@pytest.mark.parametrize("shape", [(128, 128, 32), (300, 200, 777), (513, 257, 33), (37, 5, 1000), (1, 1, 1),
                                   (200, 100, 20000), (130, 2000, 512)])
def test_random_operands_within_the_slice_bound(ctx, shape):
    M, N, K = shape
    rng = np.random.default_rng(M + 7 * N + 11 * K)
    A = rng.standard_normal((M, K)) + 1j * rng.standard_normal((M, K))
    B = rng.standard_normal((N, K)) + 1j * rng.standard_normal((N, K))
    ref = A @ B.T
    got = gemm(ctx, tv.OZAKI, A, B)
    assert np.isfinite(got).all()
    assert np.abs(got - ref).max() <= bound(7, A, B)
    # and as accurate as the native fp64 contraction to within a small factor
    native = gemm(ctx, tv.FP64, A, B)
    assert np.abs(got - ref).max() <= 64 * max(np.abs(native - ref).max(), 1e-300) + bound(7, A, B) / 8


def test_error_falls_with_the_slice_count(ctx):
    rng = np.random.default_rng(5)
    A = rng.standard_normal((256, 640)) + 1j * rng.standard_normal((256, 640))
    B = rng.standard_normal((384, 640)) + 1j * rng.standard_normal((384, 640))
    ref = A @ B.T
    errs = []
    for G in range(2, 9):
        e = np.abs(gemm(ctx, tv.OZAKI_SLICES(G), A, B) - ref).max()
        assert e <= bound(G, A, B), (G, e)
        errs.append(e)
    # 7 more bits per slice until fp64 rounding takes over
    for G in range(2, 6):
        assert errs[G - 2 + 1] < errs[G - 2] / 16, errs


def test_rows_of_very_different_magnitude(ctx):
    """Each row carries its own power-of-two scale, so rows far apart in size
    keep their relative accuracy."""
    rng = np.random.default_rng(9)
    A = rng.standard_normal((200, 300)) + 1j * rng.standard_normal((200, 300))
    B = rng.standard_normal((150, 300)) + 1j * rng.standard_normal((150, 300))
    A *= np.logspace(-30, 30, 200)[:, None]
    B *= np.logspace(20, -20, 150)[:, None]
    ref = A @ B.T
    got = gemm(ctx, tv.OZAKI, A, B)
    row_scale = np.abs(A).max(axis=1)[:, None] * np.abs(B).max(axis=1)[None, :] * 300
    assert (np.abs(got - ref) <= 9 * 2.0 ** -49 * row_scale).all()


def test_nonfinite_rows_give_nan_outputs(ctx):
    """Digits of a row holding NaN or Inf are not formed; the entries that row
    touches come out NaN (so the evolution's non-finite check still fires)."""
    rng = np.random.default_rng(13)
    A = rng.standard_normal((40, 64)) + 1j * rng.standard_normal((40, 64))
    B = rng.standard_normal((30, 64)) + 1j * rng.standard_normal((30, 64))
    A[3, 7] = np.nan
    B[5, 2] = np.inf
    got = gemm(ctx, tv.OZAKI, A, B)
    bad = np.zeros(got.shape, bool)
    bad[3, :] = True
    bad[:, 5] = True
    assert np.isnan(got[bad]).all()
    ref = A @ B.T
    assert np.abs(got[~bad] - ref[~bad]).max() <= bound(7, A[np.isfinite(A).all(1)], B[np.isfinite(B).all(1)])


def test_bad_ozaki_flags_are_rejected(ctx):
    A = np.ones((4, 4), np.complex128)
    a = torch.from_numpy(A).cuda()
    c = torch.zeros((4, 4), dtype=torch.complex128, device="cuda")
    for prec in (tv.OZAKI_SLICES(9), tv.BF16X3 | tv.OZAKI, tv.OZAKI | tv.TC_ONLY, 5 << 12):
        rc = tv._lib.lib.tevo_gemm(ctx.handle, prec, 4, 4, 4, ctypes.c_void_p(a.data_ptr()),
                                   ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(c.data_ptr()))
        assert rc == -1, hex(prec)


def rel_err(got, ref):
    return float(np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-3))


@pytest.mark.parametrize("prec,tol", [(tv.FP64 | tv.OZAKI, 1e-10), (tv.BF16X3 | tv.OZAKI, 1e-8),
                                      (tv.TF32X3 | tv.OZAKI, 1e-8)])
def test_evolve_with_ozaki_contractions_against_oracle(ctx, prec, tol):
    """XXZ, order 2, D = 16, two sweeps per step: all-Ozaki (FP64 | OZAKI) and the
    mixed forms whose fp64 rebuild and final sweep run as Ozaki GEMMs."""
    L, N, D, tau = 16, 2, 16, -0.2j
    blocks = wl.xxz_blocks(L, 0.5)
    v0 = wl.product_state("neel", L)
    ops = list(wl.pauli())
    Wo = mpo.build_mpo(*blocks, N, tau)
    W = tv.mpo_build(ctx, *blocks, N, tau)
    psi_o = fit.product_mps(v0, D)
    psi = tv.mps_init(ctx, v0, D)
    errs = []
    for k in range(4):
        psi_o, _ = fit.evolve_step(psi_o, Wo, 2, canonical=k > 0)
        tv.evolve_step(psi, W, tau, D, 2, prec)
        errs.append(rel_err(tv.measure_local(psi, ops).real, fit.measure_local(psi_o, ops).real))
    assert max(errs) < tol, errs


def test_evolve_ozaki_lri_ragged(ctx):
    """Long-range Ising, order 3 (w = 93), D = 40: ragged tiles, K of the apply
    (w D = 3720) split over several CTAs, conjugated operand of the environment
    update."""
    L, N, D, tau = 14, 3, 40, -0.2j
    blocks = wl.lr_ising_blocks(L, 0.7)
    v0 = wl.product_state("up", L)
    ops = list(wl.pauli())
    Wo = mpo.build_mpo(*blocks, N, tau)
    W = tv.mpo_build(ctx, *blocks, N, tau)
    psi_o = fit.product_mps(v0, D)
    psi = tv.mps_init(ctx, v0, D)
    for k in range(3):
        psi_o, _ = fit.evolve_step(psi_o, Wo, 2, canonical=k > 0)
        tv.evolve_step(psi, W, tau, D, 2, tv.FP64 | tv.OZAKI)
    assert rel_err(tv.measure_local(psi, ops).real, fit.measure_local(psi_o, ops).real) < 1e-10
    assert np.isfinite(psi.log_norm())


def test_ozaki_not_built_for_the_batched_form(ctx):
    blocks = wl.xxz_blocks(8, 0.5)
    W = tv.mpo_build(ctx, *blocks, 2, -0.1j)
    psis = [tv.mps_init(ctx, wl.product_state("neel", 8), 8) for _ in range(2)]
    with pytest.raises(tv.TevoError):
        tv.evolve_step_batched(psis, [W, W], 1, tv.BF16X3 | tv.OZAKI)


@pytest.mark.parametrize("shape,G", [((37, 45, 70), 8), ((130, 129, 300), 8), ((64, 40, 2100), 8),
                                     ((64, 40, 2100), 5), ((90, 33, 600), 4), ((5, 60, 9000), 8)])
def test_kernel_matches_the_cpu_model_bit_for_bit(ctx, shape, G):
    """The kernel computes exactly what tests/ozaki_model.py states: the digit
    slices, the K-split plan, the exact per-group pass sums, the two exact
    fixed-point accumulators, one rounding per entry and the fp64 sum of split
    partials. Ragged shapes, several passes and chunks, split-K, and slice
    counts that use one or both accumulators."""
    import ozaki_model
    M, N, K = shape
    rng = np.random.default_rng(M * 31 + N * 7 + K + G)
    A = rng.standard_normal((M, K)) + 1j * rng.standard_normal((M, K))
    B = rng.standard_normal((N, K)) + 1j * rng.standard_normal((N, K))
    # rows spanning several binary orders of magnitude
    A *= np.exp2(rng.integers(-30, 30, (M, 1))) * np.exp2(rng.integers(-8, 1, (M, K)))
    B *= np.exp2(rng.integers(-30, 30, (N, 1)))
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    got = gemm(ctx, tv.OZAKI_SLICES(G), A, B)
    ref = ozaki_model.gemm(A, B, G=G, num_sms=sms)
    assert np.array_equal(got.view(np.float64), ref.view(np.float64))
