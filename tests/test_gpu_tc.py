"""GPU tests of the tensor-core contraction (tevo_gemm through the C ABI) and of
the mixed-precision evolve_step against the fp64 oracle."""
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

# max |C - C_ref| / max |C_ref| for random complex Gaussian operands
GEMM_TOL = {tv.FP64: 1e-12, tv.BF16X3: 1e-4, tv.TF32X3: 1e-5, tv.TF32: 3e-3}


@pytest.fixture(scope="module")
def ctx():
    torch.cuda.set_device(0)
    return tv.Context()


def tc_gemm(ctx, prec, A, B):
    M, K = A.shape
    N = B.shape[0]
    a = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    b = torch.from_numpy(np.ascontiguousarray(B)).cuda()
    c = torch.zeros((M, N), dtype=torch.complex128, device="cuda")
    tv._lib.check(tv._lib.lib.tevo_gemm(ctx.handle, prec, M, N, K, ctypes.c_void_p(a.data_ptr()),
                                        ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(c.data_ptr())))
    return c.cpu().numpy()


@pytest.mark.parametrize("prec", [tv.FP64, tv.BF16X3, tv.TF32X3, tv.TF32])
@pytest.mark.parametrize("shape", [(128, 256, 64), (200, 300, 100), (37, 5, 1000), (1, 1, 1), (300, 600, 2000),
                                   (513, 257, 33)])
def test_gemm_matches_numpy(ctx, prec, shape):
    M, N, K = shape
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    A = rng.standard_normal((M, K)) + 1j * rng.standard_normal((M, K))
    B = rng.standard_normal((N, K)) + 1j * rng.standard_normal((N, K))
    C = tc_gemm(ctx, prec, A, B)
    ref = A @ B.T
    err = np.abs(C - ref).max() / np.abs(ref).max()
    assert err < GEMM_TOL[prec], (prec, shape, err)


def test_gemm_structured_signs(ctx):
    """Purely real / purely imaginary operands isolate the four real products and
    the sign of Ai.Bi."""
    M, N, K = 130, 260, 70
    rng = np.random.default_rng(1)
    X = rng.standard_normal((M, K))
    Y = rng.standard_normal((N, K))
    for prec in (tv.BF16X3, tv.TF32X3, tv.TF32):
        for A, B in ((X, Y), (1j * X, Y), (X, 1j * Y), (1j * X, 1j * Y)):
            C = tc_gemm(ctx, prec, A.astype(np.complex128), B.astype(np.complex128))
            ref = A @ B.T
            assert np.abs(C - ref).max() / np.abs(ref).max() < GEMM_TOL[prec]


def rel_err(got, ref):
    return float(np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-3))


@pytest.mark.parametrize("prec", [tv.BF16X3, tv.TF32X3, tv.TF32])
def test_mixed_evolve_against_oracle(ctx, prec):
    """sweeps = 2: one tensor-core sweep, then an fp64 rebuild of the right
    environments and one fp64 sweep; compared with the oracle's two fp64 sweeps."""
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
    assert max(errs) < 1e-6, errs


def test_mixed_lri_ragged(ctx):
    """Long-range Ising, order 3 (w = 93, K of G2 = 186 not a tile multiple),
    D = 40 (ragged tiles), bf16x3 sweep + fp64 sweep."""
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
        tv.evolve_step(psi, W, tau, D, 2, tv.BF16X3)
    assert rel_err(tv.measure_local(psi, ops).real, fit.measure_local(psi_o, ops).real) < 1e-6


def test_bounded_wait_gives_up_and_context_survives(ctx):
    """A device wait on a barrier that nothing completes ends after its limit with
    an error status (TEVO_ETIMEOUT) instead of hanging; the context still works."""
    code = ctypes.c_int(0)
    rc = tv._lib.lib.tevo_wait_selftest(ctx.handle, 50.0, ctypes.byref(code))
    assert rc == -7 and code.value == 7
    A = np.ones((4, 3), np.complex128)
    assert np.allclose(tc_gemm(ctx, tv.BF16X3, A, A), A @ A.T)


@pytest.mark.parametrize("prec,tol", [(tv.BF16X3 | tv.TC_ONLY, 2e-3), (tv.TF32X3 | tv.TC_ONLY, 2e-4)])
def test_tensor_core_only_forms_against_oracle(ctx, prec, tol):
    """Every sweep on the tensor cores (no fp64 sweep; fp64 QR and reductions):
    the long-range Ising chain at L = 20, D = 24, N = 3, 4 steps of 2 sweeps,
    against the fp64 oracle. The tolerance follows the split products' relative
    error per contraction (bf16x3 about 2^-16, tf32x3 about 2^-22) times the
    growth over the steps."""
    L, D, N, tau = 20, 24, 3, -0.2j
    blocks = wl.lr_ising_blocks(L, 0.7)
    v0 = wl.product_state("up", L)
    ops = list(wl.pauli())
    Wo = mpo.build_mpo(*blocks, N, tau)
    W = tv.mpo_build(ctx, *blocks, N, tau)
    psi = tv.mps_init(ctx, v0, D)
    psi_o = fit.product_mps(v0, D)
    errs = []
    for k in range(4):
        psi_o, _ = fit.evolve_step(psi_o, Wo, 2, canonical=k > 0)
        tv.evolve_step(psi, W, tau, D, 2, prec)
        ref = fit.measure_local(psi_o, ops).real
        errs.append(float(np.abs(tv.measure_local(psi, ops).real - ref).max() / max(np.abs(ref).max(), 1e-3)))
    print("tc-only", hex(prec), [f"{e:.1e}" for e in errs])
    assert max(errs) < tol, errs
