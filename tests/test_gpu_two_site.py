"""The two-site form of the fit (TEVO_TWO_SITE, Sec. 2.2) on the GPU against the
oracle's two-site fit: Theta from the GEMM engines, its leading left singular
vectors by one-sided Jacobi rotations in fp64, re-gauged by the Householder
QR."""
import numpy as np
import pytest

import workloads as wl
from oracle import dense, fit, mpo

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)
tv = pytest.importorskip("paper_2302_14181_gb300")


@pytest.fixture(scope="module")
def ctx():
    torch.cuda.set_device(0)
    return tv.Context()


def test_two_site_exact_from_a_product_state(ctx):
    """XXZ L = 8, Neel start, D = 16 (bonds do not limit), order 2, 4 steps of one
    sweep: the GPU state equals W^k|psi> (dense) and the oracle's two-site fit,
    with the rank-deficient first steps handled by the Jacobi basis."""
    L, D, tau = 8, 16, -0.2j
    blocks = wl.xxz_blocks(L, 0.5)
    W = tv.mpo_build(ctx, *blocks, 2, tau)
    Wo = mpo.build_mpo(*blocks, 2, tau)
    v0 = wl.product_state("neel", L)
    psi = tv.mps_init(ctx, v0, D)
    ref = fit.product_mps(v0, D)
    U = dense.mpo_to_dense(Wo)
    v = dense.product_vector(v0)
    ops = list(wl.pauli())
    for k in range(4):
        tv.evolve_step(psi, W, tau, D, 1, tv.FP64 | tv.TWO_SITE)
        ref, _ = fit.evolve_step_two_site(ref, Wo, 1, canonical=k > 0)
        v = U @ v
        got = tv.measure_local(psi, ops).real
        assert np.abs(got - fit.measure_local(ref, ops).real).max() < 1e-10, k
        assert np.abs(got - dense.expect_dense(v, ops, L).real).max() < 1e-10, k


@pytest.mark.parametrize("prec,tol", [(tv.FP64 | tv.TWO_SITE, 1e-10), (tv.FP64 | tv.OZAKI | tv.TWO_SITE, 1e-8)])
def test_two_site_truncating_against_oracle(ctx, prec, tol):
    """TFI L = 10, D = 6 (the bonds truncate), order 2 at tau = -0.3i from a
    seeded random state, 3 steps of 2 sweeps: observables and log-norm equal the
    oracle's two-site fit (generic singular values, so the kept subspace is
    unique)."""
    L, D, tau = 10, 6, -0.3j
    blocks = wl.tfi_blocks(L, 1.05)
    W = tv.mpo_build(ctx, *blocks, 2, tau)
    Wo = mpo.build_mpo(*blocks, 2, tau)
    start = wl.random_mps(L, 2, D, seed=3)
    psi = tv.mps_init(ctx, np.ones((L, 2)) / np.sqrt(2), D)
    for i in range(L):
        psi.set_site(i, start[i])
    ref = [x.copy() for x in start]
    logn = 0.0
    ops = list(wl.pauli())
    for k in range(3):
        tv.evolve_step(psi, W, tau, D, 2, prec)
        ref, ln = fit.evolve_step_two_site(ref, Wo, 2, canonical=k > 0)
        logn += ln
    assert np.abs(tv.measure_local(psi, ops).real - fit.measure_local(ref, ops).real).max() < tol
    assert abs(psi.log_norm() - logn) < tol


def test_two_site_flag_rules(ctx):
    L, D, tau = 6, 8, -0.1j
    blocks = wl.tfi_blocks(L, 1.05)
    W = tv.mpo_build(ctx, *blocks, 2, tau)
    psi = tv.mps_init(ctx, wl.product_state("up", L), D)
    with pytest.raises(tv.TevoError):
        tv.evolve_step(psi, W, tau, D, 2, tv.BF16X3 | tv.TWO_SITE)
    with pytest.raises(tv.TevoError):
        tv.evolve_step_batched([psi], [W], 1, tv.FP64 | tv.TWO_SITE)
