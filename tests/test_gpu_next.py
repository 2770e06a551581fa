"""Uses of evolve_step beyond real-time steps with one MPO: complex-step
splitting (Sec. 8.3) and real tau (imaginary time, towards the ground state)."""
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


def test_splitting_two_complex_steps(ctx):
    """Alternating first-order MPOs at tau (1 +- i)/2: the GPU path equals the
    oracle doing the same, and both approach exp(tau H) to second order."""
    L, D, t = 10, 32, 0.1
    blocks = wl.xxz_blocks(L, 0.5)
    tau = -1j * t
    taus = (tau * (1 + 1j) / 2, tau * (1 - 1j) / 2)
    Wg = [tv.mpo_build(ctx, *blocks, 1, s) for s in taus]
    Wo = [mpo.build_mpo(*blocks, 1, s) for s in taus]
    v0 = wl.product_state("neel", L)
    psi = tv.mps_init(ctx, v0, D)
    ref = fit.product_mps(v0, D)
    ops = list(wl.pauli())
    for k in range(8):
        j = k % 2
        tv.evolve_step(psi, Wg[j], taus[j], D, 1, tv.FP64)
        ref, _ = fit.evolve_step(ref, Wo[j], 1, canonical=k > 0)
    got, exp_o = tv.measure_local(psi, ops).real, fit.measure_local(ref, ops).real
    assert np.abs(got - exp_o).max() < 1e-10
    H = dense.hamiltonian_from_blocks(*blocks)
    v = dense.product_vector(v0)
    E = dense.expm_tau_h(H, tau)
    for _ in range(4):
        v = E @ v
    exact = dense.expect_dense(v, ops, L).real
    assert np.abs(got - exact).max() < 5e-3


def test_imaginary_time_reaches_ground_state(ctx):
    """tau = -0.1 (real): repeated normalised steps project onto the ground state
    of the transverse-field Ising chain (gap 0.37 at L = 10, g = 1.05); after
    beta = 12 the order-3 MPO's fixed point is within about 1e-4 of the exact
    ground state (from eigh) in <X_i>, and the GPU path equals the oracle."""
    L, D, N = 10, 32, 3
    blocks = wl.tfi_blocks(L, 1.05)
    tau = -0.1
    W = tv.mpo_build(ctx, *blocks, N, tau)
    Wo = mpo.build_mpo(*blocks, N, tau)
    v0 = wl.product_state("up", L)
    psi = tv.mps_init(ctx, v0, D)
    ref = fit.product_mps(v0, D)
    X, _, Z = wl.pauli()
    for k in range(120):
        tv.evolve_step(psi, W, tau, D, 1, tv.FP64)
        if k < 10:
            ref, _ = fit.evolve_step(ref, Wo, 1, canonical=k > 0)
        if k == 9:
            assert np.abs(tv.measure_local(psi, [X, Z]).real - fit.measure_local(ref, [X, Z]).real).max() < 1e-10
    H = dense.hamiltonian_from_blocks(*blocks)
    e, U = np.linalg.eigh(H)
    gs = U[:, 0]
    exact = dense.expect_dense(gs, [X], L).real
    assert np.abs(tv.measure_local(psi, [X]).real - exact).max() < 1e-3
