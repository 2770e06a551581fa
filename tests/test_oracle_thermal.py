"""Finite-temperature states by purification (the finite-chain analogue of
Sec. 8.4): the oracle's dense Gibbs averages are pinned, then the oracle's fit
of W^(N)(tau) with real tau = -beta / (2 n) applied n times to the product of
maximally entangled (physical, ancilla) pairs reproduces them up to the MPO's
order."""
import numpy as np
import pytest

import workloads as wl
from oracle import dense, fit, mpo

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def tfi(L, g=1.05):
    return wl.tfi_blocks(L, g)


def test_thermal_expect_limits_and_expm():
    L = 5
    H = dense.hamiltonian_from_blocks(*tfi(L))
    X, Y, Z = wl.pauli()
    # beta = 0: Tr(O) / d
    t0 = dense.thermal_expect(H, 0.0, [X, Z, np.eye(2)], L)
    assert np.allclose(t0[0], 0) and np.allclose(t0[1], 0) and np.allclose(t0[2], 1)
    # large beta: the ground state's values (gapped chain)
    e, U = np.linalg.eigh(H)
    gs = U[:, 0]
    ref = dense.expect_dense(gs, [X, Z], L)
    assert np.abs(dense.thermal_expect(H, 60.0, [X, Z], L) - ref).max() < 1e-10
    # against scipy's expm at beta = 0.7
    sla = pytest.importorskip("scipy.linalg")
    rho = sla.expm(-0.7 * H)
    rho /= np.trace(rho)
    for i in range(L):
        assert abs(np.trace(dense.local_op(X, i, L) @ rho) - dense.thermal_expect(H, 0.7, [X], L)[0, i]) < 1e-12


def test_purified_product_state_is_infinite_temperature():
    """Tracing the ancillas of the purified product state leaves 1/d^L."""
    L, d = 3, 2
    v = dense.product_vector(wl.purified_infinite_temperature(L, d))
    # reorder (p1 a1 p2 a2 ...) -> (p..., a...) and trace the ancillas
    psi = v.reshape([d, d] * L).transpose(list(range(0, 2 * L, 2)) + list(range(1, 2 * L, 2)))
    psi = psi.reshape(d ** L, d ** L)
    assert np.allclose(psi @ psi.conj().T, np.eye(d ** L) / d ** L)


@pytest.mark.parametrize("N", [1, 2, 3])
def test_purification_fit_matches_gibbs_state(N):
    """L = 6 TFI, beta = 1 in n steps of tau = -beta / (2 n), D not limiting:
    <X_i>, <Z_i> of the fitted purification equal the Gibbs averages up to the
    order-N MPO's error, which falls as n grows (by about 2^N for twice the
    steps)."""
    L, beta = 6, 1.0
    blocks = tfi(L)
    H = dense.hamiltonian_from_blocks(*blocks)
    X, Y, Z = wl.pauli()
    exact = dense.thermal_expect(H, beta, [X, Z], L).real
    ops = [wl.purify_op(X), wl.purify_op(Z)]
    pb = wl.purify_blocks(*blocks)
    errs = []
    for n in (5, 10):
        tau = -beta / (2 * n)
        W = mpo.build_mpo(*pb, N, tau)
        psi = fit.product_mps(wl.purified_infinite_temperature(L, 2), 64)
        psi, _, _ = fit.evolve(psi, W, n, sweeps=2)
        errs.append(np.abs(fit.measure_local(psi, ops).real - exact).max())
    assert errs[0] < 0.05 * 10 ** (-(N - 1))
    assert errs[1] < errs[0] / (2 ** N * 0.6)
