"""Pins for the oracle's fit, QR and observables (oracle/fit.py, oracle/dense.py).
CPU only."""
import numpy as np
import pytest
import scipy.linalg

import workloads as wl
from oracle import dense, fit, mpo


def crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


# ----------------------------------------------------------------------------
# Householder QR
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("m,n", [(1, 1), (4, 4), (7, 3), (64, 32), (130, 65)])
def test_qr_matches_lapack_convention(m, n):
    """Full-rank input: Q^H Q = 1, Q R = M, R upper triangular with the LAPACK
    real-diagonal convention, so R and Q equal numpy's (LAPACK zgeqrf/zungqr)."""
    rng = np.random.default_rng(m * 100 + n)
    M = crandn(rng, m, n)
    Q, R = fit.householder_qr(M)
    assert np.abs(Q.conj().T @ Q - np.eye(n)).max() < 1e-13
    assert np.abs(Q @ R - M).max() < 1e-13 * np.abs(M).max() * np.sqrt(m)
    assert np.abs(np.tril(R, -1)).max() == 0
    Qn, Rn = np.linalg.qr(M)
    assert np.abs(R - Rn).max() < 1e-12 * np.abs(Rn).max()
    assert np.abs(Q - Qn).max() < 1e-12


def test_qr_zero_and_deficient_columns():
    """Columns with no remaining norm are not reflected: Q column k is
    H_1 ... H_{k-1} e_k, orthonormal to the rest, and Q R still equals M."""
    rng = np.random.default_rng(5)
    M = np.zeros((6, 4), np.complex128)
    Q, R = fit.householder_qr(M)
    assert np.abs(Q - np.eye(6)[:, :4]).max() == 0
    M = crandn(rng, 8, 5)
    M[:, 2] = 0
    M[:, 4] = 2.0 * M[:, 0] - 1j * M[:, 1]            # exactly dependent (up to rounding)
    Q, R = fit.householder_qr(M)
    assert np.abs(Q.conj().T @ Q - np.eye(5)).max() < 1e-13
    assert np.abs(Q @ R - M).max() < 1e-12 * np.abs(M).max()
    # the dependent column is deflated: its diagonal entry of R vanishes to rounding
    assert abs(R[4, 4]) < 1e-12 and abs(R[2, 2]) == 0


# ----------------------------------------------------------------------------
# observables and overlaps against dense vectors
# ----------------------------------------------------------------------------

def test_measure_and_overlap_against_dense():
    L, d, D = 7, 2, 5
    a = wl.random_mps(L, d, D, seed=1)
    b = wl.random_mps(L, d, D, seed=2)
    va, vb = fit.to_dense(a), fit.to_dense(b)
    ops = list(wl.pauli())
    got = fit.measure_local(a, ops)
    ref = dense.expect_dense(va, ops, L)
    assert np.abs(got - ref).max() < 1e-13
    la, ph = fit.overlap(a, b)
    z = np.vdot(va, vb)
    assert abs(la - np.log(abs(z))) < 1e-12
    assert abs(np.angle(np.exp(1j * (ph - np.angle(z))))) < 1e-12


def test_measure_gauge_invariance():
    """Random invertible gauges on every bond leave <O_i> unchanged."""
    L, d, D = 8, 2, 6
    rng = np.random.default_rng(3)
    a = wl.random_mps(L, d, D, seed=3)
    b = [x.copy() for x in a]
    for i in range(L - 1):
        k = b[i].shape[2]
        G = crandn(rng, k, k) + 3 * np.eye(k)
        b[i] = np.tensordot(b[i], G, axes=([2], [0]))
        b[i + 1] = np.tensordot(np.linalg.inv(G), b[i + 1], axes=([1], [0]))
    ops = list(wl.pauli())
    assert np.abs(fit.measure_local(a, ops) - fit.measure_local(b, ops)).max() < 1e-12


def test_right_canonical_form():
    L, d, D = 9, 2, 8
    a = wl.random_mps(L, d, D, seed=4)
    r = fit.right_canonicalize(a)
    for i in range(1, L):
        A = r[i]
        G = np.einsum("asb,csb->ac", A, A.conj())
        assert np.abs(G - np.eye(A.shape[0])).max() < 1e-13
    va, vr = fit.to_dense(a), fit.to_dense(r)
    assert np.abs(va - vr).max() < 1e-13 * np.abs(va).max()


# ----------------------------------------------------------------------------
# the fit
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("model,N,state", [("tfi", 1, "up"), ("tfi", 3, "up"), ("xxz", 2, "neel"),
                                           ("lri", 3, "up")])
def test_fit_is_exact_when_bond_not_limiting(model, N, state):
    """With D >= d^(L/2) every bond holds the full space, so one sweep from the
    right-canonical guess reproduces W|psi> exactly: after k steps the MPS is
    W^k |psi_0> normalised, and the log-norm is log ||W^k psi_0||."""
    L = 8
    blocks = {"tfi": lambda: wl.tfi_blocks(L, 1.05), "xxz": lambda: wl.xxz_blocks(L, 0.5),
              "lri": lambda: wl.lr_ising_blocks(L, 0.7)}[model]()
    tau = -0.1j
    W = mpo.build_mpo(*blocks, N, tau)
    U = dense.mpo_to_dense(W)
    v0 = wl.product_state(state, L)
    psi = fit.product_mps(v0, 16)
    v = dense.product_vector(v0)
    logn = 0.0
    for k in range(6):
        psi, ln = fit.evolve_step(psi, W, sweeps=1, canonical=k > 0)
        logn += ln
        v = U @ v
        vm = fit.to_dense(psi)
        assert abs(np.linalg.norm(vm) - 1) < 1e-13
        assert abs(abs(np.vdot(vm, v)) / np.linalg.norm(v) - 1) < 1e-12
        assert abs(logn - np.log(np.linalg.norm(v))) < 1e-12


def test_tfi_first_order_against_exact_evolution():
    """The TFI workload (L = 12, g = 1.05, tau = -0.05i, 40 steps, first order):
    the error of <X_i>, <Z_i> against exp(tau H) is the MPO's method error
    (bounded by the error of the dense first-order operator) plus a truncation
    part that does not grow as D increases."""
    cfg = wl.config("tfi_L12")
    L = cfg["L"]
    blocks = wl.model_blocks(cfg)
    H = dense.hamiltonian_from_blocks(*blocks)
    E = dense.expm_tau_h(H, cfg["tau"])
    W = mpo.build_mpo(*blocks, cfg["N"], cfg["tau"])
    U = dense.mpo_to_dense(W)
    X, _, Z = wl.pauli()
    v0 = wl.initial_vectors(cfg)
    v_ex = dense.product_vector(v0)
    v_mpo = v_ex.copy()
    for _ in range(cfg["steps"]):
        v_ex = E @ v_ex
        v_mpo = U @ v_mpo
    ref = dense.expect_dense(v_ex, [X, Z], L).real
    method = np.abs(dense.expect_dense(v_mpo, [X, Z], L).real - ref).max()
    errs = []
    for Dc in (8, 16, 64):
        psi = fit.product_mps(v0, Dc)
        psi, _, _ = fit.evolve(psi, W, cfg["steps"], sweeps=1)
        errs.append(np.abs(fit.measure_local(psi, [X, Z]).real - ref).max())
    assert 1e-4 < method < 3e-3
    assert abs(errs[-1] - method) < 1e-10          # D = 64: no truncation, only method error
    assert errs[0] >= errs[1] - 1e-12 >= errs[2] - 2e-12


def test_norm_drift_order():
    """For anti-Hermitian tau H the order-N MPO is unitary up to O(tau^(N+1)): the
    log-norm per step shrinks by about 2^(N+1) when tau halves."""
    L = 8
    blocks = wl.xxz_blocks(L, 0.5)
    v0 = wl.product_state("neel", L)
    for N in (1, 2):
        drift = []
        for t in (0.2, 0.1):
            W = mpo.build_mpo(*blocks, N, -1j * t)
            psi = fit.product_mps(v0, 16)
            _, logn, _ = fit.evolve(psi, W, 4, sweeps=1)
            drift.append(abs(logn) / 4)
        assert np.log2(drift[0] / drift[1]) > N + 1 - 0.5


def _reflect_dense(M, L, d):
    """Matrix of the chain operator with the site order reversed."""
    t = M.reshape((d,) * (2 * L))
    perm = list(range(L - 1, -1, -1)) + list(range(2 * L - 1, L - 1, -1))
    return t.transpose(perm).reshape(d ** L, d ** L)


def test_reflection_symmetry():
    """Algorithms 1 + 2 give an operator that commutes with reflecting a uniform
    chain, so a reflection-symmetric initial state keeps <O_i> = <O_{L+1-i}> when
    D does not truncate. The extension and the approximate compression treat
    rows and columns differently, so for the full pipeline the reflected operator
    differs at order tau^(N+1) only."""
    L, N = 6, 3
    blocks = wl.lr_ising_blocks(L, 0.7)
    for variant, sym_exact in ((mpo.EXACT, True), (mpo.FULL, False)):
        asym = []
        for t in (0.2, 0.1):
            M = dense.mpo_to_dense(mpo.build_mpo(*blocks, N, -1j * t, variant))
            asym.append(np.abs(M - _reflect_dense(M, L, 2)).max())
        if sym_exact:
            assert asym[0] < 1e-14
        else:
            assert asym[0] > 1e-8 and np.log2(asym[0] / asym[1]) > N + 1 - 0.25
    L = 10
    blocks = wl.lr_ising_blocks(L, 0.7)
    W = mpo.build_mpo(*blocks, N, -0.2j, mpo.EXACT)
    psi = fit.product_mps(wl.product_state("up", L), 32)
    psi, _, _ = fit.evolve(psi, W, 5, sweeps=1)
    obs = fit.measure_local(psi, list(wl.pauli())).real
    assert np.abs(obs - obs[:, ::-1]).max() < 1e-12


def test_expm_by_eigh_matches_scipy():
    blocks = wl.xxz_blocks(6, 0.5)
    H = dense.hamiltonian_from_blocks(*blocks)
    tau = -0.3j
    assert np.abs(dense.expm_tau_h(H, tau) - scipy.linalg.expm(tau * H)).max() < 1e-12


def test_dense_hamiltonians_from_model_definitions():
    """The finite-state expansion of Sec. 2.3 equals Kronecker sums written from
    the model definitions (TFI, XXZ with bond couplings, long-range Ising, spin 1)."""
    X, Y, Z = wl.pauli()
    L = 6
    op = lambda o, i: dense.local_op(o, i, L)
    H = dense.hamiltonian_from_blocks(*wl.tfi_blocks(L, 1.05))
    ref = sum(-op(Z, i) @ op(Z, i + 1) for i in range(L - 1)) + sum(-1.05 * op(X, i) for i in range(L))
    assert np.abs(H - ref).max() < 1e-13
    J = np.array([0.6, 1.4, 0.9, 1.2, 0.7])
    H = dense.hamiltonian_from_blocks(*wl.xxz_blocks(L, 0.5, J))
    ref = sum(J[i] / 4 * (op(X, i) @ op(X, i + 1) + op(Y, i) @ op(Y, i + 1) + 0.5 * op(Z, i) @ op(Z, i + 1))
              for i in range(L - 1))
    assert np.abs(H - ref).max() < 1e-13
    H = dense.hamiltonian_from_blocks(*wl.lr_ising_blocks(L, 0.7))
    Jr = lambda r: np.sum(wl.LR_A * wl.LR_B ** r)
    ref = sum(-Jr(j - i) * op(Z, i) @ op(Z, j) for i in range(L) for j in range(i + 1, L)) + \
        sum(-0.7 * op(X, i) for i in range(L))
    assert np.abs(H - ref).max() < 1e-13
    Sx, Sy, Sz = wl.spin_one()
    L = 4
    op = lambda o, i: dense.local_op(o, i, L)
    H = dense.hamiltonian_from_blocks(*wl.spin1_blocks(L, 1.0, 0.3))
    ref = sum(op(Sx, i) @ op(Sx, i + 1) + op(Sy, i) @ op(Sy, i + 1) + op(Sz, i) @ op(Sz, i + 1)
              for i in range(L - 1)) + sum(0.3 * op(Sz @ Sz, i) for i in range(L))
    assert np.abs(H - ref).max() < 1e-13


def test_cylinder_hamiltonian_from_definition():
    """The 2-D TFI cylinder with spiral boundary conditions (Sec. 2.4): the MPO's
    expansion equals -sum (Z_i Z_{i+1} + Z_i Z_{i+W}) - g sum X_i written as
    Kronecker products, and the order-N MPO's bond follows the Sec. 8.3 table
    with chi = W."""
    Lx, Wc, g = 2, 4, 3.5
    L = Lx * Wc
    blocks = wl.tfi_cylinder_blocks(Lx, Wc, g)
    H = dense.hamiltonian_from_blocks(*blocks)
    X, _, Z = wl.pauli()
    ref = np.zeros_like(H)
    for i in range(L):
        ref -= g * dense.local_op(X, i, L)
        for r in (1, Wc):
            if i + r < L:
                ref -= dense.local_op(Z, i, L) @ dense.local_op(Z, i + r, L)
    assert np.abs(H - ref).max() == 0.0
    small = blocks
    for N, w in ((1, 1 + Wc), (2, 1 + Wc + Wc ** 2), (3, 1 + 3 * Wc + Wc ** 2 + Wc ** 3)):
        W = mpo.build_mpo(*small, N, -0.1j)
        assert max(x.shape[0] for x in W) == w


def test_two_site_fit_exact_when_bonds_do_not_limit():
    """Two-site fit (Sec. 2.2, the (i)DMRG row in its two-site form): from the Neel
    product state with D = 16 = 2^(L/2), every step reproduces the dense
    W|psi> (normalised) exactly, with no completion rule for the rank-deficient
    start: each bond's basis comes from the SVD of the two-site target."""
    L = 8
    blocks = wl.xxz_blocks(L, 0.5)
    W = mpo.build_mpo(*blocks, 2, -0.2j)
    U = dense.mpo_to_dense(W)
    v = dense.product_vector(wl.product_state("neel", L))
    psi = fit.product_mps(wl.product_state("neel", L), 16)
    for k in range(4):
        psi, _ = fit.evolve_step_two_site(psi, W, 1, canonical=k > 0)
        v = U @ v
        assert abs(abs(np.vdot(v / np.linalg.norm(v), fit.to_dense(psi))) - 1) < 1e-12


def test_two_site_fit_beats_svd_truncation_and_single_site():
    """Truncating regime (TFI L = 10, D = 6, one step of the order-2 MPO at
    tau = -0.3i from a seeded random right-canonical state): the two-site fit's
    infidelity with the exact target after one sweep is at most that of the
    target's sequential SVD truncation to the same bonds (the variational
    optimum is no worse than that compression), and at most the single-site
    fit's after one sweep."""
    L = 10
    blocks = wl.tfi_blocks(L, 1.05)
    W = mpo.build_mpo(*blocks, 2, -0.3j)
    psi0 = fit.right_canonicalize(wl.random_mps(L, 2, 6, seed=3))
    t = dense.mpo_to_dense(W) @ fit.to_dense(psi0)
    t /= np.linalg.norm(t)

    def infid(ph):
        x = fit.to_dense(ph)
        return 1 - abs(np.vdot(t, x)) / np.linalg.norm(x)

    out, rest, chi = [], t.reshape(1, -1), 1
    for i in range(L - 1):
        Us, S, Vh = np.linalg.svd(rest.reshape(chi * 2, -1), full_matrices=False)
        k = min(6, len(S))
        out.append(Us[:, :k].reshape(chi, 2, k))
        rest, chi = S[:k, None] * Vh[:k], k
    out.append(rest.reshape(chi, 2, 1))
    two, _ = fit.evolve_step_two_site(psi0, W, 1, canonical=True)
    one, _ = fit.evolve_step(psi0, W, 1, canonical=True)
    assert infid(two) <= infid(out) + 1e-12
    assert infid(two) <= infid(one) + 1e-12
    assert infid(out) > 1e-3          # the bond really truncates
