"""Oracle: dense references for small chains (L <= 12).

TEST INFRASTRUCTURE ONLY (see the package docstring).

  * ``hamiltonian_from_blocks`` writes out the finite-state expansion of Sec. 2.3,
    H = sum_i (D_i + C_i B_{i+1} + C_i A_{i+1} B_{i+2} + ...), term by term.
  * ``mpo_to_dense`` contracts per-site W_i[w_l, s, s', w_r] into a d^L x d^L
    matrix with the boundary vectors of Eq. boundary already sliced in.
  * ``expm_tau_h`` is exp(tau H) from numpy.linalg.eigh of the Hermitian H.
  * ``thermal_expect`` is the Gibbs average Tr(O_i e^{-beta H}) / Tr(e^{-beta H})
    of single-site operators, also from eigh (the finite-temperature states of
    Sec. 8.4, here on a finite chain).

Pins: tests/test_oracle_fit.py checks the expansion against Kronecker-sum
Hamiltonians written directly from the model definitions, and eigh against
scipy.linalg.expm; tests/test_oracle_thermal.py checks the Gibbs averages at
beta = 0 (Tr O / d), at large beta (the ground state's values) and against
scipy.linalg.expm.
"""
from __future__ import annotations

import numpy as np


def _kron_chain(ops):
    out = np.ones((1, 1), np.complex128)
    for o in ops:
        out = np.kron(out, o)
    return out


def hamiltonian_from_blocks(A, B, C, D):
    """Dense H of an L-site chain from its per-site blocks (Sec. 2.3 expansion).

    A term starting at site i and ending at site j > i is
        sum over the chi-paths  C_i[k0] A_{i+1}[k0,k1] ... A_{j-1}[.,k] B_j[k],
    with identities elsewhere; plus the on-site D_i."""
    L, d = D.shape[0], D.shape[1]
    I = np.eye(d, dtype=np.complex128)
    H = np.zeros((d ** L, d ** L), np.complex128)
    for i in range(L):
        H += _kron_chain([D[i] if k == i else I for k in range(L)])
    chi = C.shape[1]
    for i in range(L):
        # vector over chi of operator strings on sites i..j-1 (as lists of d x d)
        # represented as dense operators on sites i..cur
        partial = [C[i][k] for k in range(chi)]          # operators on site i
        for j in range(i + 1, L):
            # close the strings at site j with B_j
            term = np.zeros((d ** (j - i + 1), d ** (j - i + 1)), np.complex128)
            for k in range(chi):
                term += np.kron(partial[k], B[j][k])
            H += np.kron(np.kron(np.eye(d ** i), term), np.eye(d ** (L - j - 1)))
            # extend the strings through site j with A_j
            if j < L - 1:
                partial = [sum(np.kron(partial[k], A[j][k, k2]) for k in range(chi))
                           for k2 in range(chi)]
    return H


def mpo_to_dense(W):
    """Contract W_1 ... W_L (W_1 has w_l = 1, W_L has w_r = 1) into a matrix."""
    M = W[0][0]                                       # [s, s', w]
    d = M.shape[0]
    M = M.reshape(d, d, -1)
    for Wi in W[1:]:
        # M[S, S', w] x Wi[w, s, s', v] -> [S s, S' s', v]
        t = np.tensordot(M, Wi, axes=([2], [0]))       # [S, S', s, s', v]
        n = M.shape[0]
        M = t.transpose(0, 2, 1, 3, 4).reshape(n * d, n * d, -1)
    return M[:, :, 0]


def expm_tau_h(H, tau):
    """exp(tau H) for Hermitian H via its eigen-decomposition."""
    e, U = np.linalg.eigh(H)
    return (U * np.exp(tau * e)) @ U.conj().T


def product_vector(vectors):
    v = np.ones(1, np.complex128)
    for x in vectors:
        v = np.kron(v, x)
    return v


def local_op(op, i, L):
    d = op.shape[0]
    return np.kron(np.kron(np.eye(d ** i), op), np.eye(d ** (L - i - 1)))


def expect_dense(v, ops, L):
    """<v|O_i|v>/<v|v> for every operator and site; [len(ops), L]."""
    n = np.vdot(v, v)
    out = np.zeros((len(ops), L), np.complex128)
    for k, O in enumerate(ops):
        for i in range(L):
            out[k, i] = np.vdot(v, local_op(O, i, L) @ v) / n
    return out


def thermal_expect(H, beta, ops, L):
    """Tr(O_i e^{-beta H}) / Tr(e^{-beta H}) for every operator and site;
    [len(ops), L]. Eigenvalues are shifted by the smallest one before the
    exponential (the shift cancels in the ratio)."""
    e, U = np.linalg.eigh(H)
    w = np.exp(-beta * (e - e.min()))
    rho = (U * w) @ U.conj().T
    Z = np.trace(rho)
    out = np.zeros((len(ops), L), np.complex128)
    for k, O in enumerate(ops):
        for i in range(L):
            out[k, i] = np.trace(local_op(O, i, L) @ rho) / Z
    return out
