"""Oracle: applying W^(N)(tau) to a finite MPS by a single-site variational fit.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper applies the MPO to the MPS and fits the product back into an MPS of
fixed bond dimension by minimising the 2-norm difference with a DMRG-like
sweeping scheme (Sec. 2.2 and Table 1, "(i)DMRG" row, cost O(w D^3)); in its
benchmark every time step is one such variational fit at fixed bond dimension
(Sec. 8.2). The paper does not spell out the sweep, so the following reading is
fixed here and shared, as a written specification, with the GPU path:

  * bonds D_i = min(D, d^i, d^(L-i)); a product state sits in index 0 of every
    bond, the rest zero;
  * a time step starts from phi = psi (right-canonical, built once by an LQ
    sweep if psi is not yet canonical) and the right environments of <phi|W|psi>;
  * one sweep = sites 1..L-1 moving right (QR, keep Q, drop R, grow the left
    environment) then sites L..2 moving left (the same step on the mirrored
    chain); after the last sweep the centre is recomputed at site 1;
  * the centre is normalised and log of its norm accumulated separately;
  * the mirrored chain reads A^T[r, s, l] = A[l, s, r] and W^T[r, s, s', l] =
    W[l, s, s', r], so the leftward step is the rightward step verbatim, and its
    "LQ" is the QR of the plain transpose of the centre;
  * Householder QR in the LAPACK convention (real beta = -sign(Re alpha)||x||,
    tau = (beta - alpha)/beta, v_1 = 1); a column whose remaining norm is at most
    2^-42 times the Frobenius norm of the matrix is not reflected (tau = 0), so
    completion directions of rank-deficient centres are fixed by the arithmetic,
    not by rounding noise.

Each contraction uses numpy matmul as its only library primitive.

Pins: tests/test_oracle_fit.py (QR against its definition and LAPACK's R up to
phases; exact fit against the dense product W|psi> when D is not limiting;
agreement with exp(tau H) within the MPO's error order; gauge invariance of
expectation values; reflection symmetry; overlaps against dense vectors).
"""
from __future__ import annotations

import numpy as np

DEFLATE = 2.0 ** -42


# ----------------------------------------------------------------------------
# Householder QR
# ----------------------------------------------------------------------------

def householder_qr(M, deflate=DEFLATE):
    """Thin QR of an m x n complex matrix (m >= n): returns Q (m x n, orthonormal
    columns) and R (n x n, upper triangular) with M = Q R.

    Column k: alpha = x[0], beta = -sign(Re alpha) ||x|| (sign(0) = +1),
    tau_k = (beta - alpha)/beta, v = x/(alpha - beta) with v[0] = 1, and the
    trailing block is updated by H_k^H = I - conj(tau_k) v v^H. Columns whose
    remaining norm is <= deflate * ||M||_F keep tau_k = 0 (H_k = I). Q is
    H_1 H_2 ... H_n applied to the first n columns of the identity."""
    M = np.array(M, dtype=np.complex128, copy=True)
    m, n = M.shape
    assert m >= n
    tol = deflate * np.sqrt(np.sum(np.abs(M) ** 2))
    taus = np.zeros(n, np.complex128)
    V = np.zeros((m, n), np.complex128)
    for k in range(n):
        x = M[k:, k]
        alpha = x[0]
        nrm = np.sqrt(np.sum(np.abs(x) ** 2))
        if nrm <= tol or nrm == 0.0:
            M[k + 1:, k] = 0
            continue
        beta = -nrm if alpha.real >= 0 else nrm
        t = (beta - alpha) / beta
        v = x / (alpha - beta)
        v[0] = 1.0
        taus[k] = t
        V[k:, k] = v
        # H^H applied to columns k..n-1
        blk = M[k:, k:]
        w = v.conj() @ blk
        M[k:, k:] = blk - np.conj(t) * np.outer(v, w)
        M[k, k] = beta
        M[k + 1:, k] = 0
    R = np.triu(M[:n, :n])
    Q = np.zeros((m, n), np.complex128)
    Q[:n, :n] = np.eye(n)
    for k in range(n - 1, -1, -1):
        if taus[k] == 0:
            continue
        v = V[k:, k]
        w = v.conj() @ Q[k:, :]
        Q[k:, :] -= taus[k] * np.outer(v, w)
    return Q, R


# ----------------------------------------------------------------------------
# contractions (numpy matmul as the primitive)
# ----------------------------------------------------------------------------

def mirror_site(A):
    """A^T[r, s, l] = A[l, s, r]."""
    return np.ascontiguousarray(A.transpose(2, 1, 0))


def mirror_mpo(W):
    """W^T[r, s, s', l] = W[l, s, s', r]."""
    return np.ascontiguousarray(W.transpose(3, 1, 2, 0))


def make_T(Lenv, A, W):
    """T[p, s, v, b] = sum_{a, w, s'} L[p, w, a] A[a, s', b] W[w, s, s', v].

    Lenv: [Dphi_l, w_l, Dpsi_l]; A: [Dpsi_l, d, Dpsi_r]; W: [w_l, d, d, w_r].
    Two steps: X = L . A over the ket bond, then X . W over (w_l, s')."""
    p, wl, a = Lenv.shape
    _, d, b = A.shape
    wr = W.shape[3]
    X = (Lenv.reshape(p * wl, a) @ A.reshape(a, d * b)).reshape(p, wl, d, b)
    # group (w_l, s') for the MPO contraction
    Xg = X.transpose(0, 3, 1, 2).reshape(p * b, wl * d)           # [(p b), (w s')]
    Wg = W.transpose(0, 2, 1, 3).reshape(wl * d, d * wr)          # [(w s'), (s v)]
    T = (Xg @ Wg).reshape(p, b, d, wr).transpose(0, 2, 3, 1)      # [p, s, v, b]
    return np.ascontiguousarray(T)


def apply_T(T, Renv):
    """B[p, s, q] = sum_{v, b} T[p, s, v, b] R[q, v, b]."""
    p, d, wr, b = T.shape
    q = Renv.shape[0]
    return (T.reshape(p * d, wr * b) @ Renv.reshape(q, wr * b).T).reshape(p, d, q)


def env_next(Q, T):
    """L'[q, v, b] = sum_{p, s} conj(Q[p, s, q]) T[p, s, v, b]."""
    p, d, q = Q.shape
    _, _, wr, b = T.shape
    return (Q.reshape(p * d, q).conj().T @ T.reshape(p * d, wr * b)).reshape(q, wr, b)


def env_from_site(Lenv, Phi, A, W):
    """Environment one site further right for <Phi|W|A>."""
    return env_next(Phi, make_T(Lenv, A, W))


# ----------------------------------------------------------------------------
# canonical forms and the fit
# ----------------------------------------------------------------------------

def right_canonicalize(tensors):
    """LQ sweep from site L to 2 on the mirrored chain: the transpose of site i,
    read as a (D_i d) x D_{i-1} matrix, is factored as Q R; site i becomes Q
    (mirrored back) and R^T is absorbed into the right bond of site i-1."""
    t = [x.copy() for x in tensors]
    L = len(t)
    for i in range(L - 1, 0, -1):
        Tm = mirror_site(t[i])                       # [Dr, d, Dl]
        r, d, l = Tm.shape
        Q, R = householder_qr(Tm.reshape(r * d, l))
        t[i] = mirror_site(Q.reshape(r, d, l))
        t[i - 1] = np.tensordot(t[i - 1], R, axes=([2], [1]))   # [.., .., k]
    return t


def product_mps(vectors, D):
    """Product state in index 0 of each bond, padded to D_i = min(D, d^i, d^(L-i))."""
    L, d = vectors.shape
    dims = [int(min(D, d ** min(i, 60), d ** min(L - i, 60))) for i in range(L + 1)]
    out = []
    for i in range(L):
        A = np.zeros((dims[i], d, dims[i + 1]), np.complex128)
        A[0, :, 0] = vectors[i]
        out.append(A)
    return out


def _step_right(Lenv, psi_i, W_i, Rnext):
    """One rightward site step: B = T R, B = Q R', new left environment from conj(Q)."""
    T = make_T(Lenv, psi_i, W_i)
    B = apply_T(T, Rnext)
    p, d, q = B.shape
    Q, _ = householder_qr(B.reshape(p * d, q))
    Q = Q.reshape(p, d, q)
    return Q, env_next(Q, T)


def evolve_step(psi, W, sweeps=1, canonical=False):
    """One time step |psi> -> W|psi> fitted at the bond dimensions of psi.

    Returns (phi, log_norm): phi right-canonical with its centre at site 1 and
    normalised; log_norm = log ||fitted W|psi>||."""
    L = len(psi)
    phi = [x.copy() for x in psi] if canonical else right_canonicalize(psi)
    one = np.ones((1, 1, 1), np.complex128)
    # right environments of <phi|W|psi>, built on the mirrored chain
    Renv = [None] * (L + 1)
    Renv[L] = one
    for i in range(L - 1, 0, -1):
        Renv[i] = env_from_site(Renv[i + 1], mirror_site(phi[i]), mirror_site(psi[i]), mirror_mpo(W[i]))
    Lenv = [None] * (L + 1)
    Lenv[0] = one
    for _ in range(sweeps):
        for i in range(0, L - 1):
            phi[i], Lenv[i + 1] = _step_right(Lenv[i], psi[i], W[i], Renv[i + 1])
        for i in range(L - 1, 0, -1):
            Qm, Renv[i] = _step_right(Renv[i + 1], mirror_site(psi[i]), mirror_mpo(W[i]), Lenv[i])
            phi[i] = mirror_site(Qm)
    # centre at site 1 (mirrored apply with the left boundary)
    Tm = make_T(Renv[1], mirror_site(psi[0]), mirror_mpo(W[0]))
    centre = mirror_site(apply_T(Tm, Lenv[0]))
    nrm = np.sqrt(np.sum(np.abs(centre) ** 2))
    phi[0] = centre / nrm
    return phi, float(np.log(nrm))


def two_site_theta(Lenv, A1, A2, W1, W2, Renv):
    """Theta[(p s), (q s')] = sum L[p,w,a] A1[a,t,b] A2[b,t',c] W1[w,s,t,v]
    W2[v,s',t',u] R[q,u,c]: the target W|psi> projected on the environments of
    two neighbouring sites. Returns (Theta as a (Dp d) x (Dq d) matrix, the
    left site's T of make_T, for the environment update)."""
    T = make_T(Lenv, A1, W1)                                     # [p, s, v, b]
    TR = make_T(Renv, mirror_site(A2), mirror_mpo(W2))           # [q, s', v, b]
    p, d, v, b = T.shape
    q = TR.shape[0]
    return T.reshape(p * d, v * b) @ TR.reshape(q * d, v * b).T, T


def _two_site_right(Lenv, A1, A2, W1, W2, Renv, k):
    """One rightward two-site update: the k leading left singular vectors of
    Theta become the left site (Q = U[:, :k], left-canonical) and the left
    environment grows through conj(Q)."""
    theta, T = two_site_theta(Lenv, A1, A2, W1, W2, Renv)
    U, _, _ = np.linalg.svd(theta, full_matrices=False)
    Q = U[:, :k].reshape(Lenv.shape[0], A1.shape[1], k)
    return Q, env_next(Q, T)


def evolve_step_two_site(psi, W, sweeps=1, canonical=False):
    """One time step |psi> -> W|psi> fitted by two-site updates at the bond
    dimensions of psi (the (i)DMRG row of Table 1 in its two-site form, Sec. 2.2).

    As evolve_step, but each update treats a pair of neighbouring sites: the
    target projected on their environments, Theta, is cut by its singular value
    decomposition (numpy.linalg.svd) and the leading D_i singular vectors become
    the site moving away from the pair's far side. The basis of every bond is
    chosen from the target's Schmidt decomposition on the pair, so a bond can
    take directions that the guess phi = psi does not contain (a rank-deficient
    start needs no completion rule). One sweep = pairs (1,2)..(L-1,L) moving
    right, then (L,L-1)..(2,1) moving left; the centre is then recomputed at
    site 1 and normalised as in evolve_step. Returns (phi, log_norm)."""
    L = len(psi)
    phi = [x.copy() for x in psi] if canonical else right_canonicalize(psi)
    one = np.ones((1, 1, 1), np.complex128)
    Renv = [None] * (L + 1)
    Renv[L] = one
    for i in range(L - 1, 0, -1):
        Renv[i] = env_from_site(Renv[i + 1], mirror_site(phi[i]), mirror_site(psi[i]), mirror_mpo(W[i]))
    Lenv = [None] * (L + 1)
    Lenv[0] = one
    for _ in range(sweeps):
        for i in range(0, L - 1):
            k = psi[i].shape[2]
            phi[i], Lenv[i + 1] = _two_site_right(Lenv[i], psi[i], psi[i + 1], W[i], W[i + 1], Renv[i + 2], k)
        for i in range(L - 1, 0, -1):
            k = psi[i].shape[0]
            Qm, Renv[i] = _two_site_right(Renv[i + 1], mirror_site(psi[i]), mirror_site(psi[i - 1]),
                                          mirror_mpo(W[i]), mirror_mpo(W[i - 1]), Lenv[i - 1], k)
            phi[i] = mirror_site(Qm)
    Tm = make_T(Renv[1], mirror_site(psi[0]), mirror_mpo(W[0]))
    centre = mirror_site(apply_T(Tm, Lenv[0]))
    nrm = np.sqrt(np.sum(np.abs(centre) ** 2))
    phi[0] = centre / nrm
    return phi, float(np.log(nrm))


def evolve(psi, W, steps, sweeps=1, canonical=False, observe=None):
    """Repeated time steps; returns (psi, total log norm, [observe(psi) per step])."""
    logn = 0.0
    rec = []
    for k in range(steps):
        psi, ln = evolve_step(psi, W, sweeps, canonical=canonical)
        canonical = True
        logn += ln
        if observe is not None:
            rec.append(observe(psi))
    return psi, logn, rec


# ----------------------------------------------------------------------------
# observables
# ----------------------------------------------------------------------------

def transfer_left(E, A, B):
    """E'[a, b] = sum_{a0, b0, s} conj(A[a0, s, a]) E[a0, b0] B[b0, s, b]."""
    t = np.tensordot(E, B, axes=([1], [0]))                 # [a0, s, b]
    return np.tensordot(A.conj(), t, axes=([0, 1], [0, 1]))  # [a, b]


def measure_local(tensors, ops):
    """<O_i> = <phi|O_i|phi>/<phi|phi> for every site i and every d x d operator in
    ops; returns [len(ops), L] complex. General gauge: left and right transfer
    environments are both built."""
    L = len(tensors)
    El = [None] * (L + 1)
    El[0] = np.ones((1, 1), np.complex128)
    for i in range(L):
        El[i + 1] = transfer_left(El[i], tensors[i], tensors[i])
    Er = [None] * (L + 1)
    Er[L] = np.ones((1, 1), np.complex128)
    for i in range(L - 1, -1, -1):
        Er[i] = transfer_left(Er[i + 1], mirror_site(tensors[i]), mirror_site(tensors[i]))
    norm = El[L][0, 0].real
    out = np.zeros((len(ops), L), np.complex128)
    for i in range(L):
        A = tensors[i]
        for k, O in enumerate(ops):
            OA = np.einsum("st,atb->asb", O, A)
            M = np.tensordot(El[i], OA, axes=([1], [0]))            # [a, s, b]
            M = np.tensordot(A.conj(), M, axes=([0, 1], [0, 1]))     # [b', b]
            out[k, i] = np.sum(M * Er[i + 1]) / norm
    return out


def overlap(a, b):
    """<a|b> as (log|z|, arg z), rescaling the transfer matrix at every site."""
    E = np.ones((1, 1), np.complex128)
    logs = 0.0
    for A, B in zip(a, b):
        E = transfer_left(E, A, B)
        s = np.sqrt(np.sum(np.abs(E) ** 2))
        if s == 0:
            return -np.inf, 0.0
        E = E / s
        logs += np.log(s)
    z = E[0, 0]
    return float(logs + np.log(abs(z))), float(np.angle(z))


def to_dense(tensors):
    """Contract an MPS into its d^L state vector (small chains only)."""
    v = tensors[0].reshape(-1, tensors[0].shape[2])
    for A in tensors[1:]:
        v = (v @ A.reshape(A.shape[0], -1)).reshape(-1, A.shape[2])
    return v.reshape(-1)
