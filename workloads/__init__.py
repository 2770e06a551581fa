"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds no arithmetic of the time-evolution method itself. It only
produces inputs:

* local operators (Pauli and spin matrices),
* the four blocks (A, B, C, D) of a Hamiltonian written as a first-degree MPO
  in the upper-triangular form of Sec. 2.3 (Eq. jordan_mpo),
* product initial states and random MPS tensors,
* the named workloads (chain model, length, bond caps, order, time step).

Block conventions (per site i, complex128, row-major):
    A[i] : [chi, chi, d, d]   middle-level block  (left virtual, right virtual, out, in)
    B[i] : [chi, d, d]        middle -> "done"    (left virtual, out, in)
    C[i] : [chi, d, d]        "not yet" -> middle (right virtual, out, in)
    D[i] : [d, d]             single-site term
so that H = sum_i (D_i + C_i B_{i+1} + C_i A_{i+1} B_{i+2} + ...), Sec. 2.3.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "pauli", "spin_half", "spin_one", "tfi_blocks", "xxz_blocks", "lr_ising_blocks",
    "spin1_blocks", "random_blocks", "product_state", "random_product_vectors",
    "random_mps", "bond_dims", "LR_A", "LR_B", "CONFIGS", "config", "batched_chains",
    "purify_blocks", "purify_op", "purified_infinite_temperature", "tfi_cylinder_blocks",
]

# ----------------------------------------------------------------------------
# local operators
# ----------------------------------------------------------------------------

def pauli():
    X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
    Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
    Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)
    return X, Y, Z


def spin_half():
    X, Y, Z = pauli()
    return X / 2, Y / 2, Z / 2


def spin_one():
    s2 = np.sqrt(2.0)
    Sx = np.array([[0, 1, 0], [1, 0, 1], [0, 1, 0]], dtype=np.complex128) / s2
    Sy = np.array([[0, -1j, 0], [1j, 0, -1j], [0, 1j, 0]], dtype=np.complex128) / s2
    Sz = np.diag([1.0, 0.0, -1.0]).astype(np.complex128)
    return Sx, Sy, Sz


def _stack(L, A, B, C, D):
    return (np.ascontiguousarray(np.broadcast_to(A, (L,) + A.shape)).copy(),
            np.ascontiguousarray(np.broadcast_to(B, (L,) + B.shape)).copy(),
            np.ascontiguousarray(np.broadcast_to(C, (L,) + C.shape)).copy(),
            np.ascontiguousarray(np.broadcast_to(D, (L,) + D.shape)).copy())


# ----------------------------------------------------------------------------
# Hamiltonian MPO blocks
# ----------------------------------------------------------------------------

def tfi_blocks(L, g, J=None):
    """H = -sum_i J_i Z_i Z_{i+1} - g sum_i X_i  (chi = 1, d = 2).

    J is a per-bond array of length L-1 (bond i couples sites i, i+1; the
    coupling is carried by the C block of site i); None means J_i = 1."""
    X, _, Z = pauli()
    Jb = np.ones(L) if J is None else np.concatenate([np.asarray(J, float), [0.0]])
    A = np.zeros((L, 1, 1, 2, 2), np.complex128)
    B = np.broadcast_to(Z, (L, 1, 2, 2)).copy()
    C = np.stack([(-Jb[i] * Z)[None] for i in range(L)])
    D = np.broadcast_to(-g * X, (L, 2, 2)).copy()
    return A, B, C, D


def xxz_blocks(L, Delta, J=None):
    """H = sum_i J_i (Sx Sx + Sy Sy + Delta Sz Sz)_{i,i+1}, S = sigma/2 (chi = 3, d = 2)."""
    Sx, Sy, Sz = spin_half()
    Jb = np.ones(L) if J is None else np.concatenate([np.asarray(J, float), [0.0]])
    A = np.zeros((L, 3, 3, 2, 2), np.complex128)
    B = np.broadcast_to(np.stack([Sx, Sy, Delta * Sz]), (L, 3, 2, 2)).copy()
    C = np.stack([Jb[i] * np.stack([Sx, Sy, Sz]) for i in range(L)])
    D = np.zeros((L, 2, 2), np.complex128)
    return A, B, C, D


# J(r) = sum_k LR_A[k] * LR_B[k]**r approximates 1/r^2 on r = 1..99. The decay
# rates were drawn once from numpy.random.default_rng(2302) (one uniform draw in
# each of [0.05,0.30], [0.30,0.55], [0.55,0.80], [0.80,0.95]) and the amplitudes
# solved by linear least squares of r*(J(r) - 1/r^2) over r = 1..99.
LR_A = np.array([4.511695931857767, -0.7457194772543838, 0.1316528565075884, 0.06041576711400206])
LR_B = np.array([0.25128989459017265, 0.3826022585551031, 0.6486240218124196, 0.8358200884077653])


def lr_ising_blocks(L, g, a=LR_A, b=LR_B):
    """H = -sum_{i<j} J(j-i) Z_i Z_j - g sum_i X_i, J(r) = sum_k a_k b_k^r (chi = len(a), d = 2).

    C_k = -a_k b_k Z, A = diag(b_k) (x) identity, B_k = Z, D = -g X (Sec. 2.4, long-range example)."""
    X, _, Z = pauli()
    chi = len(a)
    A1 = np.zeros((chi, chi, 2, 2), np.complex128)
    for k in range(chi):
        A1[k, k] = b[k] * np.eye(2)
    B1 = np.stack([Z] * chi)
    C1 = np.stack([-a[k] * b[k] * Z for k in range(chi)])
    return _stack(L, A1, B1, C1, -g * X)


def tfi_cylinder_blocks(Lx, Wc, g, J=1.0):
    """Transverse-field Ising model on a cylinder of circumference Wc and length
    Lx with spiral boundary conditions (Sec. 2.4, the 2-D example): the sites
    are numbered along a helix, i = 0 .. Wc Lx - 1, and site i couples to i + 1
    (around the cylinder) and to i + Wc (along it),
        H = -J sum_i (Z_i Z_{i+1} + Z_i Z_{i+Wc}) - g sum_i X_i
    (bonds that would leave the chain are absent). As an MPO the middle level is
    a shift register of Wc places (chi = Wc): C puts -J Z in place 0, A moves
    place k to k + 1, B closes a bond from place 0 (range 1) and from place
    Wc - 1 (range Wc)."""
    X, _, Z = pauli()
    L = Wc * Lx
    A1 = np.zeros((Wc, Wc, 2, 2), np.complex128)
    for k in range(Wc - 1):
        A1[k, k + 1] = np.eye(2)
    B1 = np.zeros((Wc, 2, 2), np.complex128)
    B1[0] = Z
    B1[Wc - 1] = B1[Wc - 1] + Z
    C1 = np.zeros((Wc, 2, 2), np.complex128)
    C1[0] = -J * Z
    return _stack(L, A1, B1, C1, -g * X)


def spin1_blocks(L, J=1.0, Dz=0.3):
    """H = J sum_i S_i . S_{i+1} + Dz sum_i (Sz_i)^2 for spin 1 (chi = 3, d = 3)."""
    Sx, Sy, Sz = spin_one()
    A1 = np.zeros((3, 3, 3, 3), np.complex128)
    B1 = J * np.stack([Sx, Sy, Sz])
    C1 = np.stack([Sx, Sy, Sz])
    return _stack(L, A1, B1, C1, Dz * (Sz @ Sz))


def random_blocks(L, chi, d, seed, scale=1.0, a_scale=0.5, uniform=True):
    """Seeded complex Gaussian blocks (for construction tests). A is scaled so its
    spectral radius stays below one."""
    rng = np.random.default_rng(seed)

    def cg(*shape):
        return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) * scale

    n = 1 if uniform else L
    A = cg(n, chi, chi, d, d) * a_scale / max(1.0, chi * d)
    B = cg(n, chi, d, d)
    C = cg(n, chi, d, d)
    D = cg(n, d, d)
    if uniform:
        return _stack(L, A[0], B[0], C[0], D[0])
    return A, B, C, D


def purify_op(O):
    """O acting on the physical leg of a (physical, ancilla) pair: O (x) 1."""
    return np.kron(O, np.eye(O.shape[-1], dtype=np.complex128))


def purify_blocks(A, B, C, D):
    """Hamiltonian blocks on the doubled site (physical (x) ancilla, dimension
    d^2): every operator entry O becomes O (x) 1, so the MPO acts on the
    physical legs only (the purification of a thermal state)."""
    def lift(X):
        d = X.shape[-1]
        out = np.zeros(X.shape[:-2] + (d * d, d * d), np.complex128)
        for idx in np.ndindex(*X.shape[:-2]):
            out[idx] = purify_op(X[idx])
        return out
    return lift(A), lift(B), lift(C), lift(D)


# ----------------------------------------------------------------------------
# states
# ----------------------------------------------------------------------------

def bond_dims(L, d, D):
    """D_i = min(D, d^i, d^(L-i)) for the bonds i = 0..L (D_0 = D_L = 1)."""
    out = []
    for i in range(L + 1):
        out.append(int(min(D, d ** min(i, 60), d ** min(L - i, 60))))
    return out


def product_state(kind, L, d=2):
    """Site vectors [L, d] of a product state: 'up' (all sites in basis state 0),
    'neel' (0,1,0,1,... starting with 0 on the first site)."""
    v = np.zeros((L, d), np.complex128)
    if kind == "up":
        v[:, 0] = 1
    elif kind == "neel":
        for i in range(L):
            v[i, i % 2] = 1
    else:
        raise ValueError(kind)
    return v


def purified_infinite_temperature(L, d):
    """Site vectors [L, d^2] of the product of maximally entangled
    (physical, ancilla) pairs sum_s |s>|s> / sqrt(d): tracing out the ancillas
    leaves the infinite-temperature state 1/d^L."""
    v = np.zeros((L, d * d), np.complex128)
    for s in range(d):
        v[:, s * d + s] = 1.0 / np.sqrt(d)
    return v


def random_product_vectors(L, d, seed):
    """Seeded i.i.d. complex Gaussian site vectors, each normalised."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((L, d)) + 1j * rng.standard_normal((L, d))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def random_mps(L, d, D, seed):
    """Seeded random complex MPS tensors [D_{i-1}, d, D_i] (not canonical)."""
    rng = np.random.default_rng(seed)
    dims = bond_dims(L, d, D)
    out = []
    for i in range(L):
        shp = (dims[i], d, dims[i + 1])
        out.append((rng.standard_normal(shp) + 1j * rng.standard_normal(shp)) / np.sqrt(dims[i] * d))
    return out


# ----------------------------------------------------------------------------
# named workloads (shapes of the paper's benchmark settings, Sec. 8)
# ----------------------------------------------------------------------------

CONFIGS = {
    # transverse-field Ising, first order, exact-diagonalisation size
    "tfi_L12": dict(model="tfi", L=12, d=2, chi=1, g=1.05, N=1, tau=-0.05j, D=16,
                    steps=40, sweeps=1, state="up"),
    # XXZ chain, orders 2 and 3
    "xxz_L64_N2": dict(model="xxz", L=64, d=2, chi=3, Delta=0.5, N=2, tau=-0.1j, D=128,
                       steps=50, sweeps=2, state="neel"),
    "xxz_L64_N3": dict(model="xxz", L=64, d=2, chi=3, Delta=0.5, N=3, tau=-0.2j, D=128,
                       steps=25, sweeps=2, state="neel"),
    # long-range Ising (sum of four exponentials), order 3, D = 256
    "lri_L100_N3_D256": dict(model="lri", L=100, d=2, chi=4, g=0.7, N=3, tau=-0.2j, D=256,
                             steps=25, sweeps=2, state="up"),
    # spin-1 Heisenberg with single-ion anisotropy, order 4
    "spin1_L128_N4_D512": dict(model="spin1", L=128, d=3, chi=3, Dz=0.3, N=4, tau=-0.25j, D=512,
                               steps=16, sweeps=2, state="random", seed=5),
}


def config(name, **override):
    c = dict(CONFIGS[name])
    c.update(override)
    return c


def model_blocks(cfg):
    m, L = cfg["model"], cfg["L"]
    if m == "tfi":
        return tfi_blocks(L, cfg["g"], cfg.get("J"))
    if m == "xxz":
        return xxz_blocks(L, cfg["Delta"], cfg.get("J"))
    if m == "lri":
        return lr_ising_blocks(L, cfg["g"])
    if m == "spin1":
        return spin1_blocks(L, 1.0, cfg["Dz"])
    raise ValueError(m)


def initial_vectors(cfg):
    if cfg["state"] == "random":
        return random_product_vectors(cfg["L"], cfg["d"], cfg.get("seed", 0))
    return product_state(cfg["state"], cfg["L"], cfg["d"])


def batched_chains(n=64, seed=64):
    """Independent chains of uneven size: model in {tfi, xxz}, one coupling per bond
    drawn from U[0.5, 1.5], L in [16, 80], D in {32, 64, 128}, N in {2, 3}, tau = -0.1i."""
    rng = np.random.default_rng(seed)
    out = []
    for c in range(n):
        model = ["tfi", "xxz"][int(rng.integers(2))]
        L = int(rng.integers(16, 81))
        D = int([32, 64, 128][int(rng.integers(3))])
        N = int(rng.integers(2, 4))
        J = rng.uniform(0.5, 1.5, L - 1)
        cfg = dict(model=model, L=L, d=2, chi=1 if model == "tfi" else 3, N=N, tau=-0.1j, D=D,
                   steps=10, sweeps=1, state="neel" if model == "xxz" else "up", J=J)
        if model == "tfi":
            cfg["g"] = 1.05
        else:
            cfg["Delta"] = 0.5
        out.append(cfg)
    return out
