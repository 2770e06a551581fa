"""Pins for the oracle's MPO construction (oracle/mpo.py) against what the paper
prints and what the mathematics fixes. CPU only."""
import itertools
import math

import numpy as np
import pytest

import workloads as wl
from oracle import dense, mpo


def sym(*ops):
    """{X Y Z}: sum over the distinct orderings of the multiset of operators
    (Sec. 5 footnote: {BD} = BD + DB, {ABB} = ABB + BAB + BBA)."""
    ids = [id(o) for o in ops]
    seen, out = set(), 0
    for perm in itertools.permutations(range(len(ops))):
        key = tuple(ids[p] for p in perm)
        if key in seen:
            continue
        seen.add(key)
        m = np.eye(ops[0].shape[0], dtype=np.complex128)
        for p in perm:
            m = m @ ops[p]
        out = out + m
    return out


def prod(*ops):
    m = np.eye(ops[0].shape[0], dtype=np.complex128)
    for o in ops:
        m = m @ o
    return m


@pytest.fixture(params=[2, 3])
def scalar_blocks(request):
    d = request.param
    A, B, C, D = wl.random_blocks(1, 1, d, seed=11 + d)
    blk = (A[0], B[0], C[0], D[0])
    ops = (A[0][0, 0], B[0][0], C[0][0], D[0])
    return blk, ops


TAU = 0.37 - 0.21j


def entry(O, a, b, d):
    E = O.entries.get((a, b))
    return np.zeros((d, d), np.complex128) if E is None else E[0, 0]


def check_table(O, table, d, tol=1e-13):
    assert sorted(O.levels) == sorted(table)
    for a, row in table.items():
        for b, expect in row.items():
            got = entry(O, a, b, d)
            assert np.abs(got - expect).max() < tol * max(1.0, np.abs(expect).max()), (a, b)
    # everything not listed is zero
    for (a, b), E in O.entries.items():
        if b not in table[a]:
            assert np.abs(E).max() < tol, (a, b)


def test_eq_W1_first_order_plain(scalar_blocks):
    """Eq. W1 (Sec. 3): Algorithm 1 alone at N = 1 gives [[1 + tau D, C], [tau B, A]]."""
    blk, (A, B, C, D) = scalar_blocks
    d = D.shape[0]
    I = np.eye(d)
    O = mpo.build_level_mpo(blk, 1, TAU, mpo.PLAIN)
    check_table(O, {(1,): {(1,): I + TAU * D, (2,): C}, (2,): {(1,): TAU * B, (2,): A}}, d)


def test_eq_W2_second_order_plain(scalar_blocks):
    """Eq. W2 (Sec. 3): Algorithm 1 alone at N = 2, six levels."""
    blk, (A, B, C, D) = scalar_blocks
    d = D.shape[0]
    I = np.eye(d)
    t = TAU
    O = mpo.build_level_mpo(blk, 2, t, mpo.PLAIN)
    table = {
        (1, 1): {(1, 1): I + t * D + t ** 2 / 2 * D @ D, (1, 2): C, (2, 1): C, (2, 2): C @ C,
                 (2, 3): C @ D, (3, 2): D @ C},
        (1, 2): {(1, 1): t / 2 * B + t ** 2 / 2 * D @ B, (1, 2): A, (2, 2): C @ A, (2, 3): C @ B,
                 (3, 2): D @ A},
        (2, 1): {(1, 1): t / 2 * B + t ** 2 / 2 * B @ D, (2, 1): A, (2, 2): A @ C, (2, 3): A @ D,
                 (3, 2): B @ C},
        (2, 2): {(1, 1): t ** 2 / 2 * B @ B, (2, 2): A @ A, (2, 3): A @ B, (3, 2): B @ A},
        (2, 3): {(1, 1): t ** 2 / 2 * B, (2, 3): A},
        (3, 2): {(1, 1): t ** 2 / 2 * B, (3, 2): A},
    }
    check_table(O, table, d)


def test_exact_compression_second_order_table(scalar_blocks):
    """Sec. 4 worked result (after the basis change): four levels. The paper keeps
    (2,3) where Algorithm 2 keeps its copy-permutation twin (3,2)."""
    blk, (A, B, C, D) = scalar_blocks
    d = D.shape[0]
    I = np.eye(d)
    t = TAU
    O = mpo.build_level_mpo(blk, 2, t, mpo.EXACT)
    table = {
        (1, 1): {(1, 1): I + t * D + t ** 2 / 2 * D @ D, (1, 2): C, (2, 2): C @ C, (3, 2): C @ D + D @ C},
        (1, 2): {(1, 1): t * B + t ** 2 / 2 * (D @ B + B @ D), (1, 2): A, (2, 2): C @ A + A @ C,
                 (3, 2): C @ B + A @ D + D @ A + B @ C},
        (2, 2): {(1, 1): t ** 2 / 2 * B @ B, (2, 2): A @ A, (3, 2): A @ B + B @ A},
        (3, 2): {(1, 1): t ** 2 / 2 * B, (3, 2): A},
    }
    check_table(O, table, d)


def test_extension_second_order_table(scalar_blocks):
    """Sec. 5 worked result (extension + exact compression, N = 2). The printed
    tau/3 {CCD} in the (1,1) -> (2,3) entry reads tau/3 {CDD} (it must give the
    appendix's tau^2/6 {CDD} after Algorithm 4). The kept level is (3,2), whose
    row is the mirror of the paper's (2,3) row: its one non-symmetric product
    per term appears in reversed order."""
    blk, (A, B, C, D) = scalar_blocks
    d = D.shape[0]
    I = np.eye(d)
    t = TAU
    O = mpo.build_level_mpo(blk, 2, t, mpo.EXTENDED)
    table = {
        (1, 1): {(1, 1): I + t * D + t ** 2 / 2 * D @ D + t ** 3 / 6 * D @ D @ D, (1, 2): C,
                 (2, 2): C @ C + t / 3 * sym(C, C, D),
                 (3, 2): sym(C, D) + t / 3 * sym(C, D, D)},
        (1, 2): {(1, 1): t * B + t ** 2 / 2 * sym(D, B) + t ** 3 / 6 * sym(B, D, D), (1, 2): A,
                 (2, 2): sym(A, C) + t / 3 * (sym(A, C, D) + sym(B, C, C)),
                 (3, 2): sym(B, C) + sym(A, D) + t / 3 * (sym(B, C, D) + sym(A, D, D))},
        (2, 2): {(1, 1): t ** 2 / 2 * B @ B + t ** 3 / 6 * sym(B, B, D),
                 (2, 2): A @ A + t / 3 * (sym(A, B, C) + sym(A, A, D)),
                 (3, 2): sym(A, B) + t / 3 * (sym(A, B, D) + sym(B, B, C))},
        (3, 2): {(1, 1): t ** 2 / 2 * B + t ** 3 / 6 * (sym(B, D) + D @ B),
                 (2, 2): t / 3 * (sym(A, C) + C @ A),
                 (3, 2): A + t / 3 * (sym(A, D) + D @ A + sym(B, C) + C @ B)},
    }
    check_table(O, table, d)


def test_appendix_first_order(scalar_blocks):
    """Appendix: optimal first-order MPO (full pipeline at N = 1)."""
    blk, (A, B, C, D) = scalar_blocks
    d = D.shape[0]
    I = np.eye(d)
    t = TAU
    O = mpo.build_level_mpo(blk, 1, t, mpo.FULL)
    table = {
        (1,): {(1,): I + t * D + t ** 2 / 2 * D @ D, (2,): C + t / 2 * sym(C, D)},
        (2,): {(1,): t * B + t ** 2 / 2 * sym(B, D), (2,): A + t / 2 * (sym(A, D) + sym(B, C))},
    }
    check_table(O, table, d)


def test_appendix_second_order(scalar_blocks):
    """Appendix: optimal second-order MPO (full pipeline at N = 2), all nine entries."""
    blk, (A, B, C, D) = scalar_blocks
    d = D.shape[0]
    I = np.eye(d)
    t = TAU
    O = mpo.build_level_mpo(blk, 2, t, mpo.FULL)
    table = {
        (1, 1): {(1, 1): I + t * D + t ** 2 / 2 * D @ D + t ** 3 / 6 * D @ D @ D,
                 (1, 2): C + t / 2 * sym(C, D) + t ** 2 / 6 * sym(C, D, D),
                 (2, 2): C @ C + t / 3 * sym(C, C, D)},
        (1, 2): {(1, 1): t * B + t ** 2 / 2 * sym(B, D) + t ** 3 / 6 * sym(B, D, D),
                 (1, 2): A + t / 2 * (sym(B, C) + sym(A, D)) + t ** 2 / 6 * (sym(C, B, D) + sym(A, D, D)),
                 (2, 2): sym(A, C) + t / 3 * (sym(A, C, D) + sym(C, C, B))},
        (2, 2): {(1, 1): t ** 2 / 2 * B @ B + t ** 3 / 6 * sym(B, B, D),
                 (1, 2): t / 2 * sym(A, B) + t ** 2 / 6 * (sym(A, B, D) + sym(B, B, C)),
                 (2, 2): A @ A + t / 3 * (sym(A, B, C) + sym(A, A, D))},
    }
    check_table(O, table, d)


@pytest.mark.parametrize("chi", [1, 2, 3, 4])
def test_bond_dimension_table(chi):
    """Sec. 8.3 table: w = 1+chi, 1+chi+chi^2, 1+3chi+chi^2+chi^3,
    1+5chi+4chi^2+chi^3+chi^4 for N = 1..4 (full pipeline); after Algorithm 2
    alone the counts are 1+chi, 1+2chi+chi^2, 1+4chi+2chi^2+chi^3,
    1+6chi+5chi^2+2chi^3+chi^4 (same readings)."""
    A, B, C, D = wl.random_blocks(1, chi, 1, seed=chi)
    blk = (A[0], B[0], C[0], D[0])
    c = chi
    full = [1 + c, 1 + c + c ** 2, 1 + 3 * c + c ** 2 + c ** 3, 1 + 5 * c + 4 * c ** 2 + c ** 3 + c ** 4]
    exact = [1 + c, 1 + 2 * c + c ** 2, 1 + 4 * c + 2 * c ** 2 + c ** 3,
             1 + 6 * c + 5 * c ** 2 + 2 * c ** 3 + c ** 4]
    Ns = (1, 2, 3, 4) if chi <= 3 else (1, 2, 3)
    for N in Ns:
        assert mpo.bond_dimension(blk, N, mpo.FULL) == full[N - 1]
        assert mpo.bond_dimension(blk, N, mpo.EXACT) == exact[N - 1]


def _steps_mpo(blk, N, tau, steps):
    O = mpo.LevelMPO(blk, N)
    if "extend" in steps:
        O.extend(tau)
    O.fold(tau)
    if "exact" in steps:
        O.compress_exact()
    return O.dense()


def _chain(blk_dense, L):
    out = []
    for i in range(L):
        W = blk_dense
        if i == 0:
            W = W[0:1]
        if i == L - 1:
            W = W[..., 0:1]
        out.append(W)
    return out


@pytest.mark.parametrize("N,chi", [(2, 1), (2, 2), (3, 1), (3, 2)])
def test_exact_compression_is_exact(N, chi):
    """Sec. 4: Algorithm 2 applied to Algorithm 1's output changes no operator:
    the dense chain operator is the same before and after it. (After the
    extension step the rows of copy-permuted levels differ at order tau^(N+1),
    see the (2,3) row of the Sec. 5 table, so there the merge is only accurate
    to the order of the MPO; the order test below covers that case.)"""
    A, B, C, D = wl.random_blocks(1, chi, 2, seed=40 + N + chi)
    blk = (A[0], B[0], C[0], D[0])
    L = 5
    W0 = dense.mpo_to_dense(_chain(_steps_mpo(blk, N, TAU, ()), L))
    W1 = dense.mpo_to_dense(_chain(_steps_mpo(blk, N, TAU, ("exact",)), L))
    assert np.abs(W0 - W1).max() < 1e-12 * np.abs(W0).max()


@pytest.mark.parametrize("model", ["tfi", "xxz", "lri"])
def test_error_order(model):
    """Secs. 8.1-8.2: the order-N MPO approximates exp(tau H) with an error
    O(tau^(N+1)); every variant keeps the order and the full pipeline is no less
    accurate than exact compression alone."""
    L = 6
    if model == "tfi":
        blocks = wl.tfi_blocks(L, 1.05)
    elif model == "xxz":
        blocks = wl.xxz_blocks(L, 0.5)
    else:
        blocks = wl.lr_ising_blocks(L, 0.7)
    H = dense.hamiltonian_from_blocks(*blocks)
    taus = [0.2, 0.1, 0.05]
    for N in (1, 2, 3):
        for variant in (mpo.PLAIN, mpo.EXACT, mpo.EXTENDED, mpo.FULL):
            errs = []
            for t in taus:
                U = dense.mpo_to_dense(mpo.build_mpo(*blocks, N, -1j * t, variant))
                errs.append(np.linalg.norm(U - dense.expm_tau_h(H, -1j * t), 2))
            slope = np.log2(errs[1] / errs[2])
            assert slope > N + 1 - 0.25, (N, variant, errs)


def test_full_pipeline_not_worse_than_exact_only():
    """Sec. 8.1: the extended + approximately compressed MPO is more precise than
    the exact-only one at equal tau (spin-1 Heisenberg chain)."""
    L = 5
    blocks = wl.spin1_blocks(L, 1.0, 0.3)
    H = dense.hamiltonian_from_blocks(*blocks)
    for N in (1, 2, 3):
        for t in (0.1, 0.05):
            E = dense.expm_tau_h(H, -1j * t)
            e_full = np.linalg.norm(dense.mpo_to_dense(mpo.build_mpo(*blocks, N, -1j * t, mpo.FULL)) - E, 2)
            e_exact = np.linalg.norm(dense.mpo_to_dense(mpo.build_mpo(*blocks, N, -1j * t, mpo.EXACT)) - E, 2)
            assert e_full <= e_exact * 1.0001, (N, t, e_full, e_exact)


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_commuting_closed_form(N):
    """With B = C = 0 the chain is a product of single-site terms. The full
    pipeline gives, per site, sum_{k=0}^{N+1} tau^k D^k / k! (Algorithm 1's
    factors C(N,a) tau^a (N-a)!/N! = tau^a/a! plus the extension's
    tau^(N+1)/(N+1)!); Algorithm 1 alone gives the sum up to k = N."""
    d, L = 2, 4
    A, B, C, D = wl.random_blocks(L, 1, d, seed=70 + N)
    B[:] = 0
    C[:] = 0
    t = 0.3 + 0.1j
    for variant, kmax in ((mpo.FULL, N + 1), (mpo.PLAIN, N)):
        U = dense.mpo_to_dense(mpo.build_mpo(A, B, C, D, N, t, variant))
        site = sum(np.linalg.matrix_power(D[0], k) * t ** k / math.factorial(k) for k in range(kmax + 1))
        expect = np.ones((1, 1))
        for _ in range(L):
            expect = np.kron(expect, site)
        assert np.abs(U - expect).max() < 1e-13 * np.abs(expect).max()


def test_site_dependent_couplings_match_dense():
    """Per-site construction with bond-dependent couplings still approximates
    exp(tau H) to order N+1."""
    L = 6
    J = np.array([0.6, 1.4, 0.9, 1.2, 0.7])
    blocks = wl.xxz_blocks(L, 0.5, J)
    H = dense.hamiltonian_from_blocks(*blocks)
    errs = []
    for t in (0.1, 0.05):
        U = dense.mpo_to_dense(mpo.build_mpo(*blocks, 2, -1j * t))
        errs.append(np.linalg.norm(U - dense.expm_tau_h(H, -1j * t), 2))
    assert np.log2(errs[0] / errs[1]) > 2.75


@pytest.mark.parametrize("variant", [mpo.FULL, mpo.PLAIN])
def test_complex_step_splitting_is_second_order(variant):
    """Sec. 8.3: two first-order operators at the complex steps tau (1 + i)/2 and
    tau (1 - i)/2 compose to a second-order approximation of exp(tau H): the
    error falls by 2^3 when tau halves."""
    L = 6
    blocks = wl.xxz_blocks(L, 0.5)
    H = dense.hamiltonian_from_blocks(*blocks)
    errs = []
    for t in (0.2, 0.1, 0.05):
        tau = -1j * t
        U1 = dense.mpo_to_dense(mpo.build_mpo(*blocks, 1, tau * (1 + 1j) / 2, variant))
        U2 = dense.mpo_to_dense(mpo.build_mpo(*blocks, 1, tau * (1 - 1j) / 2, variant))
        errs.append(np.linalg.norm(U2 @ U1 - dense.expm_tau_h(H, tau), 2))
    assert np.log2(errs[0] / errs[1]) > 2.9 and np.log2(errs[1] / errs[2]) > 2.9
