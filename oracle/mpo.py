"""Oracle: order-N time-evolution MPO W^(N)(tau) from a first-degree Hamiltonian MPO.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Follows arXiv:2302.14181:
  * Sec. 2.3, Eq. jordan_mpo: H ~ [[1, C, D], [0, A, B], [0, 0, 1]] with levels
    1 ("not yet acted"), 2 ("acting", dimension chi), 3 ("done").
  * Sec. 2.5, Eq. Hsq: H^M as a sparse block MPO whose levels are M-tuples over
    {1, 2, 3}; an entry is the operator product on the physical legs (copy 1
    leftmost) and the direct product on the virtual legs.
  * Algorithm 3 (Sec. 5): extension of H^N by the (N+1)-th power.
  * Algorithm 1 (Sec. 3): fold the columns of the pure {1,3} levels into (1,...,1).
  * Algorithm 2 (Sec. 4): exact compression of copy-permutation-equivalent levels.
  * Algorithm 4 (Sec. 6): approximate compression of the levels without a 1.
  * Eq. boundary (Sec. 3): finite-chain boundaries select level (1,...,1).

Readings of the paper taken here:
  * Algorithm 3 loops over the columns b with **no** 1 (the printed "1 in b"
    double counts the (1,1) entry at N = 1; "1 not in b" reproduces both tables
    of the appendix entry by entry).
  * "Sort the 1's (3's) to the front" in Algorithm 2 is a stable partition: the
    relative order of the other entries is kept (a full sort contradicts the
    bond-dimension table of Sec. 8.3 at N = 3).
  * Algorithm 4 removes the levels with no 1 and at least one 3; its factor uses
    the number of 3s.
  * Pipeline order: H^N -> Alg. 3 -> Alg. 1 -> Alg. 2 -> Alg. 4.

Pins: tests/test_oracle_mpo.py (appendix closed forms, Eqs. W1 and W2, the
N = 2 worked tables, the bond-dimension table, exactness of Alg. 2, the
commuting closed form, error order tau^(N+1) against exp(tau H)).
"""
from __future__ import annotations

import itertools
import math

import numpy as np

# variants of the construction
PLAIN = 0      # Algorithm 1 only
EXACT = 1      # Algorithms 1 + 2
EXTENDED = 2   # Algorithms 3 + 1 + 2
FULL = 3       # Algorithms 3 + 1 + 2 + 4 (the paper's recommended MPO)


def all_levels(M):
    """All M-tuples over {1, 2, 3} (the levels of H^M, Sec. 2.5)."""
    return list(itertools.product((1, 2, 3), repeat=M))


def copy_block(blk, x, y):
    """Single-copy block of Eq. jordan_mpo for the transition x -> y as a tensor
    [left virtual, right virtual, d_out, d_in]; None where the block is zero."""
    A, B, C, D = blk
    d = D.shape[0]
    if (x, y) in ((1, 1), (3, 3)):
        return np.eye(d, dtype=np.complex128)[None, None]
    if (x, y) == (1, 2):
        return C[None]                   # [1, chi, d, d]
    if (x, y) == (1, 3):
        return D[None, None]
    if (x, y) == (2, 2):
        return A                         # [chi, chi, d, d]
    if (x, y) == (2, 3):
        return B[:, None]                # [chi, 1, d, d]
    return None


def power_entry(blk, a, b):
    """Entry H^M[a, b] of the M-th power (Sec. 2.5): operator product over the
    copies in copy order, direct (Kronecker) product of the virtual legs with
    copy 1 most significant. Returns [chi^n2(a), chi^n2(b), d, d] or None."""
    P = None
    for x, y in zip(a, b):
        X = copy_block(blk, x, y)
        if X is None:
            return None
        if P is None:
            P = X.copy()
        else:
            d = P.shape[2]
            P = np.einsum("abij,cdjk->acbdik", P, X).reshape(
                P.shape[0] * X.shape[0], P.shape[1] * X.shape[1], d, d)
    return P


def _stable_front(c, v):
    """c with all entries equal to v moved to the front, the rest in order."""
    return tuple([x for x in c if x == v] + [x for x in c if x != v])


class LevelMPO:
    """An operator-valued block matrix over a set of levels: entries[(a, b)] is a
    tensor [vdim(a), vdim(b), d, d]; absent entries are zero."""

    def __init__(self, blk, N):
        self.blk, self.N = blk, N
        self.d = blk[3].shape[0]
        self.chi = blk[0].shape[0]
        self.levels = all_levels(N)
        self.entries = {}
        for a in self.levels:
            for b in self.levels:
                E = power_entry(blk, a, b)
                if E is not None:
                    self.entries[(a, b)] = E

    def vdim(self, a):
        return self.chi ** a.count(2)

    def add(self, a, b, E):
        if E is None:
            return
        if (a, b) in self.entries:
            self.entries[(a, b)] = self.entries[(a, b)] + E
        else:
            self.entries[(a, b)] = E.copy()

    def remove(self, c):
        self.levels.remove(c)
        for key in [k for k in self.entries if c in k]:
            del self.entries[key]

    # -- Algorithm 3 --------------------------------------------------------
    def extend(self, tau):
        """O[a, b] += tau N!/((N+1)! n1(a_e) n3(b_e)) H^{N+1}[a_e, b_e], summed over the
        insertion positions of a 1 into a and of a 3 into b; rows a with a 3 but
        no 2 are skipped, columns b range over the levels without a 1."""
        N = self.N
        updates = []
        for a in self.levels:
            if 2 not in a and 3 in a:
                continue
            for b in self.levels:
                if 1 in b:
                    continue
                acc = None
                for c in range(N + 1):
                    ae = a[:c] + (1,) + a[c:]
                    for dpos in range(N + 1):
                        be = b[:dpos] + (3,) + b[dpos:]
                        E = power_entry(self.blk, ae, be)
                        if E is None:
                            continue
                        coef = tau * math.factorial(N) / (
                            math.factorial(N + 1) * ae.count(1) * be.count(3))
                        acc = coef * E if acc is None else acc + coef * E
                if acc is not None:
                    updates.append((a, b, acc))
        for a, b, E in updates:
            self.add(a, b, E)

    # -- Algorithm 1 --------------------------------------------------------
    def fold(self, tau):
        """For a = 1..N and every arrangement b of a threes and N-a ones: add
        tau^a (N-a)!/N! times column b to column (1,...,1), then delete level b."""
        N = self.N
        one = (1,) * N
        for a in range(1, N + 1):
            coef = tau ** a * math.factorial(N - a) / math.factorial(N)
            perms = sorted(set(itertools.permutations((3,) * a + (1,) * (N - a))))
            for b in perms:
                for r in list(self.levels):
                    if (r, b) in self.entries:
                        self.add(r, one, coef * self.entries[(r, b)])
                self.remove(b)

    # -- Algorithm 2 --------------------------------------------------------
    def compress_exact(self):
        """Merge rows c into s_c (1s moved to the front) when n3 <= n1, and
        columns c into s_r (3s moved to the front) when n3 > n1."""
        for c in list(self.levels):
            if c not in self.levels:
                continue
            n1, n3 = c.count(1), c.count(3)
            sc, sr = _stable_front(c, 1), _stable_front(c, 3)
            if n3 <= n1 and sc != c:
                for b in list(self.levels):
                    if (c, b) in self.entries:
                        self.add(sc, b, self.entries[(c, b)])
                self.remove(c)
            elif n3 > n1 and sr != c:
                for r in list(self.levels):
                    if (r, c) in self.entries:
                        self.add(r, sr, self.entries[(r, c)])
                self.remove(c)

    # -- Algorithm 4 --------------------------------------------------------
    def compress_approx(self, tau):
        """For every level a with no 1 and at least one 3: add tau^n3 (N-n3)!/N!
        times column a to column b (a with its 3s replaced by 1s), delete a."""
        N = self.N
        for a in list(self.levels):
            if 1 in a or 3 not in a:
                continue
            n3 = a.count(3)
            b = tuple(1 if x == 3 else x for x in a)
            coef = tau ** n3 * math.factorial(N - n3) / math.factorial(N)
            for r in list(self.levels):
                if (r, a) in self.entries:
                    self.add(r, b, coef * self.entries[(r, a)])
            self.remove(a)

    # -- dense form ---------------------------------------------------------
    def ordered_levels(self):
        one = (1,) * self.N
        return [one] + sorted(l for l in self.levels if l != one)

    def dense(self):
        """W[w_l, s, s', w_r] with level (1,...,1) at index 0."""
        lv = self.ordered_levels()
        off, w = {}, 0
        for l in lv:
            off[l] = w
            w += self.vdim(l)
        W = np.zeros((w, self.d, self.d, w), np.complex128)
        for (a, b), E in self.entries.items():
            W[off[a]:off[a] + E.shape[0], :, :, off[b]:off[b] + E.shape[1]] = E.transpose(0, 2, 3, 1)
        return W


def build_level_mpo(blk, N, tau, variant=FULL):
    """Run the construction on one site's blocks; returns the LevelMPO."""
    O = LevelMPO(blk, N)
    if variant in (EXTENDED, FULL):
        O.extend(tau)
    O.fold(tau)
    if variant in (EXACT, EXTENDED, FULL):
        O.compress_exact()
    if variant == FULL:
        O.compress_approx(tau)
    return O


def site_blocks(A, B, C, D, i):
    return (A[i], B[i], C[i], D[i])


def build_mpo(A, B, C, D, N, tau, variant=FULL):
    """Per-site dense W_i[w_l, s, s', w_r] for a finite chain of L = len(D) sites.
    The first site keeps only the row of level (1,...,1), the last site only its
    column (Eq. boundary). Sites with identical blocks share one construction."""
    L = D.shape[0]
    cache = {}
    out = []
    for i in range(L):
        blk = site_blocks(A, B, C, D, i)
        key = b"".join(np.ascontiguousarray(x).tobytes() for x in blk)
        if key not in cache:
            cache[key] = build_level_mpo(blk, N, tau, variant).dense()
        W = cache[key]
        if i == 0:
            W = W[0:1]
        if i == L - 1:
            W = W[..., 0:1]
        out.append(np.ascontiguousarray(W))
    return out


def bond_dimension(blk, N, variant=FULL, tau=0.1):
    O = build_level_mpo(blk, N, tau, variant)
    return sum(O.vdim(l) for l in O.levels)
