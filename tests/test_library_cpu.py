"""CPU-side checks of the C ABI library: it loads, exports every symbol the
header declares, and its host MPO construction agrees with the oracle's.
No GPU call is made here."""
import ctypes

import numpy as np
import pytest

import workloads as wl
from oracle import dense, mpo

tv = pytest.importorskip("paper_2302_14181_gb300")


def test_exports_every_declared_symbol():
    declared = tv._lib.declared_symbols()
    assert len(declared) >= 20
    for name in declared:
        assert hasattr(tv._lib.lib, name), name


def test_strerror_names_codes():
    for code in range(0, -9, -1):
        assert tv._lib.lib.tevo_strerror(code)
        assert tv.tevo_strerror(code) == tv._lib.lib.tevo_strerror(code).decode()


def test_binding_carries_the_c_names_of_the_compute_entries():
    for name in ("mpo_build", "mpo_build_host", "mps_init", "evolve_step", "evolve_step_batched",
                 "measure_local", "mps_overlap", "tevo_gemm", "tevo_gemm_noalloc", "tevo_wait_selftest",
                 "tevo_strerror"):
        assert name in tv._lib.declared_symbols(), name
        assert callable(getattr(tv, name)), name


def test_gemm_binding_checks_operands_before_the_library():
    torch = pytest.importorskip("torch")
    z = torch.zeros((2, 3), dtype=torch.complex128)   # host memory: refused before any library call
    for f in (tv.tevo_gemm, tv.tevo_gemm_noalloc):
        with pytest.raises(TypeError):
            f(None, tv.FP64, z, z, z)
        with pytest.raises(TypeError):
            f(None, tv.FP64, np.zeros((2, 3), np.complex128), z, z)


MODELS = {
    "tfi": lambda L: wl.tfi_blocks(L, 1.05),
    "xxz": lambda L: wl.xxz_blocks(L, 0.5),
    "xxz_bonds": lambda L: wl.xxz_blocks(L, 0.5, np.linspace(0.5, 1.5, L - 1)),
    "lri": lambda L: wl.lr_ising_blocks(L, 0.7),
    "spin1": lambda L: wl.spin1_blocks(L, 1.0, 0.3),
    "random": lambda L: wl.random_blocks(L, 2, 2, seed=9, uniform=False),
}


@pytest.mark.parametrize("model", sorted(MODELS))
@pytest.mark.parametrize("N", [1, 2, 3])
@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_host_mpo_matches_oracle(model, N, variant):
    """The C++ construction and the oracle agree as chain operators (dense
    contraction on L = 4; level order inside a bond may differ) and in the
    bond dimensions."""
    L = 4
    blocks = MODELS[model](L)
    tau = 0.31 - 0.17j
    Wc = tv.mpo_build_host(*blocks, N, tau, variant)
    Wo = mpo.build_mpo(*blocks, N, tau, variant)
    assert [w.shape for w in Wc] == [w.shape for w in Wo]
    Mc, Mo = dense.mpo_to_dense(Wc), dense.mpo_to_dense(Wo)
    assert np.abs(Mc - Mo).max() < 1e-13 * max(1.0, np.abs(Mo).max())


@pytest.mark.parametrize("chi,N", [(1, 4), (3, 4), (4, 3), (2, 5)])
def test_host_mpo_bond_table(chi, N):
    """Bond dimensions of the Sec. 8.3 table (and their N = 5 continuation
    computed by the oracle) from the C++ construction."""
    A, B, C, D = wl.random_blocks(3, chi, 1, seed=chi)
    Wc = tv.mpo_build_host(A, B, C, D, N, 0.1)
    Wo = mpo.build_mpo(A, B, C, D, N, 0.1)
    assert Wc[1].shape == Wo[1].shape
    if N <= 4:
        c = chi
        table = [1 + c, 1 + c + c ** 2, 1 + 3 * c + c ** 2 + c ** 3, 1 + 5 * c + 4 * c ** 2 + c ** 3 + c ** 4]
        assert Wc[1].shape[0] == table[N - 1]


def test_host_mpo_rejects_bad_arguments():
    A, B, C, D = wl.tfi_blocks(4, 1.0)
    w = (ctypes.c_int * 5)()
    n = ctypes.c_size_t(0)
    p = lambda a: np.ascontiguousarray(a).ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    f = tv._lib.lib.mpo_build_host
    assert f(1, 2, 1, p(A), p(B), p(C), p(D), 1, 0.0, -0.1, 3, w, None, ctypes.byref(n)) == -1   # L < 2
    assert f(4, 2, 1, p(A), p(B), p(C), p(D), 0, 0.0, -0.1, 3, w, None, ctypes.byref(n)) == -1   # N < 1
    assert f(4, 2, 1, p(A), p(B), p(C), p(D), 2, 0.0, -0.1, 7, w, None, ctypes.byref(n)) == -1   # variant
    assert f(4, 2, 1, None, p(B), p(C), p(D), 2, 0.0, -0.1, 3, w, None, ctypes.byref(n)) == -1   # NULL
    assert f(4, 2, 1, p(A), p(B), p(C), p(D), 2, 0.0, -0.1, 3, w, None, ctypes.byref(n)) == 0
    small = np.zeros(1, np.complex128)
    assert f(4, 2, 1, p(A), p(B), p(C), p(D), 2, 0.0, -0.1, 3, w,
             small.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(ctypes.c_size_t(1))) == -1
