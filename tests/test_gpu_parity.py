"""GPU parity: the CUDA path through the C ABI against the fp64 oracle, element by
element on the same seeded inputs. Tolerances: fp64 form 1e-10 relative on
observables (max_i |o_i - o_i^ref| / max(max_i |o_i^ref|, 1e-3)); tensor-core
forms 1e-6 on the same measure."""
import numpy as np
import pytest

import workloads as wl
from oracle import fit, mpo

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)
tv = pytest.importorskip("paper_2302_14181_gb300")

FP64_TOL = 1e-10
MIXED_TOL = 1e-6


@pytest.fixture(scope="module")
def ctx():
    torch.cuda.set_device(0)
    return tv.Context()


def rel_err(got, ref):
    return float(np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-3))


def ops_for(d):
    return list(wl.pauli()) if d == 2 else list(wl.spin_one())


def run_both(ctx, blocks, v0, N, tau, D, steps, sweeps, precision=0, variant=mpo.FULL, check_every=True):
    ops = ops_for(v0.shape[1])
    Wo = mpo.build_mpo(*blocks, N, tau, variant)
    psi_o = fit.product_mps(v0, D)
    W = tv.mpo_build(ctx, *blocks, N, tau, variant)
    psi = tv.mps_init(ctx, v0, D)
    errs = []
    logn = 0.0
    for k in range(steps):
        psi_o, ln = fit.evolve_step(psi_o, Wo, sweeps, canonical=k > 0)
        logn += ln
        tv.evolve_step(psi, W, tau, D, sweeps, precision)
        if check_every or k == steps - 1:
            ref = fit.measure_local(psi_o, ops).real
            got = tv.measure_local(psi, ops).real
            errs.append(rel_err(got, ref))
    return errs, logn, psi.log_norm(), psi, psi_o


@pytest.mark.parametrize("case", [
    # (name, blocks, initial, N, tau, D, steps, sweeps)
    ("tfi_L12_N1", lambda: wl.tfi_blocks(12, 1.05), lambda: wl.product_state("up", 12), 1, -0.05j, 16, 8, 1),
    ("xxz_L16_N2", lambda: wl.xxz_blocks(16, 0.5), lambda: wl.product_state("neel", 16), 2, -0.2j, 16, 5, 2),
    ("xxz_L14_N3", lambda: wl.xxz_blocks(14, 0.5), lambda: wl.product_state("neel", 14), 3, -0.4j, 12, 4, 1),
    ("lri_L20_N3", lambda: wl.lr_ising_blocks(20, 0.7), lambda: wl.product_state("up", 20), 3, -0.2j, 24, 4, 2),
    ("spin1_L10_N2", lambda: wl.spin1_blocks(10, 1.0, 0.3), lambda: wl.random_product_vectors(10, 3, 5), 2,
     -0.25j, 20, 3, 2),
    ("bonds_L18_N2", lambda: wl.xxz_blocks(18, 0.5, np.linspace(0.5, 1.5, 17)),
     lambda: wl.product_state("neel", 18), 2, -0.1j, 20, 3, 1),
])
def test_fp64_matches_oracle(ctx, case):
    name, blocks, v0, N, tau, D, steps, sweeps = case
    errs, logn_o, logn_g, _, _ = run_both(ctx, blocks(), v0(), N, tau, D, steps, sweeps)
    assert max(errs) < FP64_TOL, (name, errs)
    assert abs(logn_o - logn_g) < 1e-10 * max(1.0, abs(logn_o)), (name, logn_o, logn_g)


@pytest.mark.parametrize("variant", [mpo.PLAIN, mpo.EXACT, mpo.EXTENDED])
def test_fp64_other_mpo_variants(ctx, variant):
    errs, lo, lg, _, _ = run_both(ctx, wl.xxz_blocks(12, 0.5), wl.product_state("neel", 12), 2, -0.1j, 16, 3, 1,
                                  variant=variant)
    assert max(errs) < FP64_TOL


def test_edge_minimal_chain(ctx):
    """L = 2 (one bond), D = 1 (product-state fit) and D larger than any bond."""
    for L, D in ((2, 1), (2, 4), (5, 1), (6, 100)):
        errs, lo, lg, _, _ = run_both(ctx, wl.tfi_blocks(L, 1.05), wl.product_state("up", L), 2, -0.1j, D, 3, 1)
        assert max(errs) < FP64_TOL, (L, D, errs)
        assert abs(lo - lg) < 1e-10


def test_non_canonical_start(ctx):
    """A random (non-canonical) state set site by site: the step first brings it to
    right-canonical form (LQ sweep) exactly as the oracle does."""
    L, D, N, tau = 9, 8, 2, -0.15j
    blocks = wl.xxz_blocks(L, 0.5)
    A = wl.random_mps(L, 2, D, seed=21)
    Wo = mpo.build_mpo(*blocks, N, tau)
    W = tv.mpo_build(ctx, *blocks, N, tau)
    psi = tv.mps_init(ctx, wl.product_state("up", L), D)
    for i, a in enumerate(A):
        psi.set_site(i, a)
    ops = ops_for(2)
    assert rel_err(tv.measure_local(psi, ops).real, fit.measure_local(A, ops).real) < FP64_TOL
    psi_o = A
    for k in range(3):
        psi_o, _ = fit.evolve_step(psi_o, Wo, 2, canonical=k > 0)
        tv.evolve_step(psi, W, tau, D, 2, tv.FP64)
        assert rel_err(tv.measure_local(psi, ops).real, fit.measure_local(psi_o, ops).real) < FP64_TOL


def assert_equal_up_to_bond_phases(got, ref, tol):
    """got_i = conj(P_i) ref_i P_(i+1) for diagonal phase matrices P_i on the
    bonds (the gauge freedom that leaves the state unchanged: a Householder
    column whose leading entry is zero in exact arithmetic takes its sign from
    rounding). The phases of bond i+1 are fitted column by column from site i,
    given those of bond i; the outer bonds carry the state's global phase."""
    p = np.ones(1, complex)
    for i, (a, b) in enumerate(zip(got, ref)):
        bl = np.conj(p)[:, None, None] * b
        c = np.einsum("lsr,lsr->r", np.conj(bl), a)
        q = np.where(np.abs(c) > 0, c / np.where(np.abs(c) > 0, np.abs(c), 1), 1)
        assert np.abs(a - bl * q[None, None, :]).max() < tol, i
        p = q


def test_tensors_right_canonical_and_close(ctx):
    """After a step the stored tensors are right-canonical (sites 2..L) and equal
    the oracle's tensors up to rounding (same Householder convention) and up to
    the phases of reflections whose sign rounding decides (a product-state
    start has exact zeros there)."""
    L, D = 10, 8
    blocks = wl.xxz_blocks(L, 0.5)
    _, _, _, psi, psi_o = run_both(ctx, blocks, wl.product_state("neel", L), 2, -0.2j, D, 2, 1)
    got = [psi.site(i) for i in range(L)]
    for i in range(1, L):
        G = np.einsum("asb,csb->ac", got[i], got[i].conj())
        assert np.abs(G - np.eye(got[i].shape[0])).max() < 1e-12
    assert_equal_up_to_bond_phases(got, psi_o, 1e-9)


def test_tensors_equal_the_oracle_from_a_generic_state(ctx):
    """From a random (entangled, full-rank) state every Householder sign is
    decided by a nonzero leading entry: after a step the tensors equal the
    oracle's up to rounding, with no phase freedom left."""
    L, D = 10, 8
    blocks = wl.xxz_blocks(L, 0.5)
    A = wl.random_mps(L, 2, D, seed=77)
    Wo = mpo.build_mpo(*blocks, 2, -0.2j)
    W = tv.mpo_build(ctx, *blocks, 2, -0.2j)
    psi = tv.mps_init(ctx, np.ones((L, 2)) / np.sqrt(2), D)
    for i in range(L):
        psi.set_site(i, A[i])
    psi_o = A
    for k in range(2):
        psi_o, _ = fit.evolve_step(psi_o, Wo, 2, canonical=k > 0)
        tv.evolve_step(psi, W, -0.2j, D, 2, tv.FP64)
    for i in range(L):
        assert np.abs(psi.site(i) - psi_o[i]).max() < 1e-9, i


def test_measure_and_overlap_random_states(ctx):
    L, D = 11, 7
    a = wl.random_mps(L, 2, D, seed=31)
    b = wl.random_mps(L, 2, D, seed=32)
    pa = tv.mps_init(ctx, wl.product_state("up", L), D)
    pb = tv.mps_init(ctx, wl.product_state("up", L), D)
    for i in range(L):
        pa.set_site(i, a[i])
        pb.set_site(i, b[i])
    ops = ops_for(2)
    assert rel_err(tv.measure_local(pa, ops), fit.measure_local(a, ops)) < 1e-12
    la, ph = tv.mps_overlap(pa, pb)
    lo, po = fit.overlap(a, b)
    assert abs(la - lo) < 1e-11
    assert abs(np.angle(np.exp(1j * (ph - po)))) < 1e-11


def test_error_codes(ctx):
    L = 6
    blocks = wl.tfi_blocks(L, 1.0)
    W = tv.mpo_build(ctx, *blocks, 2, -0.1j)
    psi = tv.mps_init(ctx, wl.product_state("up", L), 4)
    with pytest.raises(tv.TevoError) as e:
        tv.evolve_step(psi, W, -0.2j, 4, 1, tv.FP64)       # tau mismatch
    assert e.value.code == -3
    with pytest.raises(tv.TevoError) as e:
        tv.evolve_step(psi, W, -0.1j, 8, 1, tv.FP64)       # D mismatch
    assert e.value.code == -2
    with pytest.raises(tv.TevoError) as e:
        tv.evolve_step(psi, W, -0.1j, 4, 0, tv.FP64)       # no sweep
    assert e.value.code == -1
    W2 = tv.mpo_build(ctx, *wl.tfi_blocks(L + 1, 1.0), 2, -0.1j)
    with pytest.raises(tv.TevoError) as e:
        tv.evolve_step(psi, W2, -0.1j, 4, 1, tv.FP64)      # chain length mismatch
    assert e.value.code == -2
    # the state is still usable
    tv.evolve_step(psi, W, -0.1j, 4, 1, tv.FP64)


def test_gpu_mpo_upload_matches_host(ctx):
    blocks = wl.lr_ising_blocks(5, 0.7)
    W = tv.mpo_build(ctx, *blocks, 3, -0.2j)
    Wh = tv.mpo_build_host(*blocks, 3, -0.2j)
    for i in range(5):
        assert np.array_equal(W.site(i), Wh[i])
