"""Parity at the workloads' own sizes: the spin-1 order-4 chain (d = 3, w = 160)
at reduced length, the XXZ chain at full size (L = 64, D = 128) against the
oracle run here, and the long-range Ising headline chain (L = 100, D = 256,
w = 93) against the oracle's stored values in tests/golden (written by
tests/golden/make_golden.py, which calls only oracle/)."""
import json
import os

import numpy as np
import pytest

import workloads as wl
from oracle import fit, mpo

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)
tv = pytest.importorskip("paper_2302_14181_gb300")

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def ctx():
    torch.cuda.set_device(0)
    return tv.Context()


def rel_err(got, ref):
    return float(np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-3))


def test_spin1_order4_reduced(ctx):
    """Spin-1 Heisenberg + single-ion anisotropy, order 4 (w = 160), seeded random
    product state, D = 27 (truncating at the middle bonds), fp64 and bf16x3."""
    cfg = wl.config("spin1_L128_N4_D512", L=8, D=27)
    blocks = wl.model_blocks(cfg)
    v0 = wl.initial_vectors(cfg)
    ops = list(wl.spin_one())
    Wo = mpo.build_mpo(*blocks, cfg["N"], cfg["tau"])
    W = tv.mpo_build(ctx, *blocks, cfg["N"], cfg["tau"])
    assert W.bond_dims()[1] == 160
    ref_psi = fit.product_mps(v0, cfg["D"])
    p64 = tv.mps_init(ctx, v0, cfg["D"])
    pmx = tv.mps_init(ctx, v0, cfg["D"])
    for k in range(3):
        ref_psi, _ = fit.evolve_step(ref_psi, Wo, 2, canonical=k > 0)
        tv.evolve_step(p64, W, cfg["tau"], cfg["D"], 2, tv.FP64)
        tv.evolve_step(pmx, W, cfg["tau"], cfg["D"], 2, tv.BF16X3)
    ref = fit.measure_local(ref_psi, ops).real
    assert rel_err(tv.measure_local(p64, ops).real, ref) < 1e-10
    assert rel_err(tv.measure_local(pmx, ops).real, ref) < 1e-6


@pytest.mark.parametrize("name", ["xxz_L64_N2", "xxz_L64_N3"])
def test_xxz_full_size(ctx, name):
    cfg = wl.config(name)
    blocks = wl.model_blocks(cfg)
    v0 = wl.initial_vectors(cfg)
    ops = list(wl.pauli())
    Wo = mpo.build_mpo(*blocks, cfg["N"], cfg["tau"])
    W = tv.mpo_build(ctx, *blocks, cfg["N"], cfg["tau"])
    ref_psi = fit.product_mps(v0, cfg["D"])
    psi = tv.mps_init(ctx, v0, cfg["D"])
    for k in range(2):
        ref_psi, _ = fit.evolve_step(ref_psi, Wo, cfg["sweeps"], canonical=k > 0)
        tv.evolve_step(psi, W, cfg["tau"], cfg["D"], cfg["sweeps"], tv.FP64)
    assert rel_err(tv.measure_local(psi, ops).real, fit.measure_local(ref_psi, ops).real) < 1e-10


def _golden(name):
    path = os.path.join(GOLDEN, name + ".json")
    if not os.path.exists(path):
        pytest.skip(f"{path} not generated")
    return json.load(open(path))


@pytest.mark.parametrize("prec,tol", [(tv.BF16X3, 1e-10), (tv.FP64, 1e-10)])
def test_lri_headline_size_first_steps(ctx, prec, tol):
    """The long-range Ising chain at full size: after one and two steps the
    observables equal the oracle's (the mixed form ends with an fp64 sweep)."""
    g = _golden("lri_L100_N3_D256")
    cfg = wl.config("lri_L100_N3_D256")
    W = tv.mpo_build(ctx, *wl.model_blocks(cfg), cfg["N"], cfg["tau"])
    psi = tv.mps_init(ctx, wl.initial_vectors(cfg), cfg["D"])
    nsteps = 2 if prec != tv.FP64 else 1
    for k in range(1, nsteps + 1):
        tv.evolve_step(psi, W, cfg["tau"], cfg["D"], cfg["sweeps"], prec)
        ref = np.array(g["steps"][str(k)])
        got = tv.measure_local(psi, list(wl.pauli())).real
        assert rel_err(got, ref) < tol, (k, rel_err(got, ref))
        assert abs(psi.log_norm() - g["log_norm"][k - 1]) < 1e-9


@pytest.mark.parametrize("N", [2, 3])
@pytest.mark.parametrize("tau", [0.1, 0.2, 0.4])
def test_xxz_to_t5_against_golden(ctx, N, tau):
    """The XXZ chain at full size (L = 64, D = 128, Neel start, 2 sweeps per
    step) to t = 5 at each time step tau in {0.1, 0.2, 0.4} (-i); tau = 0.4 takes
    12 steps and a last step with the MPO built at 0.2. The fp64 form against
    the oracle's stored observables at every recorded step (1e-10 relative,
    log-norm to 1e-9); the fp32-class variant (a tf32x3 tensor-core sweep, then
    an fp64 sweep) is printed beside it and bounded by 1e-4."""
    g = _golden(f"xxz_L64_N{N}_tau{tau}")
    cfg = wl.config(f"xxz_L64_N{N}", tau=-1j * tau)
    assert g["config"]["D"] == cfg["D"] and g["config"]["sweeps"] == cfg["sweeps"] and g["config"]["N"] == N
    blocks = wl.model_blocks(cfg)
    ops = list(wl.pauli())
    W = tv.mpo_build(ctx, *blocks, N, cfg["tau"])
    last = g["config"].get("last_tau")
    tau_last = complex(*last) if last else cfg["tau"]
    W_last = tv.mpo_build(ctx, *blocks, N, tau_last) if last else W
    steps = g["config"]["steps"]
    out = {}
    for name, prec in (("fp64", tv.FP64), ("tf32x3", tv.TF32X3)):
        psi = tv.mps_init(ctx, wl.initial_vectors(cfg), cfg["D"])
        errs = {}
        for k in range(1, steps + 1):
            Wk, tk = (W_last, tau_last) if k == steps else (W, cfg["tau"])
            tv.evolve_step(psi, Wk, tk, cfg["D"], cfg["sweeps"], prec)
            if str(k) in g["steps"]:
                errs[k] = rel_err(tv.measure_local(psi, ops).real, np.array(g["steps"][str(k)]))
        out[name] = (max(errs.values()), abs(psi.log_norm() - g["log_norm"][-1]))
    print(f"xxz N={N} tau={tau}: fp64 {out['fp64'][0]:.2e} (log-norm {out['fp64'][1]:.1e}), "
          f"tf32x3 {out['tf32x3'][0]:.2e} (log-norm {out['tf32x3'][1]:.1e})")
    assert out["fp64"][0] < 1e-10 and out["fp64"][1] < 1e-9
    assert out["tf32x3"][0] < 1e-4


def test_spin1_L32_D128_to_t1(ctx):
    """Spin-1 Heisenberg + single-ion anisotropy, order 4 (w = 160, d = 3) at
    L = 32, D = 128, seeded random product start, 4 steps of tau = -0.25i (t = 1)
    against the oracle's stored observables: fp64 at 1e-10, every contraction as
    Ozaki-scheme GEMMs at 1e-8, and the bf16x3 mixed forms at 1e-6."""
    g = _golden("spin1_L32_N4_D128")
    cfg = wl.config("spin1_L128_N4_D512", L=32, D=128)
    assert g["config"]["D"] == 128 and g["config"]["L"] == 32 and g["config"]["steps"] == 4
    blocks = wl.model_blocks(cfg)
    ops = list(wl.spin_one())
    W = tv.mpo_build(ctx, *blocks, cfg["N"], cfg["tau"])
    assert W.bond_dims()[16] == 160
    res = {}
    for name, prec, tol in (("fp64", tv.FP64, 1e-10), ("fp64+oz", tv.FP64 | tv.OZAKI, 1e-8),
                            ("bf16x3", tv.BF16X3, 1e-6), ("bf16x3+oz", tv.BF16X3 | tv.OZAKI, 1e-6)):
        psi = tv.mps_init(ctx, wl.initial_vectors(cfg), cfg["D"])
        errs = []
        for k in range(1, 5):
            tv.evolve_step(psi, W, cfg["tau"], cfg["D"], cfg["sweeps"], prec)
            errs.append(rel_err(tv.measure_local(psi, ops).real, np.array(g["steps"][str(k)])))
        res[name] = max(errs)
        assert res[name] < tol, (name, errs)
    print("spin1 L=32 D=128 t=1:", {k: f"{v:.2e}" for k, v in res.items()})


def test_tfi_first_order_40_steps_against_exact(ctx):
    """The first-order TFI workload (L = 12, g = 1.05, tau = -0.05i, D = 16, 40
    steps): the GPU's fp64 observables equal the oracle's (1e-10 relative) and so
    carry the same error against exact evolution (dense exp(tau H) from eigh of
    the 4096 x 4096 Hamiltonian): the MPO's method error plus truncation."""
    from oracle import dense
    cfg = wl.config("tfi_L12")
    L = cfg["L"]
    blocks = wl.model_blocks(cfg)
    X, _, Z = wl.pauli()
    E = dense.expm_tau_h(dense.hamiltonian_from_blocks(*blocks), cfg["tau"])
    v_ex = dense.product_vector(wl.initial_vectors(cfg))
    Wo = mpo.build_mpo(*blocks, cfg["N"], cfg["tau"])
    W = tv.mpo_build(ctx, *blocks, cfg["N"], cfg["tau"])
    psi = tv.mps_init(ctx, wl.initial_vectors(cfg), cfg["D"])
    psi_o = fit.product_mps(wl.initial_vectors(cfg), cfg["D"])
    for k in range(cfg["steps"]):
        v_ex = E @ v_ex
        psi_o, _ = fit.evolve_step(psi_o, Wo, cfg["sweeps"], canonical=k > 0)
        tv.evolve_step(psi, W, cfg["tau"], cfg["D"], cfg["sweeps"], tv.FP64)
    exact = dense.expect_dense(v_ex, [X, Z], L).real
    got = tv.measure_local(psi, [X, Z]).real
    ref = fit.measure_local(psi_o, [X, Z]).real
    assert rel_err(got, ref) < 1e-10
    e_gpu, e_orc = np.abs(got - exact).max(), np.abs(ref - exact).max()
    assert abs(e_gpu - e_orc) < 1e-10
    assert 1e-4 < e_gpu < 3e-3   # first order at tau = 0.05 over t = 2: the method error
