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
