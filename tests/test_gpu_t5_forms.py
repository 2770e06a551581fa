"""The headline chain to t = 5 on the GPU: the long-range Ising chain (L = 100,
D = 256, N = 3, tau = -0.2i, 2 sweeps per step, 25 steps, from all up), every
form against the fp64 oracle's stored observables (tests/golden, written by
tests/golden/make_golden.py from the oracle alone). Error measure: the largest
|<X_i>|, |<Y_i>|, |<Z_i>| deviation over all sites at the recorded steps.

Forms and bounds:
  * TEVO_FP64 | TEVO_OZAKI (every contraction as exact bf16 digit-slice
    products on the tensor cores, the benchmark's form): <= 1e-8;
  * TEVO_FP64 (the fp64 form): <= 1e-10;
  * TEVO_BF16X3 (a bf16x3 tensor-core sweep, then a native fp64 sweep) and
    TEVO_BF16X3 | TEVO_OZAKI (the fp64 sweep as Ozaki-scheme GEMMs): <= 2e-6.
    One tensor-core sweep moves the fit's trajectory by about 1e-6 at t = 5
    whatever its precision; the bound records that level.
The fp64 form takes about 12 minutes and the bf16x3 form about 8."""
import json
import os

import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)
tv = pytest.importorskip("paper_2302_14181_gb300")

HERE = os.path.dirname(os.path.abspath(__file__))
NAME = "lri_L100_N3_D256"


@pytest.fixture(scope="module")
def setup():
    torch.cuda.set_device(0)
    ctx = tv.Context()
    cfg = wl.config(NAME)
    W = tv.mpo_build(ctx, *wl.model_blocks(cfg), cfg["N"], cfg["tau"])
    g = json.load(open(os.path.join(HERE, "golden", NAME + ".json")))
    assert g["config"]["sweeps"] == cfg["sweeps"] and g["config"]["D"] == cfg["D"]
    return ctx, cfg, W, g


def evolve_errors(setup, prec):
    ctx, cfg, W, g = setup
    ops = list(wl.pauli())
    psi = tv.mps_init(ctx, wl.initial_vectors(cfg), cfg["D"])
    errs = {}
    for k in range(1, cfg["steps"] + 1):
        tv.evolve_step(psi, W, cfg["tau"], cfg["D"], cfg["sweeps"], prec)
        if str(k) in g["steps"]:
            got = tv.measure_local(psi, ops).real
            errs[k] = float(np.abs(got - np.array(g["steps"][str(k)])).max())
    assert abs(psi.log_norm() - g["log_norm"][-1]) < 1e-6
    return errs


@pytest.mark.parametrize("name,prec,bound", [
    ("fp64+oz", tv.FP64 | tv.OZAKI, 1e-8),
    ("bf16x3+oz", tv.BF16X3 | tv.OZAKI, 2e-6),
    ("bf16x3", tv.BF16X3, 2e-6),
    ("fp64", tv.FP64, 1e-10),
])
def test_headline_chain_to_t5(setup, name, prec, bound):
    errs = evolve_errors(setup, prec)
    print(name, {k: f"{v:.2e}" for k, v in errs.items()})
    assert max(errs.values()) <= bound, errs
