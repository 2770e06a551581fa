"""The spin-1 precision workload at reduced length: spin-1 Heisenberg with
single-ion anisotropy D_z = 0.3 (d = 3), order N = 4 (w = 160), tau = -0.25i,
L = 32, D = 256, seeded random product start, 16 steps (t = 4), 2 sweeps per
step, each form against the fp64 oracle's stored observables
(tests/golden/spin1_L32_N4_D256.json, written by tests/golden/make_golden.py
from the oracle alone). Error: the largest |<S^a_i>| deviation over all sites,
a = x, y, z.

This trajectory amplifies any difference in rounding: the GPU's native fp64
form, which differs from the oracle only in the order of its sums, stays at
1e-15 to t = 2 and reaches about 1e-10 at t = 4. So each form has a bound up to
t = 3 (step 12) and a looser one at t = 4 (step 16):
  * fp64: 1e-11 / 1e-9;
  * every contraction as Ozaki-scheme GEMMs: 1e-8 / 1e-6;
  * a bf16x3 sweep, then an fp64 sweep (native or as Ozaki-scheme GEMMs):
    1e-6 / 5e-5.
The full-size step times come from `bench.py --c5`."""
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

PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "spin1_L32_N4_D256.json")


@pytest.mark.parametrize("name,prec,bound3,bound4", [
    ("fp64", tv.FP64, 1e-11, 1e-9),
    ("fp64+oz", tv.FP64 | tv.OZAKI, 1e-8, 1e-6),
    ("bf16x3+oz", tv.BF16X3 | tv.OZAKI, 1e-6, 5e-5),
    ("bf16x3", tv.BF16X3, 1e-6, 5e-5),
])
def test_spin1_L32_D256_to_t4(name, prec, bound3, bound4):
    if not os.path.exists(PATH):
        pytest.skip(f"{PATH} not generated")
    g = json.load(open(PATH))
    torch.cuda.set_device(0)
    ctx = tv.Context()
    cfg = wl.config("spin1_L128_N4_D512", L=32, D=256)
    assert (g["config"]["L"], g["config"]["D"], g["config"]["steps"]) == (32, 256, 16)
    W = tv.mpo_build(ctx, *wl.model_blocks(cfg), cfg["N"], cfg["tau"])
    ops = list(wl.spin_one())
    psi = tv.mps_init(ctx, wl.initial_vectors(cfg), cfg["D"])
    errs = {}
    for k in range(1, 17):
        tv.evolve_step(psi, W, cfg["tau"], cfg["D"], cfg["sweeps"], prec)
        if str(k) in g["steps"]:
            errs[k] = float(np.abs(tv.measure_local(psi, ops).real - np.array(g["steps"][str(k)])).max())
    print("spin1 L=32 D=256", name, {k: f"{v:.2e}" for k, v in errs.items()})
    assert max(v for k, v in errs.items() if k <= 12) <= bound3, errs
    assert errs[16] <= bound4, errs
