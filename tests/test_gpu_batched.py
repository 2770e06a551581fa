"""The batched form: independent chains stepped together (worker streams, then a
captured CUDA graph) give each chain exactly its single-chain result, and the
fp64 form matches the oracle."""
import numpy as np
import pytest

import workloads as wl
from oracle import fit, mpo

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)
tv = pytest.importorskip("paper_2302_14181_gb300")


@pytest.fixture(scope="module")
def ctx():
    torch.cuda.set_device(0)
    return tv.Context()


def small_chains(seed=3, n=6):
    rng = np.random.default_rng(seed)
    out = []
    for c in range(n):
        L = int(rng.integers(6, 13))
        model = ["tfi", "xxz"][c % 2]
        J = rng.uniform(0.5, 1.5, L - 1)
        blocks = wl.tfi_blocks(L, 1.05, J) if model == "tfi" else wl.xxz_blocks(L, 0.5, J)
        v0 = wl.product_state("up" if model == "tfi" else "neel", L)
        out.append(dict(blocks=blocks, v0=v0, N=2 + c % 2, D=[4, 8, 16][c % 3], tau=-0.1j))
    return out


@pytest.mark.parametrize("prec", [tv.FP64, tv.TF32X3 | tv.TC_ONLY, tv.BF16X3])
def test_batched_equals_single_chain(ctx, prec):
    chains = small_chains()
    ops = list(wl.pauli())
    Ws = [tv.mpo_build(ctx, *c["blocks"], c["N"], c["tau"]) for c in chains]
    psis_b = [tv.mps_init(ctx, c["v0"], c["D"]) for c in chains]
    psis_s = [tv.mps_init(ctx, c["v0"], c["D"]) for c in chains]
    sweeps = 2 if (prec & 0xFF) == tv.BF16X3 else 1
    for step in range(8):          # warm-up, three timed schedules, two captures, replays
        tv.evolve_step_batched(psis_b, Ws, sweeps, prec)
        for c, p, W in zip(chains, psis_s, Ws):
            tv.evolve_step(p, W, c["tau"], c["D"], sweeps, prec)
        for pb, ps in zip(psis_b, psis_s):
            a = tv.measure_local(pb, ops)
            b = tv.measure_local(ps, ops)
            assert np.abs(a - b).max() < 1e-13, (step, np.abs(a - b).max())
            assert pb.log_norm() == ps.log_norm()


def test_batched_fp64_against_oracle(ctx):
    chains = small_chains(seed=5, n=4)
    ops = list(wl.pauli())
    Ws = [tv.mpo_build(ctx, *c["blocks"], c["N"], c["tau"]) for c in chains]
    psis = [tv.mps_init(ctx, c["v0"], c["D"]) for c in chains]
    refs = [fit.product_mps(c["v0"], c["D"]) for c in chains]
    Wo = [mpo.build_mpo(*c["blocks"], c["N"], c["tau"]) for c in chains]
    for step in range(6):
        tv.evolve_step_batched(psis, Ws, 1, tv.FP64)
        refs = [fit.evolve_step(r, w, 1, canonical=step > 0)[0] for r, w in zip(refs, Wo)]
    for p, r in zip(psis, refs):
        got, ref = tv.measure_local(p, ops).real, fit.measure_local(r, ops).real
        assert np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-3) < 1e-10
