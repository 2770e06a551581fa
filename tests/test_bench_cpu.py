"""Host logic of bench.py, on the CPU.

* step_flops, the useful-flop count behind the bench's TFLOP/s figure, equals 8x
  the complex multiply-adds of every matmul the oracle's contractions perform in
  one step (counted while the oracle runs, not re-derived).
* traffic_from_profiles reports a recorded dram figure only while the kernel's
  source file still has the recorded hash.
"""
import hashlib
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402
import workloads as wl  # noqa: E402
from oracle import fit, mpo  # noqa: E402


class _Counted(np.ndarray):
    """ndarray view whose matmuls add M*K*N to a shared counter."""

    counter = None

    def __array_ufunc__(self, ufunc, method, *inputs, **kwargs):
        args = [np.asarray(x) if isinstance(x, _Counted) else x for x in inputs]
        if ufunc is np.matmul and method == "__call__":
            a, b = args
            assert a.ndim == 2 and b.ndim == 2
            _Counted.counter[0] += a.shape[0] * a.shape[1] * b.shape[1]
        out = getattr(ufunc, method)(*args, **kwargs)
        return out.view(_Counted) if isinstance(out, np.ndarray) else out


def _counting(fn):
    def wrapped(*arrays):
        out = fn(*[np.asarray(x).view(_Counted) for x in arrays])
        return np.asarray(out)
    return wrapped


@pytest.mark.parametrize("sweeps", [1, 2])
@pytest.mark.parametrize("case", [
    ("xxz_L7_N2_D4", lambda: wl.xxz_blocks(7, 0.5), lambda: wl.product_state("neel", 7), 2, 4),
    ("lri_L6_N3_D6", lambda: wl.lr_ising_blocks(6, 0.7), lambda: wl.product_state("up", 6), 3, 6),
])
def test_step_flops_counts_the_oracle_contractions(monkeypatch, case, sweeps):
    name, blocks, v0, N, D = case
    W = mpo.build_mpo(*blocks(), N, -0.1j)
    psi = fit.product_mps(v0(), D)
    # one step first, so that the counted step starts from a right-canonical state
    psi, _ = fit.evolve_step(psi, W, 1, canonical=False)
    counter = [0]
    monkeypatch.setattr(_Counted, "counter", counter)
    for f in ("make_T", "apply_T", "env_next"):
        monkeypatch.setattr(fit, f, _counting(getattr(fit, f)))
    fit.evolve_step(psi, W, sweeps, canonical=True)
    dims = [a.shape[0] for a in psi] + [psi[-1].shape[2]]
    wl_ = [w.shape[0] for w in W]
    wr_ = [w.shape[3] for w in W]
    assert counter[0] > 0
    assert bench.step_flops(dims, wl_, wr_, psi[0].shape[1], sweeps) == 8.0 * counter[0], name


def test_traffic_only_while_source_unchanged(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("__global__ void k() {}\n")
    h = hashlib.sha256(src.read_bytes()).hexdigest()[:16]
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.txt").write_text(
        "# kernel bytes hash file\nk_kernel 123456 %s k.cu\nother 1 0000000000000000 k.cu\n" % h)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_from_profiles("k_kernel") == 123456.0
    assert bench.traffic_from_profiles("other") is None          # recorded for another source
    assert bench.traffic_from_profiles("missing_kernel") is None
    src.write_text("__global__ void k() { /* changed */ }\n")
    assert bench.traffic_from_profiles("k_kernel") is None


def test_single_replica_throughput():
    torch = pytest.importorskip("torch")  # noqa: F841
    v, ms = bench.replica_throughput(250.0, 2, "cpu")
    assert ms == 250.0 and v == pytest.approx(8.0)


def test_reference_arm_prints_one_contract_line(monkeypatch, capsys):
    import json
    from types import SimpleNamespace
    orig = bench.oracle_sample
    # the oracle timed as it stands, on a small interior shape so the test is quick
    monkeypatch.setattr(bench, "oracle_sample",
                        lambda cfg, seconds=0.0, seed=7: orig(dict(cfg, D=16), seconds=0.0, seed=seed))
    monkeypatch.delenv("RANK", raising=False)
    bench.reference_arm(SimpleNamespace(warmup=1, steps=2, gpus=1))
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == "sweeps/s"
    assert line["value"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "sweeps/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["config"]["workload"] == bench.WORKLOAD


def test_reference_arm_is_silent_off_rank_zero(monkeypatch, capsys):
    from types import SimpleNamespace
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setattr(bench, "oracle_sample", lambda *a, **k: pytest.fail("rank 1 must not run the oracle"))
    bench.reference_arm(SimpleNamespace(warmup=1, steps=1, gpus=2))
    assert capsys.readouterr().out == ""


def test_probe_cases_issue_their_calls(monkeypatch, capsys):
    """The fixed workloads behind the ncu captures in profiles/ (bench.py --probe),
    run against a stand-in of the binding that records the calls."""
    import types
    torch = pytest.importorskip("torch")
    calls = []

    class Handle:
        def bond_dims(self):
            return [1] + [93] * 19 + [1]

        def prof_enable(self, on=True):
            pass

        def prof_read(self, c):
            return (1.0, 5, 1e12, 0.0)

        def launch_count(self, reset=False):
            return 0

    fake = types.ModuleType("paper_2302_14181_gb300")
    fake.FP64, fake.TF32, fake.TF32X3, fake.BF16X3, fake.TC_ONLY, fake.OZAKI = 0, 1, 2, 3, 0x100, 0x200
    fake._lib = types.SimpleNamespace(PROF_GEMMOZ=4, PROF_OZSPLIT=5, PROF_QR=2, PROF_FORMQ=3)
    fake.Context = lambda: Handle()
    fake.mpo_build = lambda ctx, *a: Handle()
    fake.mps_init = lambda ctx, v0, D: (calls.append(("init", D)), Handle())[1]
    fake.evolve_step = lambda psi, W, tau, D, sweeps, prec: calls.append(("step", sweeps, prec))
    fake.measure_local = lambda psi, ops: calls.append(("measure",))
    fake.mps_overlap = lambda a, b: (0.0, 0.0)
    fake.tevo_gemm = lambda ctx, prec, A, B, C: calls.append(("gemm", tuple(A.shape), tuple(B.shape)))
    monkeypatch.setitem(sys.modules, "paper_2302_14181_gb300", fake)
    monkeypatch.setattr(torch.cuda, "set_device", lambda *a: None)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a: None)
    monkeypatch.setattr(torch.Tensor, "cuda", lambda self: self)
    zeros = torch.zeros
    monkeypatch.setattr(torch, "zeros", lambda *a, **k: zeros(*a, **{x: v for x, v in k.items() if x != "device"}))
    from types import SimpleNamespace
    expect = {
        "kernels": [("init", 256), ("step", 1, 0), ("measure",), ("init", 256), ("step", 2, 3), ("measure",),
                    ("init", 256), ("step", 2, 0x103), ("measure",), ("init", 256), ("step", 2, 0x203),
                    ("measure",), ("init", 256)],
        "form": [("init", 256), ("step", 2, 0x200), ("step", 2, 0x200)],
        "fp64": [("init", 256), ("step", 1, 0)],
        "tc": [("init", 256), ("step", 1, 0x103), ("init", 256), ("step", 1, 0x102)],
        "qr": [("init", 256)] + [("step", 2, 0x200)] * 5,
    }
    fake.TWO_SITE = 0x400
    fake.evolve_step_batched = lambda psis, Ws, sweeps, prec: calls.append(("batched", len(psis), sweeps, prec))
    expect["batched"] = [("init", c["D"]) for c in bench.wl.batched_chains()[:8]] + [("batched", 8, 1, 0x102)] * 3
    expect["twosite"] = [("init", 64), ("step", 1, 0x400)]
    for case in bench.PROBES:
        calls.clear()
        bench.probe(SimpleNamespace(probe=case, probe_L=20, probe_sweeps=1))
        if case == "ozgemm":
            shapes = sorted({c[1:] for c in calls})
            assert shapes == sorted({((23808, 256), (512, 256)), ((512, 23808), (256, 23808)),
                                     ((256, 512), (23808, 512)), ((186, 186), (65536, 186))}), shapes
            assert len(calls) == 4 * 6                   # one warm-up and five timed calls per shape
        else:
            assert calls == expect[case], case
    assert '"probe": "qr"' in capsys.readouterr().out
