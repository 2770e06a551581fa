"""Benchmark of the time-evolution fit: W^(N)(tau) applied to a finite MPS and
fitted back to bond dimension D by variational sweeps, one step after another.

One bench step = one call of evolve_step (all sweeps of one time step, with its
environment build, QRs, centre and normalisation) on the long-range Ising chain
L = 100, D = 256, order N = 3 (w = 93), tau = -0.2i (the headline workload), by
default with every contraction as exact Ozaki-scheme digit-slice GEMMs on the
bf16 tensor cores (fp64-accurate) and fp64 QR and reductions.
The state lives in HBM across steps; the
environments (about 9.7 GB in fp64) are larger than L2, so no flush is needed.

Usage:
  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64+oz|fp64|bf16x3|bf16x3+oz|...]
  python bench.py --impl reference ...     # the fp64 oracle on the host cores
  python bench.py --verify                 # every form to t = 5 against the oracle's stored values
  python bench.py --c5                     # one step of each form on the full-size spin-1 chain
  python bench.py --oracle-step            # one full oracle step on the host cores
  python bench.py --splitting              # complex-step splitting vs the native order-2 MPO
  python bench.py --cylinder               # fidelity density vs time step, 2-D TFI cylinder
  python bench.py --probe <case>           # the fixed small workloads of the ncu captures
Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as wl  # noqa: E402

METRIC = "W^(N)·MPS fit sweeps/s & TFLOP/s vs peak at ≤1e-6 obs error, mixed vs FP64"
WORKLOAD = "lri_L100_N3_D256"
PREC = {"fp64": 0, "tf32": 1, "tf32x3": 2, "bf16x3": 3,
        "tc-tf32": 0x101, "tc-tf32x3": 0x102, "tc-bf16x3": 0x103,
        # fp64 contractions as Ozaki-scheme GEMMs (8 digit slices) on the tensor cores
        "fp64+oz": 0x200, "tf32+oz": 0x201, "tf32x3+oz": 0x202, "bf16x3+oz": 0x203}
OZ_SLICES = 8
OZ_PAIRS = OZ_SLICES * (OZ_SLICES + 1) // 2  # digit-slice products per complex product
# fp64 issue rate on GB300: 2 DFMA per clock per SM (152 SMs, 2070 MHz max SM clock)
FP64_PEAK_TFLOPS = 2 * 2 * 152 * 2.070e9 / 1e12


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def step_flops(dims, wl_, wr_, d, sweeps, canonical=True):
    """Useful flops of one evolve_step (complex MACs x 8, the MPO treated as dense)."""
    L = len(wl_)

    def right(i):
        Dp, Db, a, b = dims[i], dims[i + 1], wl_[i], wr_[i]
        g1 = Dp * a * Dp * d * Db
        g2 = Dp * (d * b) * (a * d) * Db
        g3 = Dp * d * Db * (b * Db)
        return g1, g2, g3, g3

    def left(i):
        Dp, Db, a, b = dims[i + 1], dims[i], wr_[i], wl_[i]
        g1 = Dp * a * Dp * d * Db
        g2 = Dp * (d * b) * (a * d) * Db
        g3 = Dp * d * Db * (b * Db)
        return g1, g2, g3, g3

    macs = 0
    for i in range(1, L):
        g1, g2, _, g3e = left(i)
        macs += g1 + g2 + g3e                      # right environment build
    for _ in range(sweeps):
        for i in range(L - 1):
            macs += sum(right(i))
        for i in range(L - 1, 0, -1):
            macs += sum(left(i))
    g1, g2, g3, _ = left(0)
    macs += g1 + g2 + g3                           # centre
    return 8.0 * macs


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        clk, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                clk.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not clk:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(clk), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(clk)}


# ----------------------------------------------------------------------------
# the oracle's bounded sample (cpu_baseline and --impl reference)
# ----------------------------------------------------------------------------

def oracle_sample(cfg, seconds=15.0, seed=7):
    """Time local updates of the oracle (make_T, apply, Householder QR, new
    environment) at the workload's interior-site shape on seeded random
    operands; scale to sweeps/s of a full step."""
    from oracle import fit, mpo
    L, d, D = cfg["L"], cfg["d"], cfg["D"]
    blocks = wl.model_blocks(dict(cfg, L=4))
    W = mpo.build_mpo(*blocks, cfg["N"], cfg["tau"])[1]
    w = W.shape[0]
    rng = np.random.default_rng(seed)
    cg = lambda *s: (rng.standard_normal(s) + 1j * rng.standard_normal(s)) / math.sqrt(max(s))
    El, A, Er = cg(D, w, D), cg(D, d, D), cg(D, w, D)
    n = 0
    t0 = time.perf_counter()
    while True:
        T = fit.make_T(El, A, W)
        B = fit.apply_T(T, Er)
        Q, _ = fit.householder_qr(B.reshape(D * d, D))
        fit.env_next(Q.reshape(D, d, D), T)
        n += 1
        if time.perf_counter() - t0 > seconds:
            break
    t_up = (time.perf_counter() - t0) / n
    sweeps = cfg["sweeps"]
    updates_per_step = sweeps * 2 * (L - 1) + 0.75 * (L - 1) + 1
    t_step = t_up * updates_per_step
    threads = int(os.environ.get("OPENBLAS_NUM_THREADS", os.cpu_count() or 1))
    return {"sweeps_per_s": sweeps / t_step, "t_update_s": t_up, "updates": n, "cores": threads,
            "t_step_s": t_step}


NPROF = 6
PROF_NAMES = ["gemm64", "gemm_tc", "qr", "form_q", "gemm_oz", "oz_split"]


def dtype_of(form):
    if form == "fp64":
        return "c128"
    if form == "fp64+oz":
        return ("c128 in/out; every contraction as exact bf16 digit-slice products on the tensor cores (Ozaki, "
                "8 slices) with exact fixed-point sums, rounded once to f64; c128 QR and reductions")
    base = form.replace("tc-", "").replace("+oz", "")
    if form.startswith("tc-"):
        return f"{base} contractions + c128 QR"
    if form.endswith("+oz"):
        return f"{base} contractions + c128 QR; fp64 rebuild/final sweep as Ozaki bf16 digit-slice GEMMs"
    return f"{base} contractions + c128 QR/final sweep"


def config_of(cfg, sweeps, precision, world=1):
    return {"workload": WORKLOAD, "model": "long-range Ising, J(r)=sum_k a_k b_k^r ~ 1/r^2, g=0.7",
            "L": cfg["L"], "D": cfg["D"], "N": cfg["N"], "w": 93, "tau": "-0.2i", "sweeps": sweeps,
            "precision": precision, "l2": "inputs larger than L2 (environments ~9.7 GB)",
            "parallelism": f"replicas x{world}"}


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cfg = wl.config(WORKLOAD)
    for _ in range(args.warmup):
        oracle_sample(cfg, seconds=2.0)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(oracle_sample(cfg, seconds=10.0)["sweeps_per_s"])
    wall = time.perf_counter() - t0
    v = statistics.median(vals)
    s = oracle_sample(cfg, seconds=0.1)
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "sweeps/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / max(1, args.steps),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
        "data": "synthetic", "config": config_of(cfg, cfg["sweeps"], "fp64 oracle (numpy, host cores)"),
        "cpu_baseline": {"value": v, "unit": "sweeps/s", "cores": s["cores"], "kind": "oracle",
                         "sample": "10 s of oracle local updates (make_T, apply, Householder QR, environment) "
                                   "per step at the interior-site shape D=256, w=93, d=2, scaled to one "
                                   "evolve_step of the L=100 chain"},
        "e2e": {"value": v, "unit": "sweeps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------

def traffic_from_profiles(kernel):
    """dram bytes per launch recorded in profiles/ for a kernel, if the source it
    was taken from is unchanged (checked by hash)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    for ln in open(path):
        parts = ln.split()
        if len(parts) >= 4 and parts[0] == kernel:
            src = os.path.join(ROOT, parts[3])
            if not os.path.exists(src):
                return None
            h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
            return float(parts[1]) if h == parts[2] else None
    return None


def replica_throughput(ms_local, units_local, device):
    """Whole-job throughput of independent replicas: every rank reports its own
    elapsed time; the job took the slowest rank's time and processed the units
    of all ranks (no data-path collective, only this max-reduction)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size() if dist.is_initialized() else 1
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units_local)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
    ms_max = float(t.item())
    return float(u.item()) / (ms_max / 1e3), ms_max


def our_arm(args):
    import torch
    import torch.distributed as dist
    import paper_2302_14181_gb300 as tv

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    prec = PREC[args.precision]
    cfg = wl.config(WORKLOAD)
    blocks = wl.model_blocks(cfg)
    tau, D, sweeps = cfg["tau"], cfg["D"], args.sweeps or cfg["sweeps"]
    ctx = tv.Context()
    W = tv.mpo_build(ctx, *blocks, cfg["N"], tau)
    psi = tv.mps_init(ctx, wl.initial_vectors(cfg), D)
    stream = torch.cuda.current_stream()

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()

    for _ in range(args.warmup):
        tv.evolve_step(psi, W, tau, D, sweeps, prec)
    barrier()
    dims = psi.bond_dims()
    wd = W.bond_dims()
    flops = step_flops(dims, wd[:-1], wd[1:], cfg["d"], sweeps)
    ctx.launch_count(reset=True)
    ctx.prof_enable(True)
    for c in range(NPROF):
        ctx.prof_read(c)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clocks:
        barrier()
        e0.record(stream)
        for _ in range(args.steps):
            tv.evolve_step(psi, W, tau, D, sweeps, prec)
        e1.record(stream)
        barrier()
    ctx.prof_enable(False)
    ms = e0.elapsed_time(e1)
    launches = ctx.launch_count()
    prof = {c: ctx.prof_read(c) for c in range(NPROF)}
    value, ms_max = replica_throughput(ms, args.steps * sweeps, "cuda")
    # observables after warmup + steps time steps against the oracle's stored values
    obs_err = None
    gpath = os.path.join(ROOT, "tests", "golden", WORKLOAD + ".json")
    nstep = args.warmup + args.steps
    if os.path.exists(gpath):
        g = json.load(open(gpath))
        if str(nstep) in g["steps"] and g["config"]["sweeps"] == sweeps:
            ref = np.array(g["steps"][str(nstep)])
            got = tv.measure_local(psi, list(wl.pauli())).real
            obs_err = {"step": nstep, "t": nstep * abs(tau), "max_abs": float(np.abs(got - ref).max()),
                       "against": "fp64 oracle (tests/golden)"}
    # the other forms, one step each from the same state: the plain fp64 form
    # (the comparison the metric names) and the tensor-core sweep forms (one
    # bf16x3 sweep, then an fp64 sweep: native, or as Ozaki-scheme GEMMs)
    fp64_form, other_forms = None, {}
    if not args.no_fp64_compare:
        for name in ("fp64", "bf16x3", "bf16x3+oz", "fp64+oz"):
            if PREC[name] == prec:
                continue
            barrier()
            f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            f0.record(stream)
            tv.evolve_step(psi, W, tau, D, sweeps, PREC[name])
            f1.record(stream)
            barrier()
            fms = f0.elapsed_time(f1)
            other_forms[name] = {"value": sweeps / (fms / 1e3), "unit": "sweeps/s", "ms_per_step": fms,
                                 "sweeps": sweeps, "dtype": dtype_of(name),
                                 "speedup_of_measured_form": (fms / (ms_max / args.steps))}
        fp64_form = other_forms.get("fp64")

    # the batched form (64 independent TFI/XXZ chains of uneven size, complex
    # fp32-class contractions with fp64 QR, one graph replay per step) against
    # looping the single-chain call over the same chains
    batched = None
    if not args.no_fp64_compare:
        chains = wl.batched_chains()
        bW = [tv.mpo_build(ctx, *wl.model_blocks(c), c["N"], c["tau"]) for c in chains]
        bprec = PREC["tc-tf32x3"]
        bsw = chains[0]["sweeps"]
        bps = [tv.mps_init(ctx, wl.initial_vectors(c), c["D"]) for c in chains]
        for _ in range(8):        # schedule timing, two graph captures, replays
            tv.evolve_step_batched(bps, bW, bsw, bprec)
        barrier()
        b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        b0.record(stream)
        for _ in range(3):
            tv.evolve_step_batched(bps, bW, bsw, bprec)
        b1.record(stream)
        barrier()
        bms = b0.elapsed_time(b1) / 3
        lps = [tv.mps_init(ctx, wl.initial_vectors(c), c["D"]) for c in chains]
        for c, p_, w_ in zip(chains, lps, bW):
            tv.evolve_step(p_, w_, c["tau"], c["D"], bsw, bprec)
        barrier()
        l0, l1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0.record(stream)
        for c, p_, w_ in zip(chains, lps, bW):
            tv.evolve_step(p_, w_, c["tau"], c["D"], bsw, bprec)
        l1.record(stream)
        barrier()
        lms = l0.elapsed_time(l1)
        batched = {"workload": "64 chains: TFI/XXZ, J per bond U[0.5,1.5], L in [16,80], D in {32,64,128}, "
                               "N in {2,3}, tau=-0.1i",
                   "precision": "tc-tf32x3 (tf32x3 contractions, fp64 QR)", "sweeps": bsw,
                   "ms_per_step": bms, "chain_sweeps_per_s": len(chains) * bsw / (bms / 1e3),
                   "looped_ms_per_step": lms, "looped_chain_sweeps_per_s": len(chains) * bsw / (lms / 1e3)}
        del bps, lps, bW

    # end to end through the public API with host buffers (pinned), every step:
    # upload the state, evolve, read observables and the state back
    ops = [wl.pauli()[0], wl.pauli()[2]]
    host = [torch.empty(psi.site(i).shape, dtype=torch.complex128, pin_memory=True).numpy()
            for i in range(cfg["L"])]
    for i in range(cfg["L"]):
        host[i][...] = psi.site(i)
    h2d = sum(h.nbytes for h in host)
    d2h = h2d + 16 * len(ops) * cfg["L"]
    e2e_steps = max(1, args.steps)
    parts = {"upload_s": 0.0, "evolve_s": 0.0, "measure_s": 0.0, "download_s": 0.0}
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ta = time.perf_counter()
        for i in range(cfg["L"]):
            psi.set_site(i, host[i])
        torch.cuda.synchronize()
        tb = time.perf_counter()
        tv.evolve_step(psi, W, tau, D, sweeps, prec)      # synchronises (reads the step's device flags)
        tc = time.perf_counter()
        tv.measure_local(psi, ops)                        # synchronises
        td = time.perf_counter()
        for i in range(cfg["L"]):
            host[i][...] = psi.site(i)
        te = time.perf_counter()
        parts["upload_s"] += tb - ta
        parts["evolve_s"] += tc - tb
        parts["measure_s"] += td - tc
        parts["download_s"] += te - td
    barrier()
    t_e2e = time.perf_counter() - t0
    parts = {k: v / e2e_steps for k, v in parts.items()}
    e2e_val, _ = replica_throughput(1e3 * t_e2e, e2e_steps * sweeps, "cuda")

    if rank == 0:
        peaks, src = load_peaks()
        def fp64_roof(kms, kn, kfl):
            achieved = kfl / (kms / 1e3) / 1e12 if kms > 0 else None
            return {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": achieved / FP64_PEAK_TFLOPS if achieved else None,
                    "traffic": traffic_from_profiles("zgemm_kernel"),
                    "kernel": "zgemm_kernel (fp64 complex GEMM)", "launches": kn,
                    "avg_launch_ms": kms / kn if kn else None,
                    "peak_source": "derived: 2 DFMA/clk/SM x 152 SMs x 2070 MHz (fp64 pipe)"}

        def tc_roof(kms, kn, kfl):
            base = prec & 0xFF
            passes = 1 if base == 1 else 3
            peak = peaks.get("bf16_tflops_sustained", 1700.0) * (0.5 if base in (1, 2) else 1.0)
            achieved = passes * kfl / (kms / 1e3) / 1e12 if kms > 0 else None
            return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak if achieved else None, "traffic": traffic_from_profiles("tc_gemm_kernel"),
                    "kernel": "tc_gemm_kernel (tcgen05 complex GEMM; executed flops = useful x passes)",
                    "launches": kn, "avg_launch_ms": kms / kn if kn else None, "passes": passes,
                    "useful_tflops": kfl / (kms / 1e3) / 1e12 if kms > 0 else None,
                    "peak_source": f"{src} bf16 sustained" + (" x 0.5 (tf32)" if base in (1, 2) else "")}

        def oz_roof(kms, kn, kfl):
            peak = peaks.get("bf16_tflops_sustained", 1700.0)
            achieved = OZ_PAIRS * kfl / (kms / 1e3) / 1e12 if kms > 0 else None
            return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak if achieved else None, "traffic": traffic_from_profiles("oz_gemm_kernel"),
                    "kernel": "oz_gemm_kernel (Ozaki-scheme fp64 GEMM on bf16 tcgen05; executed flops = useful x "
                              f"{OZ_PAIRS} digit-slice products)",
                    "launches": kn, "avg_launch_ms": kms / kn if kn else None, "passes": OZ_PAIRS,
                    "useful_tflops": kfl / (kms / 1e3) / 1e12 if kms > 0 else None,
                    "peak_source": f"{src} bf16 sustained"}

        g64, gtc, goz = prof[tv._lib.PROF_GEMM64], prof[tv._lib.PROF_GEMMTC], prof[tv._lib.PROF_GEMMOZ]
        roofs = {}
        if g64[0] > 0:
            roofs["fp64_gemm"] = fp64_roof(g64[0], g64[1], g64[2])
        if gtc[0] > 0:
            roofs["tc_gemm"] = tc_roof(gtc[0], gtc[1], gtc[2])
        if goz[0] > 0:
            roofs["oz_gemm"] = oz_roof(goz[0], goz[1], goz[2])
        times = {"fp64_gemm": g64[0], "tc_gemm": gtc[0], "oz_gemm": goz[0]}
        dominant = max(roofs, key=lambda k: times[k])
        roof = dict(roofs[dominant])
        roof["dominant_by_time"] = True
        other = [k for k in roofs if k != dominant]
        cpu = oracle_sample(cfg, seconds=args.cpu_seconds)
        line = {
            "metric": METRIC, "value": value, "unit": "sweeps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": dtype_of(args.precision),
            "data": "synthetic",
            "config": config_of(cfg, sweeps, args.precision, world),
            "tflops": flops * args.steps * world / (ms_max / 1e3) / 1e12,
            "roofline": roof,
            "roofline_other": {k: roofs[k] for k in other},
            "cpu_baseline": {"value": cpu["sweeps_per_s"], "unit": "sweeps/s", "cores": cpu["cores"],
                             "kind": "oracle",
                             "sample": f"{cpu['updates']} oracle local updates at the interior-site shape "
                                       f"(D=256, w=93, d=2; {cpu['t_update_s']:.2f} s each) scaled to one "
                                       f"evolve_step of the L=100 chain"},
            "e2e": {"value": e2e_val, "unit": "sweeps/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "parts_per_step": parts},
            "gpu_launches": launches,
            "obs_error": obs_err,
            "fp64_form": fp64_form,
            "other_forms": other_forms,
            "batched": batched,
            "clocks": clocks.summary(),
            "kernel_ms": {name: prof[c][0] for c, name in enumerate(PROF_NAMES)},
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def verify(args):
    """The target check: the full evolution to t = 5 (25 steps) in each form,
    observables against the oracle's stored values at every recorded step."""
    import torch
    import paper_2302_14181_gb300 as tv
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    cfg = wl.config(WORKLOAD)
    g = json.load(open(os.path.join(ROOT, "tests", "golden", WORKLOAD + ".json")))
    ctx = tv.Context()
    W = tv.mpo_build(ctx, *wl.model_blocks(cfg), cfg["N"], cfg["tau"])
    ops = list(wl.pauli())
    out = {"workload": WORKLOAD, "steps": cfg["steps"], "t": cfg["steps"] * abs(cfg["tau"]), "forms": {}}
    forms = args.verify_forms.split(",")
    for form in forms:
        prec = PREC[form]
        psi = tv.mps_init(ctx, wl.initial_vectors(cfg), cfg["D"])
        errs, t_total = {}, 0.0
        for k in range(1, cfg["steps"] + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            tv.evolve_step(psi, W, cfg["tau"], cfg["D"], cfg["sweeps"], prec)
            torch.cuda.synchronize()
            t_total += time.perf_counter() - t0
            if str(k) in g["steps"]:
                ref = np.array(g["steps"][str(k)])
                got = tv.measure_local(psi, ops).real
                errs[k] = float(np.abs(got - ref).max())
        out["forms"][form] = {"max_abs_obs_error_by_step": errs, "max_abs_obs_error": max(errs.values()),
                              "log_norm": psi.log_norm(), "log_norm_oracle": g["log_norm"][-1],
                              "seconds": t_total, "s_per_step": t_total / cfg["steps"]}
        print(json.dumps({"form": form, **out["forms"][form]}), flush=True)
    print(json.dumps(out), flush=True)


# ----------------------------------------------------------------------------
# small, fixed invocations for ncu captures (the commands in profiles/)
# ----------------------------------------------------------------------------

PROBES = ("kernels", "form", "fp64", "tc", "ozgemm", "qr", "batched", "twosite")


def oracle_step(args):
    """One full oracle evolve_step of the headline chain on the host cores (the
    thread count numpy's BLAS was started with: OPENBLAS_NUM_THREADS /
    OMP_NUM_THREADS), from the product state (the oracle's tensors have the
    workload's bond dimensions from the start, so every step costs the same).
    With --oracle-updates U > 0 only the right-environment build and the first U
    local updates of the first sweep are timed, and the step time is that
    per-update time times the step's updates (stated as extrapolated)."""
    from oracle import fit, mpo
    cfg = wl.config(WORKLOAD)
    L, D, sweeps = cfg["L"], cfg["D"], cfg["sweeps"]
    W = mpo.build_mpo(*wl.model_blocks(cfg), cfg["N"], cfg["tau"])
    psi = fit.product_mps(wl.initial_vectors(cfg), D)
    threads = int(os.environ.get("OPENBLAS_NUM_THREADS", os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)))
    line = {"impl": "oracle", "workload": WORKLOAD, "threads": threads, "host_cpus": os.cpu_count()}
    if args.oracle_updates <= 0:
        t0 = time.perf_counter()
        fit.evolve_step(psi, W, sweeps, canonical=False)
        dt = time.perf_counter() - t0
        line.update({"s_per_step": dt, "sweeps_per_s": sweeps / dt, "measured": "one full evolve_step"})
    else:
        # interior local updates (full bond dimension on both sides) on seeded
        # random operands of the step's shapes; the step is that time times its
        # updates (the environment build counted as 3/4 of an update each)
        rng = np.random.default_rng(7)
        w = W[L // 2].shape[0]
        cg = lambda *sh: (rng.standard_normal(sh) + 1j * rng.standard_normal(sh)) / math.sqrt(max(sh))
        El, A, Er = cg(D, w, D), cg(D, cfg["d"], D), cg(D, w, D)
        t1 = time.perf_counter()
        for _ in range(args.oracle_updates):
            fit._step_right(El, A, W[L // 2], Er)
        t_up = (time.perf_counter() - t1) / args.oracle_updates
        updates = sweeps * 2 * (L - 1) + 0.75 * (L - 1) + 1
        dt = t_up * updates
        line.update({"s_per_step": dt, "sweeps_per_s": sweeps / dt, "t_interior_update_s": t_up,
                     "measured": f"{args.oracle_updates} interior local updates (T build, apply, Householder QR, "
                                 f"environment); step = {updates:g} updates x that time (extrapolated)"})
    print(json.dumps(line), flush=True)


def splitting_study(args):
    """Sec. 8.3's comparison at scale: the XXZ chain (Neel start, D = 64) at
    L in {16, 64} and dt in {0.1, 0.2, 0.4}: 10 steps of the native order-2 MPO
    (bond 1 + chi + chi^2 = 13) against 10 pairs of order-1 MPOs at the complex
    steps dt (1 +- i)/2 (bond 1 + chi = 4 each), fp64 form, 2 sweeps per step.
    Reported per case: seconds per time step of each scheme (CUDA events), the
    log-norm change per step of each, and the largest log-norm of the first
    (amplifying, Re tau > 0) factor: the growth that truncation errors in
    high-energy components see between the two factors."""
    import torch
    import paper_2302_14181_gb300 as tv
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    ctx = tv.Context()
    stream = torch.cuda.current_stream()
    D, nsteps = 64, 10
    for L in (16, 64):
        blocks = wl.xxz_blocks(L, 0.5)
        v0 = wl.product_state("neel", L)
        for dt in (0.1, 0.2, 0.4):
            tau = -1j * dt
            taus = (tau * (1 + 1j) / 2, tau * (1 - 1j) / 2)
            W2 = tv.mpo_build(ctx, *blocks, 2, tau)
            W1 = [tv.mpo_build(ctx, *blocks, 1, x) for x in taus]
            out = {"L": L, "dt": dt, "D": D, "steps": nsteps, "w_native": W2.bond_dims()[L // 2],
                   "w_split": W1[0].bond_dims()[L // 2]}
            for name in ("native", "split"):
                psi = tv.mps_init(ctx, v0, D)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                first = []
                ln0 = psi.log_norm()
                for _ in range(nsteps):
                    if name == "native":
                        tv.evolve_step(psi, W2, tau, D, 2, tv.FP64)
                    else:
                        l0 = psi.log_norm()
                        tv.evolve_step(psi, W1[0], taus[0], D, 2, tv.FP64)
                        first.append(psi.log_norm() - l0)
                        tv.evolve_step(psi, W1[1], taus[1], D, 2, tv.FP64)
                e1.record(stream)
                torch.cuda.synchronize()
                out[name] = {"s_per_step": e0.elapsed_time(e1) / 1e3 / nsteps,
                             "log_norm_per_step": (psi.log_norm() - ln0) / nsteps}
                if first:
                    out[name]["first_factor_log_norm_max"] = max(first)
            print(json.dumps(out), flush=True)


def cylinder_study(args):
    """The paper's efficiency workload (Sec. 8.2) on a finite cylinder: the 2-D
    transverse-field Ising model, circumference 4 with spiral boundary
    conditions (chi = 4), length --cyl-Lx, g = 3.5 (paramagnetic side), bond
    dimension D. A ground state by imaginary time (60 steps of tau = -0.1, order
    3, from a seeded random state), the middle spin flipped, then evolution to
    T = 1 with step dt and MPO order N, against a reference with dt = 0.01 at
    order 3: the fidelity density f = log|<ref|psi>| / L and the wall time of
    each run (fp64 form, 2 sweeps per step)."""
    import torch
    import paper_2302_14181_gb300 as tv
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    ctx = tv.Context()
    Wc, Lx, g, D = 4, args.cyl_Lx, 3.5, args.cyl_D
    L = Wc * Lx
    blocks = wl.tfi_cylinder_blocks(Lx, Wc, g)
    X = wl.pauli()[0]
    plus = np.tile(np.array([1.0, 1.0], np.complex128) / math.sqrt(2), (L, 1))
    gs = tv.mps_init(ctx, plus, D)
    for i, a in enumerate(wl.random_mps(L, 2, D, seed=9)):
        gs.set_site(i, a)
    Wg = tv.mpo_build(ctx, *blocks, 3, -0.1)
    for _ in range(60):
        tv.evolve_step(gs, Wg, -0.1, D, 2, tv.FP64)
    sites = [gs.site(i) for i in range(L)]
    sites[L // 2] = np.einsum("st,atb->asb", X, sites[L // 2])

    def start():
        psi = tv.mps_init(ctx, plus, D)
        for i in range(L):
            psi.set_site(i, sites[i])
        return psi

    def run(N, dt):
        W = tv.mpo_build(ctx, *blocks, N, -1j * dt)
        psi = start()
        n = int(round(1.0 / dt))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(n):
            tv.evolve_step(psi, W, -1j * dt, D, 2, tv.FP64)
        torch.cuda.synchronize()
        return psi, time.perf_counter() - t0, W.bond_dims()[L // 2]

    ref, t_ref, _ = run(3, 0.01)
    print(json.dumps({"cylinder": f"W=4 x Lx={Lx}", "L": L, "D": D, "g": g, "reference": "N=3, dt=0.01",
                      "reference_s": t_ref}), flush=True)
    for N in (1, 2, 3):
        for dt in (0.25, 0.2, 0.1, 0.05):
            psi, secs, w = run(N, dt)
            la, _ = tv.mps_overlap(ref, psi)
            print(json.dumps({"N": N, "w": w, "dt": dt, "steps": int(round(1.0 / dt)), "seconds": secs,
                              "fidelity_density": la / L}), flush=True)


def c5_forms(args):
    """The spin-1 workload at full size (L = 128, D = 512, N = 4, d = 3, w = 160,
    tau = -0.25i, 2 sweeps): one time step in each form from the same state (the
    state after --warmup steps of the form every contraction as Ozaki-scheme
    GEMMs, so the bonds are populated), timed with CUDA events. The forms'
    accuracy at this size comes from the reduced run of the same chain
    (tests/test_gpu_c5.py)."""
    import torch
    import paper_2302_14181_gb300 as tv
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    cfg = wl.config("spin1_L128_N4_D512")
    tau, D = cfg["tau"], cfg["D"]
    ctx = tv.Context()
    W = tv.mpo_build(ctx, *wl.model_blocks(cfg), cfg["N"], tau)
    psi = tv.mps_init(ctx, wl.initial_vectors(cfg), D)
    for _ in range(args.warmup):
        tv.evolve_step(psi, W, tau, D, cfg["sweeps"], PREC["fp64+oz"])
    dims = psi.bond_dims()
    wd = W.bond_dims()
    flops = step_flops(dims, wd[:-1], wd[1:], cfg["d"], cfg["sweeps"])
    stream = torch.cuda.current_stream()
    out = {"workload": "spin1_L128_N4_D512", "L": cfg["L"], "D": D, "N": cfg["N"], "w": max(wd),
           "warmup_steps": args.warmup, "useful_tflop_per_step": flops / 1e12, "forms": {}}
    for name in args.c5_forms.split(","):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        tv.evolve_step(psi, W, tau, D, cfg["sweeps"], PREC[name])
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        out["forms"][name] = {"s_per_step": ms / 1e3, "sweeps_per_s": cfg["sweeps"] / (ms / 1e3),
                              "useful_tflops": flops / (ms / 1e3) / 1e12}
        print(json.dumps({"form": name, **out["forms"][name]}), flush=True)
    print(json.dumps(out), flush=True)


def probe(args):
    """One fixed workload per case, on the long-range Ising chain at length
    --probe-L (the per-site shapes of the L = 100 chain at its interior sites):
      kernels  every form of evolve_step once from the product state (fp64 with
               1 sweep; bf16x3, bf16x3 tensor-core only and bf16x3 + Ozaki with
               2), observables after each, then one overlap;
      form     two steps of the benchmark's form (every contraction as
               Ozaki-scheme GEMMs), 2 sweeps each;
      fp64     one fp64 step, 1 sweep;
      tc       one bf16x3 and one tf32x3 tensor-core-only step, each from the
               product state, with --probe-sweeps sweeps;
      ozgemm   the Ozaki-scheme GEMM alone at the interior-site shapes, timed
               with the library's events (kernel and slicing per launch);
      qr       two untimed steps of the benchmark's form, then three steps with
               the library's events on: QR factorisation and Q formation time
               per step and per call;
      batched  the first 8 chains of the batched workload, three batched steps
               (tensor-core tf32x3 contractions, fp64 QR one launch per column);
      twosite  one step of the two-site fit (fp64) on the XXZ chain L = 16,
               D = 64, order 3, from the Neel state."""
    import torch
    import paper_2302_14181_gb300 as tv
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    ctx = tv.Context()
    cfg = wl.config(WORKLOAD, L=args.probe_L)
    tau, D = cfg["tau"], cfg["D"]
    W = tv.mpo_build(ctx, *wl.model_blocks(cfg), cfg["N"], tau)
    v0 = wl.initial_vectors(cfg)
    X, _, Z = wl.pauli()
    case = args.probe
    if case == "kernels":
        psi = None
        for prec in (tv.FP64, tv.BF16X3, tv.BF16X3 | tv.TC_ONLY, tv.BF16X3 | tv.OZAKI):
            psi = tv.mps_init(ctx, v0, D)
            tv.evolve_step(psi, W, tau, D, 1 if prec == tv.FP64 else 2, prec)
            tv.measure_local(psi, [X, Z])
        print(json.dumps({"overlap": tv.mps_overlap(psi, tv.mps_init(ctx, v0, D))}))
    elif case == "form":
        psi = tv.mps_init(ctx, v0, D)
        for _ in range(2):
            tv.evolve_step(psi, W, tau, D, 2, PREC["fp64+oz"])
    elif case == "fp64":
        psi = tv.mps_init(ctx, v0, D)
        tv.evolve_step(psi, W, tau, D, 1, tv.FP64)
    elif case == "tc":
        for prec in (tv.BF16X3 | tv.TC_ONLY, tv.TF32X3 | tv.TC_ONLY):
            psi = tv.mps_init(ctx, v0, D)
            tv.evolve_step(psi, W, tau, D, args.probe_sweeps, prec)
    elif case == "ozgemm":
        w, d = W.bond_dims()[cfg["L"] // 2], cfg["d"]
        rng = np.random.default_rng(0)
        shapes = {"G1": (D * w, d * D, D), "G3": (d * D, D, w * D), "G3'": (D, w * D, d * D),
                  "G2": (w * d, D * D, w * d)}
        for name, (M, N, K) in shapes.items():
            A = torch.from_numpy(rng.standard_normal((M, K)) + 1j * rng.standard_normal((M, K))).cuda()
            B = torch.from_numpy(rng.standard_normal((N, K)) + 1j * rng.standard_normal((N, K))).cuda()
            C = torch.zeros((M, N), dtype=torch.complex128, device="cuda")
            tv.tevo_gemm(ctx, tv.OZAKI, A, B, C)                    # warm-up
            ctx.prof_enable(True)
            for c in (tv._lib.PROF_GEMMOZ, tv._lib.PROF_OZSPLIT):
                ctx.prof_read(c)
            for _ in range(5):
                tv.tevo_gemm(ctx, tv.OZAKI, A, B, C)
            kms, kn, kfl, _ = ctx.prof_read(tv._lib.PROF_GEMMOZ)
            sms, sn, _, _ = ctx.prof_read(tv._lib.PROF_OZSPLIT)
            ctx.prof_enable(False)
            print(json.dumps({"gemm": name, "M": M, "N": N, "K": K, "kernel_ms": kms / kn,
                              "executed_tflops": OZ_PAIRS * kfl / (kms / 1e3) / 1e12,
                              "slicing_ms": sms / max(1, sn)}), flush=True)
            del A, B, C
    elif case == "qr":
        psi = tv.mps_init(ctx, v0, D)
        for _ in range(2):
            tv.evolve_step(psi, W, tau, D, 2, PREC["fp64+oz"])
        torch.cuda.synchronize()
        ctx.prof_enable(True)
        for c in (tv._lib.PROF_QR, tv._lib.PROF_FORMQ):
            ctx.prof_read(c)
        t0 = time.perf_counter()
        for _ in range(3):
            tv.evolve_step(psi, W, tau, D, 2, PREC["fp64+oz"])
        torch.cuda.synchronize()
        step_s = (time.perf_counter() - t0) / 3
        qms, qn, _, _ = ctx.prof_read(tv._lib.PROF_QR)
        fms, fn, _, _ = ctx.prof_read(tv._lib.PROF_FORMQ)
        ctx.prof_enable(False)
        print(json.dumps({"step_s": step_s, "qr_ms_per_step": qms / 3, "qr_calls_per_step": qn / 3,
                          "qr_ms_per_call": qms / max(1, qn), "form_q_ms_per_step": fms / 3,
                          "form_q_ms_per_call": fms / max(1, fn)}), flush=True)
    elif case == "batched":
        chains = wl.batched_chains()[:8]
        bW = [tv.mpo_build(ctx, *wl.model_blocks(c), c["N"], c["tau"]) for c in chains]
        bps = [tv.mps_init(ctx, wl.initial_vectors(c), c["D"]) for c in chains]
        for _ in range(3):
            tv.evolve_step_batched(bps, bW, 1, PREC["tc-tf32x3"])
    elif case == "twosite":
        xc = wl.config("xxz_L64_N3", L=16, D=64)
        xW = tv.mpo_build(ctx, *wl.model_blocks(xc), xc["N"], xc["tau"])
        xp = tv.mps_init(ctx, wl.initial_vectors(xc), xc["D"])
        tv.evolve_step(xp, xW, xc["tau"], xc["D"], 1, tv.FP64 | tv.TWO_SITE)
    torch.cuda.synchronize()
    print(json.dumps({"probe": case, "L": cfg["L"], "launches": ctx.launch_count()}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default=os.environ.get("TEVO_BENCH_PRECISION", "fp64+oz"), choices=sorted(PREC))
    ap.add_argument("--no-fp64-compare", action="store_true",
                    help="skip the steps of the other forms timed beside the measured one")
    ap.add_argument("--sweeps", type=int, default=0)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--verify", action="store_true", help="run the t = 5 evolution in each form against the oracle")
    ap.add_argument("--verify-forms", default="fp64+oz,bf16x3+oz,bf16x3,fp64")
    ap.add_argument("--probe", choices=PROBES, help="run one fixed small workload (for ncu captures) instead")
    ap.add_argument("--probe-L", type=int, default=20)
    ap.add_argument("--probe-sweeps", type=int, default=1)
    ap.add_argument("--c5", action="store_true", help="time one step of each form on the full-size spin-1 chain")
    ap.add_argument("--oracle-step", action="store_true", help="time one full oracle step on the host cores")
    ap.add_argument("--splitting", action="store_true", help="complex-step splitting against the native order-2 MPO")
    ap.add_argument("--cylinder", action="store_true", help="fidelity density vs time step on the 2-D TFI cylinder")
    ap.add_argument("--cyl-Lx", type=int, default=8)
    ap.add_argument("--cyl-D", type=int, default=64)
    ap.add_argument("--oracle-updates", type=int, default=0)
    ap.add_argument("--c5-forms", default="fp64+oz,bf16x3+oz,bf16x3,fp64")
    args = ap.parse_args()
    if args.probe:
        probe(args)
        return
    if args.c5:
        c5_forms(args)
        return
    if args.oracle_step:
        oracle_step(args)
        return
    if args.splitting:
        splitting_study(args)
        return
    if args.cylinder:
        cylinder_study(args)
        return
    if args.verify:
        verify(args)
        return
    if args.impl == "reference":
        reference_arm(args)
    else:
        our_arm(args)


if __name__ == "__main__":
    main()
