"""Write the oracle's expected values for the named workloads into tests/golden/.

Calls only ``oracle`` and the seeded input module ``workloads``; nothing here
touches the CUDA library. Usage:

    python tests/golden/make_golden.py <workload> [--steps K] [--L L] [--D D] [--tag TAG]

For every recorded step the file holds <X_i>, <Y_i>, <Z_i> (real parts) for all
sites and the accumulated log-norm; the MPO bond dimension and the full workload
description are stored beside them.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads as wl  # noqa: E402
from oracle import fit, mpo  # noqa: E402


def ops_for(d):
    return list(wl.pauli()) if d == 2 else list(wl.spin_one())


def run(name, steps=None, record=None, tag=None, last_tau=None, **override):
    """Oracle evolution of a named workload; with last_tau the final step uses
    an MPO built at that time step (a total time that is not a multiple of tau:
    e.g. 12 steps of 0.4 and one of 0.2 reach t = 5)."""
    cfg = wl.config(name, **override)
    if steps is not None:
        cfg["steps"] = steps
    A, B, C, D = wl.model_blocks(cfg)
    W = mpo.build_mpo(A, B, C, D, cfg["N"], cfg["tau"])
    W_last = mpo.build_mpo(A, B, C, D, cfg["N"], last_tau) if last_tau is not None else W
    if last_tau is not None:
        cfg["last_tau"] = last_tau
    psi = fit.product_mps(wl.initial_vectors(cfg), cfg["D"])
    ops = ops_for(cfg["d"])
    record = set(record or range(1, cfg["steps"] + 1))
    out = {"workload": name, "config": {k: (v if not isinstance(v, complex) else [v.real, v.imag])
                                        for k, v in cfg.items() if k != "J"},
           "w": int(W[1].shape[0]) if len(W) > 2 else int(W[0].shape[3]),
           "source": "oracle (fp64, numpy) via tests/golden/make_golden.py",
           "steps": {}, "log_norm": []}
    logn = 0.0
    t0 = time.time()
    for k in range(1, cfg["steps"] + 1):
        Wk = W_last if k == cfg["steps"] else W
        psi, ln = fit.evolve_step(psi, Wk, cfg["sweeps"], canonical=(k > 1))
        logn += ln
        out["log_norm"].append(logn)
        if k in record:
            obs = fit.measure_local(psi, ops).real
            out["steps"][str(k)] = [list(map(float, row)) for row in obs]
        print(f"{name} step {k}/{cfg['steps']} log_norm {logn:.6e} t {time.time() - t0:.1f}s", flush=True)
    fn = os.path.join(HERE, f"{tag or name}.json")
    with open(fn, "w") as f:
        json.dump(out, f, indent=0)
    return out


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("workload")
    ap.add_argument("--steps", type=int)
    ap.add_argument("--record", type=str, help="comma-separated steps to record (default all)")
    ap.add_argument("--L", type=int)
    ap.add_argument("--D", type=int)
    ap.add_argument("--tau", type=float, help="imaginary part magnitude: tau = -i*value")
    ap.add_argument("--tag", type=str)
    ap.add_argument("--last-tau", type=float, help="time step of the final step: tau = -i*value")
    ap.add_argument("--sweeps", type=int)
    a = ap.parse_args()
    ov = {}
    if a.L:
        ov["L"] = a.L
    if a.D:
        ov["D"] = a.D
    if a.tau:
        ov["tau"] = -1j * a.tau
    if a.sweeps:
        ov["sweeps"] = a.sweeps
    rec = [int(x) for x in a.record.split(",")] if a.record else None
    run(a.workload, steps=a.steps, record=rec, tag=a.tag,
        last_tau=(-1j * a.last_tau) if a.last_tau else None, **ov)
