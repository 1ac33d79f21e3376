"""Record the oracle's full-solve iteration counts on the benchmark workloads (test infrastructure).

The CPU-baseline leg of the benchmark times a bounded sample of oracle iterations and scales it by
the number of iterations the oracle needs for the whole solve; that number comes from this script,
which calls only the oracle and the shared input generators, and writes full_solve_counts.json.

    python oracle/record_full_solves.py dense4096 8 16 32 cg
    python oracle/record_full_solves.py stencil27_96 16 cg
    python oracle/record_full_solves.py diffusion128 1 4 cg

With --band the script measures the oracle's rounding band instead: the same solve on the
rounding-level perturbations b(1 + 1e-16 u) of the right-hand side (workloads.perturbed_rhs,
k = 1..samples-1), run in parallel processes, stored under "band" beside the unperturbed record.
Past the exact-arithmetic termination bound an iteration count depends on summation order, and
the GPU parity test of the full-size configuration checks its count against this band.

    python oracle/record_full_solves.py --band --samples 12 --jobs 6 dense4096 32
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import oracle  # noqa: E402
import workloads as wl  # noqa: E402

OUT = os.path.join(HERE, "full_solve_counts.json")


def load_workload(name):
    if name == "dense4096":
        return wl.dense_spd(4096, 0), 0, 1e-8
    if name == "poisson64":
        return wl.poisson2d(64), 0, 1e-8
    if name == "stencil27_96":
        return wl.stencil27(96, 0), 0, 1e-10
    if name == "diffusion128":
        return wl.diffusion3d(128, 0), 1, 1e-8
    raise SystemExit(f"unknown workload {name}")


def solve_once(name, v, k):
    """One oracle solve of workload `name`, variant `v` ("cg" or s), right-hand side perturbation k."""
    A, precond, tol = load_workload(name)
    b = wl.perturbed_rhs(wl.rhs(A.n, 0), k)
    t0 = time.time()
    if v == "cg":
        _, info = oracle.cg_cgear(A, b, precond=precond, tol=tol)
    else:
        s = int(v)
        _, _, info = oracle.mbpcg(A, b, wl.initial_block(A.n, s, 1), precond=precond, tol=tol)
    return dict(info, seconds=time.time() - t0, tol=tol, precond=precond, perturbation=k)


def store(name, v, update):
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    rec = data.setdefault(name, {}).setdefault(v, {})
    update(rec)
    tmp = OUT + f".tmp{os.getpid()}"
    json.dump(data, open(tmp, "w"), indent=1, sort_keys=True)
    os.replace(tmp, OUT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--band", action="store_true")
    ap.add_argument("--samples", type=int, default=12)
    ap.add_argument("--jobs", type=int, default=max(1, (os.cpu_count() or 2) - 2))
    ap.add_argument("name")
    ap.add_argument("variants", nargs="+")
    a = ap.parse_args()
    for v in a.variants:
        if not a.band:
            rec = solve_once(a.name, v, 0)
            rec.pop("perturbation")
            store(a.name, v, lambda r: r.update(rec))
            print(a.name, v, rec, flush=True)
            continue
        # spawn: the oracle library is loaded afresh in each worker process
        have = json.load(open(OUT)).get(a.name, {}).get(v) if os.path.exists(OUT) else None
        first = 1 if have and "iterations" in have else 0
        with mp.get_context("spawn").Pool(a.jobs) as pool:
            recs = pool.starmap(solve_once, [(a.name, v, k) for k in range(first, a.samples)])
        if first == 0:
            base = dict(recs.pop(0))
            base.pop("perturbation")
            store(a.name, v, lambda r: r.update(base))
        else:
            base = have
        its = [base["iterations"]] + [r["iterations"] for r in recs]
        band = {"samples": len(its), "iterations": its, "lo": min(its), "hi": max(its),
                "statuses": [base["status"]] + [r["status"] for r in recs],
                "restarts": [base["restarts"]] + [r["restarts"] for r in recs],
                "perturbation": "b (1 + 1e-16 u), u ~ U(-1,1) from seed k, stream 7000, k = 1..%d"
                                % (a.samples - 1)}
        store(a.name, v, lambda r: r.__setitem__("band", band))
        print(a.name, v, "band", band, flush=True)


if __name__ == "__main__":
    main()
