"""Record the oracle's full-solve iteration counts on the benchmark workloads (test infrastructure).

The CPU-baseline leg of the benchmark times a bounded sample of oracle iterations and scales it by
the number of iterations the oracle needs for the whole solve; that number comes from this script,
which calls only the oracle and the shared input generators, and writes full_solve_counts.json.

    python oracle/record_full_solves.py dense4096 8 16 32 cg
    python oracle/record_full_solves.py stencil27_96 16 cg
"""
from __future__ import annotations

import json
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
    raise SystemExit(f"unknown workload {name}")


def main():
    name, variants = sys.argv[1], sys.argv[2:]
    A, precond, tol = load_workload(name)
    b = wl.rhs(A.n, 0)
    for v in variants:
        t0 = time.time()
        if v == "cg":
            _, info = oracle.cg_cgear(A, b, precond=precond, tol=tol)
        else:
            s = int(v)
            _, _, info = oracle.mbpcg(A, b, wl.initial_block(A.n, s, 1), precond=precond, tol=tol)
        rec = dict(info, seconds=time.time() - t0, tol=tol, precond=precond)
        data = json.load(open(OUT)) if os.path.exists(OUT) else {}
        data.setdefault(name, {})[v] = rec
        tmp = OUT + f".tmp{os.getpid()}"
        json.dump(data, open(tmp, "w"), indent=1, sort_keys=True)
        os.replace(tmp, OUT)
        print(name, v, rec, flush=True)


if __name__ == "__main__":
    main()
