"""Benchmark: MBPCG time-to-solution (relative residual 1e-8) against Chronopoulos-Gear CG from the
same library, on one GB300.

A step is one full MBPCG solve of the workload (set-up, every Algorithm 1 iteration, the
least-squares exit and the true-residual check). Default workload: the dense SPD system
n = 4096, A = Q diag(lambda) Q^T with lambda log-uniform in [1, 1e6], FP64, s copies.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--s S] [--workload NAME]
    python bench.py --impl reference ...   (the FP64 CPU oracle, timed on the host cores)

Prints one JSON line (rank 0). Under torchrun each rank solves its own replica (the solve does
not shard across GPUs here; replicas only), the step time is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as wl  # noqa: E402

METRIC = "MBPCG time-to-relres 1e-8 vs plain CG, 1 GB300; SpMM HBM roofline %; p99 latency"
UNIT = "ms"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "traffic.json")
L2_FLUSH_BYTES = 256 << 20
# FP64 peak of GB300 from unit counts and clock: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12  # FP32 FMA pipe (no tensor cores)

WORKLOADS = {
    "dense4096": dict(desc="dense SPD n=4096, A=Q diag(lambda) Q^T, lambda=10^U[0,6], b,U~U(-1,1), FP64, tol 1e-8",
                      precond=0, tol=1e-8, s=32, precision="tc",
                      mixed_desc="dense SPD n=4096, A=Q diag(lambda) Q^T, lambda=10^U[0,6], b,U~U(-1,1); FP32 A and "
                                 "blocks with FP32 accumulation, FP64-class Grams, FP64 k x k and FP64 refinement "
                                 "to relres 1e-10", mixed_tol=1e-10),
    "dense4096_k1e4": dict(desc="dense SPD n=4096, A=Q diag(lambda) Q^T, lambda=10^U[0,4], b,U~U(-1,1), FP64, "
                                "tol 1e-8", precond=0, tol=1e-8, s=32, precision="tc",
                           mixed_desc="dense SPD n=4096, A=Q diag(lambda) Q^T, lambda=10^U[0,4], b,U~U(-1,1); FP32 A "
                                      "and blocks with FP32 accumulation, FP64-class Grams, FP64 k x k and FP64 "
                                      "refinement to relres 1e-10", mixed_tol=1e-10),
    "poisson64": dict(desc="2D 5-point Poisson 64x64 (n=4096, nnz=20224), CSR int32/FP64, tol 1e-8",
                      precond=0, tol=1e-8, s=4),
    "diffusion128": dict(desc="3D 7-point variable-coefficient diffusion 128^3 (n=2097152, nnz=14581760), "
                              "Jacobi scaling, tol 1e-8", precond=1, tol=1e-8, s=4),
    "stencil27_96": dict(desc="3D 27-point stencil 96^3 (n=884736, nnz=23393656), off-diagonals -U[0,1) per edge, "
                              "diagonal sum|off|+1e-2; FP32 blocks/SpMM with FP32 accumulation, FP64-class Grams, "
                              "FP64 k x k and FP64 refinement to relres 1e-10", precond=0, tol=1e-10, s=16,
                         precision="mixed"),
}


def make_matrix(name):
    if name == "dense4096":
        return wl.dense_spd(4096, 0)
    if name == "dense4096_k1e4":
        return wl.dense_spd(4096, 0, 0.0, 4.0)
    if name == "poisson64":
        return wl.poisson2d(64)
    if name == "diffusion128":
        return wl.diffusion3d(128, 0)
    if name == "stencil27_96":
        return wl.stencil27(96, 0)
    raise SystemExit(f"unknown workload {name}")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="dense4096", choices=sorted(WORKLOADS) + ["serving", "batch"])
    p.add_argument("--batch-size", type=int, default=32, help="batch: uneven systems solved per step")
    p.add_argument("--requests", type=int, default=2000, help="serving: requests in the stream")
    p.add_argument("--slots", type=int, default=8, help="serving: solves admitted at once")
    p.add_argument("--compare-requests", type=int, default=400,
                   help="serving: requests of the same stream also served one at a time (0: skip)")
    p.add_argument("--s", type=int, default=None)
    p.add_argument("--kernel-launches", type=int, default=20, help="launches of the dominant kernel timed alone")
    p.add_argument("--cpu-sample-iters", type=int, default=6)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-sweep", action="store_true", help="skip the sweep of s on the dense tensor-core workload")
    p.add_argument("--no-spmm-roofline", action="store_true",
                   help="skip the SpMM HBM roofline (diffusion 128^3 at s = 1, 4 in FP64; 27-point 96^3 at s = 16 in FP32)")
    p.add_argument("--precision", default=None, choices=["fp64", "tc", "mixed"],
                   help="tc: dense product on the FP16 tensor cores by exact digit splitting (FP64 accuracy); "
                        "mixed: FP32 inner solves in FP64 refinement (CSR); default: the workload's own")
    p.add_argument("--residual", default="explicit", choices=["explicit", "implicit"],
                   help="implicit: the loop carries R = W Sigma instead of updating R (MBPCG_RESIDUAL_IMPLICIT)")
    p.add_argument("--launch-mode", default="graph", choices=["graph", "eager"],
                   help="eager: host-launched loop (for profilers; same kernels and results)")
    return p.parse_args()


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.dev)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.3)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


KERNEL_SOURCES = {
    "k_dense": ("row_kernels.cuh", "mbpcg_device.cuh"),
    "k_spmm": ("row_kernels.cuh", "mbpcg_device.cuh"),
    "k_dense_tc": ("ozaki_tc.cu", "ozaki_digits.cuh", "int_to_fp64.cuh", "tcgen05.cuh", "tma.cuh", "mbpcg_device.cuh"),
}


def kernel_source_hash(kernel):
    """Hash of the sources a recorded ncu traffic figure was taken from (stale figures are dropped)."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        h.update(open(os.path.join(ROOT, "paper_2608_07327_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel, workload, s):
    try:
        data = json.load(open(PROFILE_TRAFFIC))
    except (OSError, ValueError):
        return None
    rec = data.get(f"{kernel}:{workload}:s{s}")
    if not rec or rec.get("source_hash") != kernel_source_hash(kernel):
        return None
    return rec.get("dram_bytes_per_launch")


def l2_flush(flush):
    """Leave L2 cold and clean: write the first half of `flush` (each half larger than L2), then read
    the second half, so that the written lines are evicted -- and written back -- before the timed
    region instead of during it."""
    h = flush.numel() // 2
    flush[:h].zero_()
    flush[h:].sum()


def read_ceiling_gbs(stream, flush):
    """HBM read-only bandwidth of this GPU right now: a sum over a 1 GiB FP32 tensor (torch's own
    reduction), L2 flushed before each run. A read-only stream does not reach the copy bandwidth
    of MEASURED_PEAKS.json; this is the ceiling of the kernels that only read A."""
    import torch
    x = torch.ones(1 << 28, dtype=torch.float32, device=flush.device)
    out = torch.empty((), dtype=torch.float32, device=flush.device)
    ts = []
    with torch.cuda.stream(stream):
        for i in range(6):
            l2_flush(flush)
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            torch.sum(x, dim=0, out=out)
            ev1.record(stream)
            ev1.synchronize()
            if i >= 2:
                ts.append(ev0.elapsed_time(ev1))
    del x
    return 4 * (1 << 28) / (statistics.median(ts) * 1e-3) / 1e9


BODY_UNROLL = 4  # loop iterations per pass of the library's graph loop (the passes end on whole bodies)


def launches_per_solve(info, dense, algo_cg, tc=False, mixed=False, cg_fused=False):
    """Kernels of ours launched by one solve call (the counter of the graph the library builds). The
    tensor-core dense product is four kernels (column exponents, digits of P, MMAs, split sum); the
    mixed-precision loop runs its Gram as a kernel of its own; dense CG runs one kernel per
    iteration. The graph loop runs whole passes of BODY_UNROLL iterations, so up to BODY_UNROLL - 1
    bodies after the stop launch and return at once: counted here as launched (an upper bound)."""
    inner = info["restarts"] + 1
    if algo_cg:
        setup, exit_, body = 3, 5, (1 if cg_fused else 5)
    else:
        setup, exit_, body = 8, 7, (8 if (dense or mixed) else 7)
        if tc:
            setup, body = setup + 3, body + 3
    bodies = info["iterations"] + (BODY_UNROLL - 1) * inner
    return inner * (1 + setup + exit_) + body * bodies + (0 if algo_cg else 1)


def spmm_roofline(mb, stream, flush, peak_gbs, launches=10):
    """HBM roofline of the CSR product A P alone, by the solver's own product kernel (the one the
    handle picked at create) through mbpcg_apply_dev, on the two sparse workloads
    where HBM binds: 3D diffusion 128^3 (Jacobi, FP64, s = 1 and s = 4) and the 27-point stencil 96^3
    (the FP32 product of the mixed inner solve, s = 16). Algorithmic bytes: the CSR once (12 nnz +
    4 (n + 1) in FP64, 8 nnz + 4 (n + 1) in FP32) plus P in and A P out (2 n KP values), whichever
    kernel runs (the tiled kernel reads 16-bit local column indices, 2 bytes per nonzero less); L2
    flushed before every launch; CUDA events on the handle's stream."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    names = {mb.MBPCG_PRODUCT_CSR_GATHER: "k_spmm (gather)", mb.MBPCG_PRODUCT_CSR_TILED: "k_spmm_tiled",
             mb.MBPCG_PRODUCT_CSR_WIDE: "k_spmm_wide_f"}
    cases = []
    for name, gen, s, f32, precond in (("3D 7-point diffusion 128^3", lambda: wl.diffusion3d(128, 0), 1, False, 1),
                                       ("3D 7-point diffusion 128^3", lambda: wl.diffusion3d(128, 0), 4, False, 1),
                                       ("3D 27-point stencil 96^3", lambda: wl.stencil27(96, 0), 16, True, 0)):
        A = gen()
        n, nnz = A.n, A.nnz
        kp = mb.mbpcg_k_padded_width(s)
        sv = mb.Solver(A, s=s, precond=precond, precision=mb.MBPCG_MIXED_FP32 if f32 else mb.MBPCG_FP64)
        try:
            kernel, times64 = sv.product_kernel(fp32=f32)
            dt = torch.float32 if f32 else torch.float64
            P = torch.zeros((n, kp), dtype=dt, device=dev)
            P[:, :s] = torch.as_tensor(wl.initial_block(n, s, 1), device=dev).to(dt)
            AP = torch.empty_like(P)
            if f32:
                nbytes, prec = 8.0 * nnz + 4.0 * (n + 1) + 8.0 * n * kp, "FP32"
                unroll, cps, tf = sv.spmm_tuning()
                tuning = {"shape": [unroll, cps], "times_us": [round(t, 2) for t in tf]}
            else:
                nbytes, prec = 12.0 * nnz + 4.0 * (n + 1) + 16.0 * n * kp, "FP64"
                tuning = {"times_us_gather_tiled": [round(t, 2) for t in times64]}
            ss = sv.stream
            ss.wait_stream(torch.cuda.current_stream())
            launch = lambda: mb.mbpcg_apply_dev(sv.h, 1 if f32 else 0, P, AP)  # noqa: E731
            ts = []
            with torch.cuda.stream(ss):
                if launch() != 0:
                    raise RuntimeError("mbpcg_apply_dev failed")
                for _ in range(launches):
                    l2_flush(flush)
                    ev0 = torch.cuda.Event(enable_timing=True)
                    ev1 = torch.cuda.Event(enable_timing=True)
                    ev0.record(ss)
                    launch()
                    ev1.record(ss)
                    ev1.synchronize()
                    ts.append(ev0.elapsed_time(ev1))
            ms = sum(ts) / len(ts)
            gbs = nbytes / (ms * 1e-3) / 1e9
            cases.append({"workload": name, "n": n, "nnz": int(nnz), "s": s,
                          "kernel": f"{names.get(kernel, kernel)}<{kp}> ({prec})", "autotune": tuning,
                          "kernel_ms": round(ms, 5), "algorithmic_bytes": nbytes, "achieved": round(gbs, 1),
                          "frac": round(gbs / peak_gbs, 4)})
            del P, AP
        finally:
            sv.close()
    return {"bound": "hbm", "unit": "GB/s", "peak": peak_gbs, "cases": cases,
            "timing": f"{launches} launches, L2 flushed before each (256 MB written, then another 256 MB read, so "
                      "no write-back falls in the timed launch), CUDA events on the stream",
            "peak_note": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"}


def roofline_tc(n, s, kp, k_ms, single_ms, seq_ms, read_gbs, peaks, traffic, launches):
    """Roofline of k_dense_tc, the MMA kernel of the tensor-core product (k_ms: its average
    duration over `launches` back-to-back launches). Algorithmic bytes are those of the dense
    product itself: FP64 A read once (8 n^2), P in and A P out (16 n KP). The kernel streams A as its
    8 signed base-128 digits, one byte each (8 n^2 bytes, as many as the FP64 matrix), and the
    digits of P; the fraction is reported against the measured copy bandwidth and against the
    read-only ceiling `read_gbs` (a kernel that only reads)."""
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    nbytes = 8.0 * n * n + 16.0 * n * kp
    flops = 2.0 * n * n * s
    achieved_gbs = nbytes / (k_ms * 1e-3) / 1e9
    return {"bound": "hbm", "kernel": f"k_dense_tc<{kp}> (digit stream of A + tcgen05 MMAs, the kernel alone)",
            "achieved": round(achieved_gbs, 1), "peak": hbm_peak, "unit": "GB/s",
            "frac": round(achieved_gbs / hbm_peak, 4), "traffic": traffic,
            "kernel_ms": round(k_ms, 5), "algorithmic_bytes": nbytes, "algorithmic_flops": flops,
            "fp64_equiv_tflops": round(flops / (k_ms * 1e-3) / 1e12, 3),
            "traffic_note": "DRAM bytes of one launch: A's digits (8 B per entry, the same as FP64 A) "
                            "plus P's digits and the raw partials",
            "timing": f"{launches} back-to-back launches (digits of A > L2, no flush)",
            "kernel_ms_one_launch_l2_flushed": round(single_ms, 5),
            "product_call_ms": round(seq_ms, 5),
            "product_call_frac": round(nbytes / (seq_ms * 1e-3) / 1e9 / hbm_peak, 4),
            "read_ceiling_gbs": round(read_gbs, 1), "frac_of_read_ceiling": round(achieved_gbs / read_gbs, 4),
            "peak_note": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)" if peaks else "fallback"}


def max_over_ranks(values, world, device=None):
    """Element-wise maximum of per-rank step timings over all ranks (the values as given at world
    size 1). Every rank calls it at the same point; the tensor lives on `device` (a CUDA device
    under NCCL, None for the CPU under gloo)."""
    if world <= 1:
        return [float(v) for v in values]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def resolve_precision(args, cfg, dense):
    """Name of the arithmetic a run uses: "tc" (dense only), "mixed" or "fp64"."""
    pname = args.precision or cfg.get("precision", "fp64")
    if pname == "tc" and not dense:
        pname = "fp64"
    return pname if pname in ("tc", "mixed") else "fp64"


def bench_config(args, cfg, A, s, pname, world):
    """The "config" object of the JSON line (the same for this library's arm and the reference arm)."""
    mixed = pname == "mixed"
    return {"workload": cfg.get("mixed_desc", cfg["desc"]) if mixed else cfg["desc"], "n": int(A.n),
            "nnz": int(A.nnz), "s": s, "precond": cfg["precond"],
            "tol": cfg.get("mixed_tol", cfg["tol"]) if mixed else cfg["tol"],
            "l2": "flushed before every step (256 MB written, then 256 MB read)", "launch_mode": args.launch_mode, "precision": pname,
            "residual": args.residual, "parallelism": "replicas only" if world > 1 else "single GPU"}


def run_ours(args, world, rank, local):
    import torch
    import paper_2608_07327_gb300 as mb

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    cfg = WORKLOADS[args.workload]
    s = args.s or cfg["s"]
    A = make_matrix(args.workload)
    dense = isinstance(A, wl.Dense)
    n = A.n
    b = wl.rhs(n, 0)
    U = wl.initial_block(n, s, 1)
    dev = torch.device("cuda", local)
    mode = mb.MBPCG_LAUNCH_EAGER if args.launch_mode == "eager" else mb.MBPCG_LAUNCH_GRAPH
    pname = resolve_precision(args, cfg, dense)
    prec = {"tc": mb.MBPCG_FP64_TC, "mixed": mb.MBPCG_MIXED_FP32}.get(pname, mb.MBPCG_FP64)
    mixed = prec == mb.MBPCG_MIXED_FP32
    # the mixed configuration of a workload may have its own tolerance (refinement to 1e-10)
    tol = cfg.get("mixed_tol", cfg["tol"]) if mixed else cfg["tol"]
    desc = cfg.get("mixed_desc", cfg["desc"]) if mixed else cfg["desc"]
    rmode = mb.MBPCG_RESIDUAL_IMPLICIT if args.residual == "implicit" else mb.MBPCG_RESIDUAL_EXPLICIT
    solver = mb.Solver(A, s=s, precond=cfg["precond"], launch_mode=mode, precision=prec, residual_mode=rmode)
    # the FP64 solve the mixed one is compared with: the fastest FP64 path (tensor cores for dense A)
    fp64 = (mb.Solver(A, s=s, precond=cfg["precond"], launch_mode=mode,
                      precision=mb.MBPCG_FP64_TC if dense else mb.MBPCG_FP64) if mixed else None)
    cg = mb.Solver(A, algo=mb.MBPCG_ALGO_CG, precond=cfg["precond"], launch_mode=mode)
    stream = solver.stream
    bd = torch.as_tensor(b, device=dev)
    Ud = torch.as_tensor(np.asfortranarray(U).ravel(order="F"), device=dev)
    flush = torch.zeros(2 * L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def timed(sv, Uarg, k):
        times, infos, xs = [], [], None
        for _ in range(k):
            with torch.cuda.stream(sv.stream):
                l2_flush(flush)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(sv.stream)
            x, info = sv.solve(bd, Uarg, tol=tol, maxit=400000)
            e1.record(sv.stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            infos.append(info)
            xs = x
        return times, infos, xs

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()

    timed(solver, Ud, args.warmup)
    timed(cg, None, max(1, min(args.warmup, 2)))
    if fp64 is not None:
        timed(fp64, Ud, 1)
    barrier()
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        times, infos, x = timed(solver, Ud, args.steps)
        barrier()
        wall = time.perf_counter() - t0
        cg_times, cg_infos, xc = timed(cg, None, args.steps)
        barrier()
        if fp64 is not None:
            f_times, f_infos, xf = timed(fp64, Ud, max(1, min(args.steps, 2)))
            barrier()
    once = None
    if dense and prec == mb.MBPCG_FP64_TC and world == 1:
        # the same solves with the tensor-core product rounded once (levels 5..8 exact), after the
        # timed region of the headline: an option beside the default, not the headline
        solver.set_product_rounding(mb.MBPCG_ROUND_ONCE)
        timed(solver, Ud, 1)
        o_times, o_infos, _ = timed(solver, Ud, args.steps)
        solver.set_product_rounding(mb.MBPCG_ROUND_FP32_TAIL)
        once = {"ms": round(sum(o_times) / len(o_times), 4), "iterations": o_infos[-1]["iterations"],
                "restarts": o_infos[-1]["restarts"], "relres_true": o_infos[-1]["relres_true"]}
    sweep = None
    if dense and prec == mb.MBPCG_FP64_TC and world == 1 and not args.no_sweep:
        # the configuration's sweep of s on the same system: one warm-up and one timed solve each
        sweep = {}
        for sw in (1, 2, 4, 8, 16, 32):
            if sw == s:
                sweep[str(sw)] = {"ms": round(sum(times) / len(times), 4), "iterations": infos[-1]["iterations"]}
                continue
            svw = mb.Solver(A, s=sw, precond=cfg["precond"], launch_mode=mode, precision=prec)
            try:
                Uw = torch.as_tensor(np.asfortranarray(wl.initial_block(A.n, sw, 1)).ravel(order="F"), device=dev)
                timed(svw, Uw, 1)
                w_times, w_infos, _ = timed(svw, Uw, 1)
                sweep[str(sw)] = {"ms": round(w_times[0], 4), "iterations": w_infos[-1]["iterations"],
                                  "restarts": w_infos[-1]["restarts"]}
            finally:
                svw.close()
    total_ms = sum(times)
    cg_total = sum(cg_times)
    total_ms, cg_total = max_over_ranks([total_ms, cg_total], world, dev)
    ms_per_step = total_ms / args.steps
    cg_ms = cg_total / args.steps
    info = infos[-1]
    xh = x.cpu().numpy()
    Amul = (lambda v: np.asarray(A.a) @ v) if dense else (lambda v: A.to_scipy() @ v)
    relres_check = float(np.linalg.norm(b - Amul(xh)) / np.linalg.norm(b))

    # dominant kernel alone, same launch configuration, CUDA events on its stream
    kp = mb.mbpcg_k_padded_width(s)
    P = torch.as_tensor(np.ascontiguousarray(np.pad(U, ((0, 0), (0, kp - s)))), device=dev)
    AP = torch.empty_like(P)
    tc = dense and prec == mb.MBPCG_FP64_TC
    launch_gram = None
    kstream = stream
    if dense and mixed:
        Ad = torch.as_tensor(np.asfortranarray(A.a).ravel(order="F"), device=dev)
        ftb = mb.mbpcg_k_dense_f32_bytes(n)
        ftiles = torch.empty(ftb // 4, dtype=torch.float32, device=dev)
        mb.mbpcg_k_dense_f32_prepare(n, Ad, ftiles, ftb, stream.cuda_stream)  # FP32 tiles of A, once
        P = P.float()
        AP = torch.empty_like(P)
        launch = lambda: mb.mbpcg_k_dense_f32(n, ftiles, s, P, AP, stream.cuda_stream)  # noqa: E731
        kname = "k_dense_f"
        flops = 2.0 * n * n * s
        nbytes = 4.0 * n * n + 8.0 * n * kp  # FP32 A read once, P in, AP out
    elif tc:
        Ad = torch.as_tensor(np.asfortranarray(A.a).ravel(order="F"), device=dev)
        tcb = mb.mbpcg_k_dense_tc_scratch_bytes(n, s)
        tcs = torch.empty(tcb, dtype=torch.uint8, device=dev)
        mb.mbpcg_k_dense_tc_prepare(n, Ad, s, tcs, tcb, stream.cuda_stream)  # digits of A, once
        # the whole product (column exponents and digits of P, MMAs, split sum), and its MMA kernel
        # alone on the digits of P the product leaves in scratch: the dominant kernel of an iteration
        launch_seq = lambda: mb.mbpcg_k_dense_tc_product(n, s, P, AP, tcs, tcb, stream.cuda_stream)  # noqa: E731
        with torch.cuda.stream(stream):
            launch_seq()
        launch = lambda: mb.mbpcg_k_dense_tc_mma(n, s, tcs, tcb, stream.cuda_stream)  # noqa: E731
        kname = "k_dense_tc"
        flops = 2.0 * n * n * s
        nbytes = 8.0 * n * n + 16.0 * n * kp  # algorithmic: FP64 A read once, P in, AP out
    elif dense:
        Ad = torch.as_tensor(np.asfortranarray(A.a).ravel(order="F"), device=dev)
        launch = lambda: mb.mbpcg_k_dense_product(n, Ad, s, P, AP, stream.cuda_stream)  # noqa: E731
        kname = "k_dense"
        flops = 2.0 * n * n * s
        nbytes = 8.0 * n * n + 16.0 * n * kp
    elif mixed:
        rp = torch.as_tensor(A.row_ptr, device=dev)
        ci = torch.as_tensor(A.col_idx, device=dev)
        av = torch.as_tensor(A.val.astype(np.float32), device=dev)
        P = P.float()
        AP = torch.empty_like(P)
        # the solver's own FP32 product (the shape its autotuner kept), on the solver's stream
        kstream = solver.stream
        launch = lambda: mb.mbpcg_apply_dev(solver.h, 1, P, AP)  # noqa: E731
        kname = "k_spmm_wide_f" if solver.product_kernel(fp32=True)[0] == mb.MBPCG_PRODUCT_CSR_WIDE else "k_spmm_f"
        flops = 2.0 * A.nnz * s
        nbytes = 8.0 * A.nnz + 4.0 * (n + 1) + 8.0 * n * kp  # FP32 values + int32 indices, P in, AP out
        gb = mb.mbpcg_k_scratch_bytes(n, s)
        gscr = torch.empty(gb, dtype=torch.uint8, device=dev)
        Gd = torch.empty((s, s), dtype=torch.float64, device=dev)
        launch_gram = lambda: mb.mbpcg_k_spmm_gram_f32(n, rp, ci, av, s, P, AP, Gd, gscr, gb,  # noqa: E731
                                                       stream.cuda_stream)
    else:
        # the solver's own FP64 product (the scaled matrix under Jacobi), on the solver's stream
        kstream = solver.stream
        launch = lambda: mb.mbpcg_apply_dev(solver.h, 0, P, AP)  # noqa: E731
        kname = "k_spmm"
        flops = 2.0 * A.nnz * s
        nbytes = 12.0 * A.nnz + 4.0 * (n + 1) + 16.0 * n * kp
    kstream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(kstream):
        for _ in range(3):
            launch()
        k_ms = []
        for _ in range(args.kernel_launches):
            l2_flush(flush)
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(kstream)
            launch()
            ev1.record(kstream)
            ev1.synchronize()
            k_ms.append(ev0.elapsed_time(ev1))
    k_avg = sum(k_ms) / len(k_ms)
    achieved_tflops = flops / (k_avg * 1e-3) / 1e12
    seq_ms = None
    single_ms = None
    if tc:
        # k_dense_tc reads 268 MB of digits, more than L2 (129 MB): timed as back-to-back launches,
        # no flush in between, so the launch latency of one launch hides behind the previous one
        with torch.cuda.stream(stream):
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            for _ in range(args.kernel_launches):
                launch()
            ev1.record(stream)
            ev1.synchronize()
        single_ms, k_avg = k_avg, ev0.elapsed_time(ev1) / args.kernel_launches
        achieved_tflops = flops / (k_avg * 1e-3) / 1e12
        with torch.cuda.stream(stream):
            q_ms = []
            for _ in range(max(3, args.kernel_launches // 2)):
                l2_flush(flush)
                ev0 = torch.cuda.Event(enable_timing=True)
                ev1 = torch.cuda.Event(enable_timing=True)
                ev0.record(stream)
                launch_seq()
                ev1.record(stream)
                ev1.synchronize()
                q_ms.append(ev0.elapsed_time(ev1))
        seq_ms = sum(q_ms) / len(q_ms)
    gram_ms = None
    if launch_gram is not None:
        with torch.cuda.stream(stream):
            g_ms = []
            for _ in range(max(3, args.kernel_launches // 2)):
                l2_flush(flush)
                ev0 = torch.cuda.Event(enable_timing=True)
                ev1 = torch.cuda.Event(enable_timing=True)
                ev0.record(stream)
                launch_gram()
                ev1.record(stream)
                ev1.synchronize()
                g_ms.append(ev0.elapsed_time(ev1))
        gram_ms = sum(g_ms) / len(g_ms)
    read_gbs = read_ceiling_gbs(stream, flush) if (mixed or tc) else None
    if mixed and dense:
        # FP32 A P on the CUDA cores: 16 flop per byte of A at KP = 32, at the FP32 ridge of this GPU;
        # the roof with the higher utilisation is the one that binds
        peaks = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}
        hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
        achieved_gbs = nbytes / (k_avg * 1e-3) / 1e9
        flops_pad = 2.0 * n * n * kp  # the kernel computes all KP columns
        fp32_tflops = flops_pad / (k_avg * 1e-3) / 1e12
        alu = fp32_tflops / FP32_PEAK_TFLOPS > achieved_gbs / hbm_peak
        roofline = {"bound": "alu" if alu else "hbm",
                    "kernel": f"{kname}<{kp}> (FP32 dense A P on the CUDA cores, the product alone)",
                    "achieved": round(fp32_tflops if alu else achieved_gbs, 3 if alu else 1),
                    "peak": round(FP32_PEAK_TFLOPS, 2) if alu else hbm_peak, "unit": "TFLOP/s" if alu else "GB/s",
                    "frac": round(fp32_tflops / FP32_PEAK_TFLOPS if alu else achieved_gbs / hbm_peak, 4),
                    "traffic": recorded_traffic(kname, args.workload, s),
                    "kernel_ms": round(k_avg, 5), "algorithmic_bytes": nbytes, "algorithmic_flops": flops_pad,
                    "hbm_gbs": round(achieved_gbs, 1), "hbm_frac": round(achieved_gbs / hbm_peak, 4),
                    "fp32_tflops": round(fp32_tflops, 3), "fp32_frac": round(fp32_tflops / FP32_PEAK_TFLOPS, 4),
                    "read_ceiling_gbs": round(read_gbs, 1), "frac_of_read_ceiling": round(achieved_gbs / read_gbs, 4),
                    "peak_note": ("FP32: derived, 152 SMs x 128 FMA/clk x 2 x 2.07 GHz; HBM: measured copy bandwidth "
                                  "(MEASURED_PEAKS.json hbm_gbs)" if peaks else "FP32 derived; HBM fallback")}
    elif mixed:
        peaks = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}
        hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
        achieved_gbs = nbytes / (k_avg * 1e-3) / 1e9
        roofline = {"bound": "hbm", "kernel": f"{kname}<{kp}> (FP32 SpMM, the product alone)",
                    "achieved": round(achieved_gbs, 1), "peak": hbm_peak, "unit": "GB/s",
                    "frac": round(achieved_gbs / hbm_peak, 4), "traffic": recorded_traffic(kname, args.workload, s),
                    "kernel_ms": round(k_avg, 5), "algorithmic_bytes": nbytes, "algorithmic_flops": flops,
                    "with_gram_ms": round(gram_ms, 5),
                    "with_gram_frac": round(nbytes / (gram_ms * 1e-3) / 1e9 / hbm_peak, 4),
                    "read_ceiling_gbs": round(read_gbs, 1), "frac_of_read_ceiling": round(achieved_gbs / read_gbs, 4),
                    "peak_note": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)" if peaks else "fallback"}
    elif tc:
        peaks = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}
        roofline = roofline_tc(n, s, kp, k_avg, single_ms, seq_ms, read_gbs, peaks,
                               recorded_traffic(kname, args.workload, s), args.kernel_launches)
    elif not dense and (nbytes / (float(json.load(open(PEAKS_FILE)).get("hbm_gbs", 6800.0)) if os.path.exists(PEAKS_FILE)
                                  else 6800.0) / 1e9 > flops / FP64_PEAK_TFLOPS / 1e12):
        # a sparse FP64 product whose HBM floor exceeds its FP64-pipe floor (s = 1): bound by HBM
        hbm_peak = float(json.load(open(PEAKS_FILE)).get("hbm_gbs", 6800.0)) if os.path.exists(PEAKS_FILE) else 6800.0
        gbs = nbytes / (k_avg * 1e-3) / 1e9
        roofline = {"bound": "hbm", "kernel": f"{kname}<{kp}> (the solver's FP64 CSR product alone)",
                    "achieved": round(gbs, 1), "peak": hbm_peak, "unit": "GB/s", "frac": round(gbs / hbm_peak, 4),
                    "traffic": recorded_traffic(kname, args.workload, s), "kernel_ms": round(k_avg, 5),
                    "algorithmic_bytes": nbytes, "algorithmic_flops": flops,
                    "peak_note": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)" if os.path.exists(PEAKS_FILE)
                    else "fallback"}
    else:
        roofline = {"bound": "alu", "kernel": f"{kname}<{kp}> (FP64 pipe)", "achieved": round(achieved_tflops, 4),
                    "peak": round(FP64_PEAK_TFLOPS, 4), "unit": "TFLOP/s",
                    "frac": round(achieved_tflops / FP64_PEAK_TFLOPS, 4),
                    "traffic": recorded_traffic(kname, args.workload, s),
                    "kernel_ms": round(k_avg, 5), "algorithmic_flops": flops, "algorithmic_bytes": nbytes,
                    "hbm_gbs_equiv": round(nbytes / (k_avg * 1e-3) / 1e9, 1),
                    "peak_note": "derived: 152 SMs x 2 DFMA/clk x 2 x 2.07 GHz (probe measured 1.20 TFLOP/s)"}

    # end to end through the public host-buffer API (pinned host memory in, x out)
    b_pin = torch.from_numpy(b).pin_memory()
    U_pin = torch.from_numpy(np.asfortranarray(U).ravel(order="F")).pin_memory()
    x_pin = torch.empty(n, dtype=torch.float64).pin_memory()
    e2e = []
    for it in range(args.steps + 1):
        t1 = time.perf_counter()
        st, inf = mb.mbpcg_solve(solver.h, b_pin.data_ptr(), U_pin.data_ptr(), tol, 400000, x_pin.data_ptr())
        t2 = time.perf_counter()
        if it > 0:
            e2e.append((t2 - t1) * 1e3)
    e2e_ms = sum(e2e) / len(e2e)

    line = None
    if rank == 0:
        line = {
            "metric": METRIC, "value": round(ms_per_step, 4), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if mixed else "f64", "data": "synthetic",
            "config": bench_config(args, cfg, A, s, pname, world),
            "iterations": info["iterations"], "restarts": info["restarts"], "relres_true": relres_check,
            "cg_ms": round(cg_ms, 4), "cg_iterations": cg_infos[-1]["iterations"],
            "speedup_vs_cg": round(cg_ms / ms_per_step, 4),
            "us_per_iteration": round(1e3 * ms_per_step / max(1, info["iterations"]), 3),
            "cg_us_per_iteration": round(1e3 * cg_ms / max(1, cg_infos[-1]["iterations"]), 3),
            "solves_per_s": round(world * args.steps / (total_ms * 1e-3), 4),
            "wall_s_timed": round(wall, 3),
            "roofline": roofline,
            "e2e": {"value": round(e2e_ms, 4), "unit": UNIT, "h2d_bytes_per_step": 8 * n + 8 * n * s,
                    "d2h_bytes_per_step": 8 * n + 200 * (info["restarts"] + 1)},
            "gpu_launches": sum(launches_per_solve(i, dense, False, prec == mb.MBPCG_FP64_TC, mixed) for i in infos),
            "gpu_launches_cg": sum(launches_per_solve(i, dense, True, cg_fused=dense and n % 2 == 0 and n <= 16384)
                                   for i in cg_infos),
            "clocks": clk.summary(),
        }
        if not args.no_spmm_roofline:
            peaks = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}
            line["spmm_roofline"] = spmm_roofline(mb, stream, flush, float(peaks.get("hbm_gbs", 6800.0)))
        if mixed and not dense:
            u, c, t = solver.spmm_tuning()
            line["spmm_autotune"] = {"unroll": u, "ctas_per_sm": c,
                                     "times_us_(variant,ctas_per_sm)": dict(zip(
                                         ["4,4", "4,8", "4,16", "8,4", "8,8", "8,16", "0,2 tiled", "1,1 wide1024",
                                          "1,2 wide1024", "2,2 wide512", "2,4 wide512"], [round(v, 2) for v in t]))}
        if once is not None:
            once["speedup_vs_cg"] = round(cg_ms / once["ms"], 4)
            line["round_once"] = once
        if sweep is not None:
            for v in sweep.values():
                v["speedup_vs_cg"] = round(cg_ms / v["ms"], 4)
            line["sweep_s"] = sweep
        if fp64 is not None:
            f_ms = sum(f_times) / len(f_times)
            xfh = xf.cpu().numpy()
            line["fp64_mbpcg"] = {"ms": round(f_ms, 4), "iterations": f_infos[-1]["iterations"],
                                  "restarts": f_infos[-1]["restarts"], "relres_true": f_infos[-1]["relres_true"]}
            line["speedup_vs_fp64_mbpcg"] = round(f_ms / ms_per_step, 4)
            line["rel_diff_to_fp64_solution"] = float(np.linalg.norm(xh - xfh) / np.linalg.norm(xfh))
    solver.close()
    cg.close()
    if fp64 is not None:
        fp64.close()
    return line


def host_cpu():
    """(threads the OpenMP oracle uses, CPU model) of this host."""
    threads = int(os.environ.get("OMP_NUM_THREADS", "0") or 0) or (os.cpu_count() or 1)
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return threads, model or "unknown"


def oracle_sample(args, A, s, precond, iters):
    """Time `iters` iterations (plus the set-up) of the oracle's OpenMP build (same source and bits
    as the parity oracle, independent loops shared among all host cores); returns
    (seconds per iteration, set-up seconds)."""
    import oracle
    b = wl.rhs(A.n, 0)
    U = wl.initial_block(A.n, s, 1)
    oracle.mbpcg_state(A, b, U, 1, precond=precond, omp=True)  # untimed: thread pool, first-touch pages
    setups = []
    for _ in range(2):
        t0 = time.perf_counter()
        oracle.mbpcg_state(A, b, U, 0, precond=precond, omp=True)
        setups.append(time.perf_counter() - t0)
    setup = min(setups)
    t1 = time.perf_counter()
    oracle.mbpcg_state(A, b, U, iters, precond=precond, omp=True)
    t2 = time.perf_counter()
    return max((t2 - t1) - setup, 0.0) / iters, setup


def full_solve_iterations(workload, s):
    path = os.path.join(ROOT, "oracle", "full_solve_counts.json")
    try:
        return json.load(open(path))[workload][str(s)]["iterations"]
    except (OSError, KeyError, ValueError):
        return None


def cpu_baseline(args, A, s, precond, gpu_iterations):
    per_it, setup = oracle_sample(args, A, s, precond, args.cpu_sample_iters)
    its = full_solve_iterations(args.workload, s) or gpu_iterations
    threads, model = host_cpu()
    return {"value": round((setup + per_it * its) * 1e3, 1), "unit": UNIT, "cores": threads, "kind": "oracle",
            "cpu_model": model, "build": "oracle source, gcc -O3 -fopenmp (independent loops over all host cores; "
                                         "same bits as the single-thread parity build)",
            "sample": f"{args.cpu_sample_iters} oracle iterations (+ set-up) timed on {threads} host threads, "
                      f"extrapolated linearly to the {its} iterations of the oracle's full solve "
                      f"(oracle/full_solve_counts.json)"}


def run_reference(args, world, rank):
    if rank != 0:
        return None
    cfg = WORKLOADS[args.workload]
    s = args.s or cfg["s"]
    A = make_matrix(args.workload)
    its = full_solve_iterations(args.workload, s)
    if its is None:
        return {"impl": "reference", "unavailable": f"no recorded oracle iteration count for {args.workload} s={s}"}
    pname = resolve_precision(args, cfg, isinstance(A, wl.Dense))
    if pname == "mixed":
        return {"impl": "reference", "unavailable": "the oracle is FP64 only; no oracle form of the mixed-precision "
                                                    "solve exists to time"}
    per = []
    iters = max(1, args.cpu_sample_iters // 2)
    for k in range(args.warmup + args.steps):
        p, setup = oracle_sample(args, A, s, cfg["precond"], iters)
        if k >= args.warmup:
            per.append((setup + p * its) * 1e3)
    ms = sum(per) / len(per)
    threads, model = host_cpu()
    return {"impl": "reference", "metric": METRIC, "value": round(ms, 1), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 1), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(args, cfg, A, s, pname, world),
            "cpu_baseline": {"value": round(ms, 1), "unit": UNIT, "cores": threads, "kind": "oracle",
                             "cpu_model": model,
                             "sample": f"each step: {iters} iterations (+ set-up) of the oracle's OpenMP build on "
                                       f"{threads} host threads, extrapolated linearly to the oracle's "
                                       f"{its}-iteration full solve; the step value is that extrapolation, not "
                                       f"time spent (a full oracle solve takes minutes)"},
            "e2e": {"value": round(ms, 1), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


SERVING_DESC = ("stream of requests, Poisson arrivals at 0.7x the measured single-stream solve rate; each a 2D/3D "
                "Poisson (no scaling) or 3D diffusion (Jacobi) CSR system, n log-uniform in [1e3,1e6] (24 grid sides "
                "per kind), s uniform in {1,4,8,16}, tol 1e-8, FP64; b from SplitMix64 per request")


class MatrixCache:
    """Matrices of the request stream, generated once per (kind, grid side)."""

    def __init__(self):
        self.mats = {}

    def get(self, kind, m):
        key = (kind, m)
        if key not in self.mats:
            if kind == "poisson2d":
                self.mats[key] = wl.poisson2d(m)
            elif kind == "poisson3d":
                self.mats[key] = wl.poisson3d(m)
            else:
                self.mats[key] = wl.diffusion3d(m, m)
        return self.mats[key]


def serve_stream(mb, reqs, cache, rhs, arrivals, slots):
    """Submit every request at its arrival time (seconds from start) to a server with `slots`
    slots; a second thread waits for the tickets. Returns per-request latency (s) and results."""
    import threading
    srv = mb.Server(slots=slots)
    tickets = [None] * len(reqs)
    results = [None] * len(reqs)
    ready = threading.Semaphore(0)

    def waiter():
        for i in range(len(reqs)):
            ready.acquire()
            results[i] = srv.wait(tickets[i])

    th = threading.Thread(target=waiter)
    th.start()
    lag = []
    t0 = time.perf_counter()
    for i, r in enumerate(reqs):
        delay = arrivals[i] - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(delay)
        lag.append(max(0.0, -delay))
        A = cache.get(r["kind"], r["m"])
        tickets[i] = srv.submit(A, rhs[i], s=r["s"], precond=r["precond"], algo=0, tol=1e-8, maxit=200000,
                                seed=r["rhs_seed"])
        ready.release()
    th.join()
    makespan = time.perf_counter() - t0
    stats = srv.stats()
    srv.close()
    lat = np.array([res["queue_s"] + res["run_s"] for res in results])
    return lat, results, makespan, stats, float(np.max(lag))


def run_serving(args, world, rank):
    import torch
    import paper_2608_07327_gb300 as mb
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    mb.lib()
    reqs = wl.serving_requests(args.requests, 0)
    cache = MatrixCache()
    rhs = [wl.rhs(r["n"], r["rhs_seed"]) for r in reqs]
    for r in reqs:
        cache.get(r["kind"], r["m"])
    # single-stream rate: a seeded sample of the stream served one at a time (after a warm-up)
    rng = np.random.default_rng(1)
    sample = sorted(rng.choice(len(reqs), size=min(60, len(reqs)), replace=False))
    warm = [reqs[i] for i in sample[:3]]
    serve_stream(mb, warm, cache, [rhs[i] for i in sample[:3]], [0.0] * 3, 1)
    s_lat, s_res, s_span, _, _ = serve_stream(mb, [reqs[i] for i in sample], cache, [rhs[i] for i in sample],
                                              [0.0] * len(sample), 1)
    mean_service = float(np.mean([res["run_s"] for res in s_res]))
    rate = 0.7 / mean_service
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=len(reqs)))
    arrivals -= arrivals[0]
    clk = ClockSampler(local)
    if world > 1:
        torch.distributed.barrier()
    with clk:
        lat, res, span, stats, lag = serve_stream(mb, reqs, cache, rhs, arrivals, args.slots)
    # each replica serves its own copy of the stream; the latencies reported are the worst replica's
    p50, p99, mean_lat, span_all = max_over_ranks([float(np.percentile(lat, q)) * 1e3 for q in (50, 99)]
                                                  + [float(np.mean(lat)) * 1e3, span], world, dev)
    seq = None
    if args.compare_requests > 0:
        m = min(args.compare_requests, len(reqs))
        q_lat, q_res, q_span, _, _ = serve_stream(mb, reqs[:m], cache, rhs[:m], arrivals[:m], 1)
        b_lat = lat[:m]
        seq = {"requests": m, "slots": 1, "p50_ms": round(float(np.percentile(q_lat, 50)) * 1e3, 3),
               "p99_ms": round(float(np.percentile(q_lat, 99)) * 1e3, 3),
               "batched_p50_ms_same_requests": round(float(np.percentile(b_lat, 50)) * 1e3, 3),
               "batched_p99_ms_same_requests": round(float(np.percentile(b_lat, 99)) * 1e3, 3),
               "identical_results": bool(all(np.array_equal(a["x"], b["x"]) for a, b in zip(q_res, res[:m])))}
    statuses = [r["status"] for r in res]
    relres = max(r["info"]["relres_true"] for r in res)
    launches = sum(launches_per_solve(r["info"], False, False) for r in res)
    h2d = float(np.mean([cache.get(q["kind"], q["m"]).nnz * 12 + (q["n"] + 1) * 4 + q["n"] * 8 for q in reqs]))
    line = {
        "metric": "serving p99 latency (submit to result), continuous batching", "value": round(p99, 3),
        "unit": "ms", "n_gpus": world, "steps": len(reqs), "warmup": 3, "ms_per_step": round(mean_lat, 3),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": SERVING_DESC, "requests": len(reqs), "slots": args.slots,
                   "arrival_rate_per_s": round(rate, 3), "single_stream_mean_solve_ms": round(mean_service * 1e3, 3),
                   "parallelism": "replicas only" if world > 1 else "single GPU",
                   "l2": "inputs differ per request (n up to 1e6); no flush"},
        "p50_ms": round(p50, 3), "p99_ms": round(p99, 3), "mean_ms": round(mean_lat, 3), "solves_per_s": round(world * len(reqs) / span_all, 3),
        "makespan_s": round(span_all, 3), "max_submit_lag_ms": round(lag * 1e3, 3),
        "failed": int(sum(1 for x in statuses if x != 0)), "max_relres_true": relres,
        "peak_active": stats["peak_active"], "peak_bytes": stats["peak_bytes"],
        "sequential": seq,
        "e2e": {"value": round(p99, 3), "unit": "ms", "h2d_bytes_per_step": round(h2d), "d2h_bytes_per_step":
                round(float(np.mean([q["n"] * 8 for q in reqs])))},
        "gpu_launches": launches, "clocks": clk.summary(),
    }
    return line if rank == 0 else None


BATCH_DESC = ("batch of uneven systems: the first K requests of the serving stream's generator with n "
              "log-uniform in [1e3, 1e5] (2D/3D Poisson, 3D diffusion with Jacobi), s in {1, 4, 8, 16}, tol 1e-8, "
              "FP64; one step solves all K")


def run_batch(args, world, rank):
    """K uneven systems per step, solved (a) one after another on their own handles and (b) as one
    batch (mbpcg_batch_*: one graph launch whose chains run concurrently). value = (b) per step;
    each member's result is compared bit for bit with (a). Device synchronised on both sides of
    every timed call; host wall clock (the calls are synchronous and span many streams)."""
    import torch
    import paper_2608_07327_gb300 as mb
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    mb.lib()
    reqs = wl.serving_requests(args.batch_size, 0, n_lo=1e3, n_hi=1e5)
    cache = MatrixCache()
    solvers = [mb.Solver(cache.get(r["kind"], r["m"]), s=r["s"], precond=r["precond"]) for r in reqs]
    rhs = [wl.rhs(r["n"], r["rhs_seed"]) for r in reqs]
    batch = mb.Batch(solvers)

    def solo():
        return [sv.solve(b, tol=1e-8) for sv, b in zip(solvers, rhs)]

    def batched():
        return batch.solve(rhs, tol=1e-8)

    for _ in range(args.warmup):
        ref = solo()
        got = batched()
    times = {"solo": [], "batch": []}
    clk = ClockSampler(local)
    with clk:
        for _ in range(args.steps):
            for name, fn in (("solo", solo), ("batch", batched)):
                torch.cuda.synchronize()
                if world > 1:
                    torch.distributed.barrier()
                t0 = time.perf_counter()
                out = fn()
                torch.cuda.synchronize()
                times[name].append((time.perf_counter() - t0) * 1e3)
                if name == "batch":
                    got = out
                else:
                    ref = out
    ms_batch, ms_solo = max_over_ranks([float(np.median(times["batch"])), float(np.median(times["solo"]))], world, dev)
    same = all(np.array_equal(a[0], b[0]) and a[1]["iterations"] == b[1]["iterations"] for a, b in zip(ref, got))
    iters = sum(info["iterations"] for _, info in got)
    launches = sum(launches_per_solve(info, False, False) for _, info in got)
    h2d = sum(r["n"] * 8 for r in reqs)
    batch.close()
    for sv in solvers:
        sv.close()
    line = {
        "metric": "batch of uneven systems: time per step (all K solved), one graph launch", "value": round(ms_batch, 3),
        "unit": "ms", "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_batch, 3),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": BATCH_DESC, "K": len(reqs), "n_total": int(sum(r["n"] for r in reqs)),
                   "parallelism": "replicas only" if world > 1 else "single GPU",
                   "l2": "inputs of the K systems differ; no flush"},
        "solo_sequential_ms": round(ms_solo, 3), "speedup_vs_solo": round(ms_solo / ms_batch, 3),
        "identical_results": bool(same), "iterations_total": int(iters),
        "max_relres_true": max(info["relres_true"] for _, info in got),
        "e2e": {"value": round(ms_batch, 3), "unit": "ms", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(h2d)},
        "gpu_launches": int(launches) * args.steps, "clocks": clk.summary(),
    }
    return line if rank == 0 else None


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.workload == "batch":
        line = None if args.impl == "reference" else run_batch(args, world, rank)
        if args.impl == "reference":
            line = {"impl": "reference", "unavailable": "the oracle solves one system at a time; the batch "
                    "workload has no CPU reference arm"} if rank == 0 else None
    elif args.workload == "serving":
        line = None if args.impl == "reference" else run_serving(args, world, rank)
        if args.impl == "reference":
            line = {"impl": "reference", "unavailable": "the oracle solves one system at a time; the serving "
                    "stream has no CPU reference arm"} if rank == 0 else None
    elif args.impl == "reference":
        line = run_reference(args, world, rank)
    else:
        line = run_ours(args, world, rank, local)
        if line is not None and world == 1 and not args.no_cpu_baseline:
            cfg = WORKLOADS[args.workload]
            A = make_matrix(args.workload)
            line["cpu_baseline"] = cpu_baseline(args, A, line["config"]["s"], cfg["precond"], line["iterations"])
    if line is not None:
        print(json.dumps(line), flush=True)
    if world > 1 and args.impl != "reference":
        import torch.distributed as dist
        if dist.is_initialized():
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
