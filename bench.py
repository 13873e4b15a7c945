#!/usr/bin/env python
"""Benchmark: time to k eigenpairs of randomized Krylov-Schur on one GB300.

Workload (default): the 2D convection-diffusion operator on a 1000 x 1000 grid
(n = 1e6, 5-point upwind stencil, nu = 1, b = (20, 10), FP64 CSR,
4,996,000 nonzeros); k = 20 eigenvalues of largest real part, p = 60, sketch
d = 320 with zeta = 8 nonzeros per column, tolerance 1e-8 on the residual
estimates, locking on.  A step is one complete solve (start vector, every
Arnoldi step and restart, Ritz vectors and FP64 residuals).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun each rank solves its own
replica of the problem (the solver does not shard: replicas only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time to k eigpairs (resid≤1e-8) & SpMV+RGS HBM GB/s; mixed/batched vs FP64 rKS"
WORKLOAD = ("convdiff2d_1000: 2D upwind convection-diffusion 1000x1000 (n=1e6), nu=1, b=(20,10), "
            "FP64 CSR; k=20 LR, p=60, d=320, zeta=8, tol=1e-8, locking")
# Products with A that rKS needs on this workload (measured by this solver on a
# GB300; the method's count, used to scale the bounded CPU samples).
NMATVEC_WORKLOAD = 7621
# DRAM traffic of the dominant kernel from one ncu capture, as a ratio to the
# algorithmic bytes of the captured launch (applied to the mean launch), valid
# only for the kernel source it was measured on (see _kernel_hash).
NCU_TRAFFIC = {
    # two launches of k_df_update_sketch at c = 64, 65 in the third restart (profiles/df_kernels_convdiff1000.md):
    # DRAM 541.6 / 547.1 MB against 528 / 536 MB of algorithmic bytes (the bin lists of Omega are the rest)
    "update_sketch": {"kernels_sha": "fdc1ba79cef500a9", "ratio": 1.023},
}


def _kernel_hash():
    """sha256 prefix of the update kernel's source: the kernel, the tile
    helpers it inlines and its compile-time constants (None if not found)."""
    csrc = os.path.join(ROOT, "paper_2508_05400_gb300", "csrc")
    src = open(os.path.join(csrc, "kernels_df.cu")).read()
    impl = open(os.path.join(csrc, "rks_impl.h")).read()
    parts = []
    for a, b in (("// (s, e) += sign * vals[row] for one bin-list entry", "// w'[i] = sum_p A_p x[col_p] (DF)"),
                 ("// Vector load of two consecutive rows", "// Euclidean CGS2 (Krylov-Schur baseline)")):
        i, j = src.find(a), src.find(b)
        if i < 0 or j < i:
            return None
        parts.append(src[i:j])
    parts += [ln for ln in impl.splitlines() if "kDfUpd" in ln or "kTileRows =" in ln]
    return hashlib.sha256("\n".join(parts).encode()).hexdigest()[:16]


def _peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return {"hbm_gbs": d["hbm_gbs"], "source": "of measured"}
    return {"hbm_gbs": 6800.0, "source": "of fallback"}


class Clocks:
    """nvidia-smi samples during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.file = None

    def __enter__(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        if self.proc is None or self.file is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.file.flush()
        with open(self.file.name) as f:
            rows = [ln.strip().split(", ") for ln in f if ln.strip()]
        os.unlink(self.file.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


DTYPES = {"fp64": "f64",
          "df": "df64 (fp32 pair, 48-bit significand; fp64 sketch/LS/Schur/residuals)",
          "mixed": "f32 basis (split-bf16 tensor-core restart) then df64; fp64 sketch/LS/Schur/residuals"}


def _problem():
    from paper_2508_05400_gb300 import inputs as I
    P = I.convdiff2d_problem()
    u1 = I.start_vector(P.A.n, P.u1_seed)
    return P, u1


def cpu_sample(P, u1, restarts: int = 1) -> dict:
    """The FP64 oracle on the host cores: initial expansion + ``restarts`` cycles."""
    from oracle import rks as R
    t0 = time.perf_counter()
    o = P.solver_opts()
    res = R.rks(P.A.to_scipy(), P.k, P.p, P.d, u1, zeta=P.zeta, seed=P.omega_seed, which=P.which,
                tol=o["tol"], eta_lock=o.get("eta_lock"), conv=o["conv"], max_restarts=restarts)
    dt = time.perf_counter() - t0
    return {"seconds": dt, "nmatvec": res.nmatvec, "restarts": res.restarts}


def reduce_max_over_ranks(values, device, dist, world: int):
    """Max of each value over the ranks (replicas run independently; the
    slowest rank bounds the whole job).  No-op for world = 1."""
    if world <= 1:
        return list(values)
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def run_reference(args) -> None:
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    P, u1 = _problem()
    times, nm = [], 0
    for i in range(args.warmup + args.steps):
        s = cpu_sample(P, u1, restarts=1)
        if i >= args.warmup:
            times.append(s["seconds"])
            nm = s["nmatvec"]
    per_matvec = statistics.mean(times) / nm
    total = NMATVEC_WORKLOAD or nm
    value_ms = per_matvec * total * 1e3
    sample = (f"FP64 oracle (numpy/scipy) on the full problem: initial expansion + 1 restart "
              f"({nm} products with A) per step, scaled to {total} products "
              f"({'the count this solver needs to converge' if NMATVEC_WORKLOAD else 'unscaled'})")
    line = {"impl": "reference", "metric": METRIC, "value": value_ms, "unit": "ms",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": statistics.mean(times) * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": P.A.n, "nnz": P.A.nnz},
            "cpu_baseline": {"value": value_ms, "unit": "ms", "cores": os.cpu_count(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value_ms, "unit": "ms", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args) -> None:
    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import __graft_entry__
    __graft_entry__.build()
    from paper_2508_05400_gb300 import rks

    P, u1 = _problem()
    A = P.A
    keep = P.k if args.keep < 0 else args.keep
    stream = torch.cuda.current_stream(dev)
    # inputs resident in HBM before the timed region
    d_rowptr = torch.from_numpy(A.rowptr).to(dev)
    d_colind = torch.from_numpy(A.colind).to(dev)
    d_vals = torch.from_numpy(A.vals).to(dev)
    d_u1 = torch.from_numpy(u1).to(dev)
    mk = lambda prof: rks.Solver(A.n, d_rowptr, d_colind, d_vals, P.k, P.p, P.d, which=P.which,
                                 seed=P.omega_seed, zeta=P.zeta, u1=d_u1, device=True,
                                 stream=stream.cuda_stream, profile=prof, prec=args.prec, maxit=args.maxit,
                                 keep=keep, ortho=args.ortho, aggressive=args.aggressive, **P.solver_opts())
    X_dev = torch.empty((P.k + 1, A.n), dtype=torch.float64, device=dev)
    # one untimed solve with every kernel timed (the first warm-up): the
    # per-kernel breakdown and the dominant kernel; the timed solves then put
    # events around that kernel only
    with mk(True) as s_all:
        s_all.solve(allow_noconv=False)
        breakdown = s_all.stats()
    dom = max((c for c in rks.KCLASSES if c != "other" and breakdown[c]["ms"] > 0),
              key=lambda c: breakdown[c]["ms"])
    solver = mk(rks.profile_mask(dom))

    def step():
        info = solver.solve(allow_noconv=False)
        lam, _, res = solver.eigpairs(X_out=X_dev)
        return info, lam, res

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(max(args.warmup - 1, 1)):
        step()
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    infos, agg = [], None
    with Clocks(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            info, lam, res = step()
            infos.append(info)
            st = solver.stats()
            if agg is None:
                agg = st
            else:
                for key, v in st.items():
                    if isinstance(v, dict):
                        for f in v:
                            agg[key][f] += v[f]
                    else:
                        agg[key] += v
        ev1.record(stream)
        barrier()
    ms_total = ev0.elapsed_time(ev1)
    ms_step = reduce_max_over_ranks([ms_total / args.steps], dev, dist, world)[0]
    clocks = clk.summary()

    # roofline of the dominant kernel (live CUDA-event durations of the timed solves)
    peaks = _peaks()
    d = agg[dom]
    per_launch_ms = d["ms"] / d["launches"]
    bytes_per_launch = d["bytes"] / d["launches"]
    achieved = bytes_per_launch / (per_launch_ms * 1e-3) / 1e9
    traffic = None
    rec = NCU_TRAFFIC.get(dom)
    if rec and rec.get("kernels_sha") == _kernel_hash() and args.prec == "df":
        traffic = rec["ratio"] * bytes_per_launch
    path = ("spmv_sketch", "ls", "update_sketch", "finish")
    path_bytes = sum(breakdown[c]["bytes"] for c in path)
    path_ms = sum(breakdown[c]["ms"] for c in path)
    fp64_gflops = d["flops"] / (d["ms"] * 1e-3) / 1e9
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                "peak_source": peaks["source"],
                "bytes_per_launch": bytes_per_launch, "ms_per_launch": per_launch_ms,
                "fp64_gflops": fp64_gflops}

    # end to end through the C ABI with host (pinned) buffers, copies inside
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    h_rowptr, h_colind, h_vals, h_u1 = pin(A.rowptr), pin(A.colind), pin(A.vals), pin(u1)
    h_X = torch.empty((P.k + 1, A.n), dtype=torch.float64).pin_memory()
    e2e_times = []
    barrier()
    for _ in range(0 if args.no_e2e else args.steps):
        t0 = time.perf_counter()
        with rks.Solver(A.n, h_rowptr, h_colind, h_vals, P.k, P.p, P.d, which=P.which,
                        seed=P.omega_seed, zeta=P.zeta, u1=h_u1, stream=stream.cuda_stream,
                        prec=args.prec, maxit=args.maxit, keep=keep, ortho=args.ortho,
                        aggressive=args.aggressive, **P.solver_opts()) as s2:
            s2.solve(allow_noconv=False)
            s2.eigpairs(X_out=h_X)
        e2e_times.append((time.perf_counter() - t0) * 1e3)
    barrier()
    e2e_ms = statistics.mean(e2e_times) if e2e_times else None
    kk = P.k
    if e2e_ms is not None:
        e2e_ms = reduce_max_over_ranks([e2e_ms], dev, dist, world)[0]
    h2d = A.rowptr.nbytes + A.colind.nbytes + A.vals.nbytes + u1.nbytes
    d2h = 8 * A.n * kk + 3 * 8 * kk

    info = infos[-1]
    line = {"metric": METRIC, "value": ms_step, "unit": "ms", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPES[args.prec],
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": A.n, "nnz": A.nnz, "k": P.k, "p": P.p, "d": P.d,
                       "zeta": P.zeta, "prec": args.prec, "keep": keep, "ortho": args.ortho,
                       "aggressive": bool(args.aggressive),
                       "parallelism": f"replicas{world}",
                       "l2": "inputs larger than L2 (basis 648 MB, A 80 MB)"},
            "roofline": roofline,
            "spmv_rgs_gbs": path_bytes / (path_ms * 1e-3) / 1e9 if path_ms else None,
            "e2e": {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": int(agg["launches_total"]),
            "clocks": clocks,
            "solve": {"restarts": info["restarts"], "nmatvec": info["nmatvec"],
                      "nlocked": info["nlocked"], "max_resid": info["max_resid"],
                      "max_est": info["max_est"], "host_dense_ms_per_step": agg["host_ms"] / args.steps,
                      "whitenings_per_step": agg["whitenings"] / args.steps,
                      "kernel_ms_per_step": {c: breakdown[c]["ms"] for c in rks.KCLASSES},
                      "kernel_ms_note": "one untimed solve with every kernel timed; the timed solves "
                                        "time only " + dom}}
    solver.close()
    if rank == 0 and not args.no_cpu_baseline:
        s = cpu_sample(P, u1, restarts=1)
        per = s["seconds"] / s["nmatvec"]
        line["cpu_baseline"] = {
            "value": per * info["nmatvec"] * 1e3, "unit": "ms", "cores": os.cpu_count(),
            "kind": "oracle",
            "sample": (f"FP64 oracle (numpy/scipy, host cores) on the full problem: initial "
                       f"expansion + 1 restart ({s['nmatvec']} products with A, "
                       f"{s['seconds']:.1f} s), scaled to the {info['nmatvec']} products this "
                       f"solve needed")}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--maxit", type=int, default=4000, help="restart limit of each solve")
    ap.add_argument("--ortho", default="sketch", choices=["sketch", "cgs2"],
                    help="sketch: randomized Gram-Schmidt (rKS); cgs2: the Krylov-Schur baseline "
                         "with Euclidean CGS2 (DF only)")
    ap.add_argument("--keep", type=int, default=-1,
                    help="active Schur vectors a restart keeps after locking (thick restart); "
                         "-1: k; 0: k - q as in Algorithm 1")
    ap.add_argument("--aggressive", action="store_true",
                    help="aggressive deflation: converged Schur blocks move to the front and lock")
    ap.add_argument("--prec", default="df", choices=["df", "fp64", "mixed"],
                    help="arithmetic of the n-dimensional work (see include/rks.h)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
