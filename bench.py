#!/usr/bin/env python
"""Benchmark: time to k eigenpairs of randomized Krylov-Schur on one GB300.

Workload (default): the 3D convection-diffusion operator on a 160^3 grid
(n = 4 096 000, 7-point upwind stencil, log-normal diffusivity sigma = 1 from
seed 2, convection (10, 5, 2), FP32 CSR values, 28 518 400 nonzeros); k = 50
eigenvalues of largest real part, p = 100, sketch d = 600 with zeta = 8
nonzeros per column, ||A x - l x|| / (||A||_1 ||x||) <= 1e-8 verified in FP64,
locking on, thick restart keeping k active Schur vectors.  Mixed precision:
FP32 basis, FP32 SpMV and basis updates with compensated arithmetic, the
restart product as split-BF16 on the tensor cores with FP32 accumulation, the
sketch sums, small least squares, Schur steps, residuals and Rayleigh
quotients in FP64; a double-float phase finishes below the FP32 floor.  A step
is one complete solve (start vector, every Arnoldi step and restart, Ritz
vectors, FP64 residuals and Rayleigh quotients).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload convdiff3d_160|convdiff2d_1000] [--prec mixed|df|fp64]

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
WORKLOADS = {
    "convdiff3d_160": ("convdiff3d_160: 3D upwind convection-diffusion 160^3 (n=4.096e6), log-normal nu "
                       "(sigma=1, seed 2), b=(10,5,2), FP32 CSR; k=50 LR, p=100, d=600, zeta=8, "
                       "resid<=1e-8 (FP64-verified), locking, thick restart keep=50"),
    "convdiff2d_1000": ("convdiff2d_1000: 2D upwind convection-diffusion 1000x1000 (n=1e6), nu=1, b=(20,10), "
                        "FP64 CSR; k=20 LR, p=60, d=320, zeta=8, resid<=1e-8 (FP64-verified), locking, "
                        "thick restart keep=20"),
}
DEFAULT_PREC = {"convdiff3d_160": "mixed", "convdiff2d_1000": "fp64"}
# DRAM traffic of the dominant kernel from one ncu capture, as a ratio to the
# algorithmic bytes of the captured launch (applied to the mean launch), valid
# only for the kernel source it was measured on (see _kernel_hash).
NCU_TRAFFIC = {
    # (kernel class, precision, workload): DRAM bytes / algorithmic bytes of
    # the captured launches of k_df_update_sketch (double-float, c = 64, 65,
    # third restart of the 1000^2 workload: 541.6 / 547.1 MB against 528 /
    # 536 MB; the bin lists of Omega are the rest)
    ("update_sketch", "df", "convdiff2d_1000"): {"kernels_sha": "fdc1ba79cef500a9", "ratio": 1.023},
    # k_df_update_sketch<float, 20> of the 160^3 operator at 100^3 (FP32 phase, c = 61, first
    # expansion; profiles/update_spmv_ls_convdiff3d_100_mixed.md): DRAM 275.9 MB (4.01 TB/s over
    # 68.9 us) against 252 MB of algorithmic bytes.  Applied to the mean launch of the 160^3 solve
    # (c ~ 100, FP32 and double-float launches), where the bin lists' share of the traffic is
    # smaller: an upper estimate by a few percent.
    ("update_sketch", "mixed", "convdiff3d_160"): {"kernels_sha": "03fc6acf03ac0121", "ratio": 1.095},
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
          "mixed": ("f32 basis + f32 SpMV/updates (compensated), split-bf16 tensor-core restart with f32 "
                    "accumulation; below the f32 floor df64 restarts continuing from the f32 Krylov-Schur "
                    "decomposition (relation error corrected in df64/f32); f64 sketch/LS/Schur/residuals/Rayleigh")}


def _problem(workload: str, grid: int = 0):
    """The workload's problem; grid > 0 replaces the grid side (smaller cases
    of the same operator for profiling)."""
    from paper_2508_05400_gb300 import inputs as I
    if workload == "convdiff3d_160":
        P = I.convdiff3d_problem(N=grid) if grid else I.convdiff3d_problem()
    else:
        P = I.convdiff2d_problem(N=grid) if grid else I.convdiff2d_problem()
    u1 = I.start_vector(P.A.n, P.u1_seed)
    return P, u1


class OracleSampler:
    """Bounded samples of the FP64 oracle (numpy/scipy) on the host cores.

    A sample times the oracle's Algorithm 2 (``extend``, as it stands) on the
    full problem from a decomposition of jbar columns (the mean basis size of
    the solve: the thick restart keeps k active vectors and expands to
    m = k + p) by 1 and by 1 + s steps; the difference over s is the cost of
    one product with A with its sketch, least squares and update at that
    basis size, and a solve that needed N products is estimated as N times it.
    The starting decomposition has the right sizes (its first column is the
    start vector, the others random with orthonormal sketches): the cost of a
    step does not depend on the values.  The dense Schur steps of the restarts
    are not included."""

    def __init__(self, P, u1, s: int = 3):
        import numpy as np
        import scipy.sparse as sp
        from oracle import rks as R
        from oracle import sketch as SK
        self.P, self.s = P, s
        self.A = sp.csr_matrix(P.A.to_scipy())
        self.Om = SK.omega_matrix(P.A.n, P.d, P.zeta, P.omega_seed)
        self.jbar = (P.k + P.k + P.p) // 2
        j = self.jbar
        st = R.start(self.A, self.Om, u1)
        rng = np.random.default_rng(0)
        U = np.asfortranarray(rng.standard_normal((P.A.n, j + 1)))
        U[:, 0] = st.Ua[:, 0]
        Q, _ = np.linalg.qr(rng.standard_normal((P.d, j + 1)))
        self.base = dict(Ua=U, Sa=np.asfortranarray(Q), Ba=np.zeros((j + 1, j)), Tqa=np.zeros((0, j)))
        self.st0 = st

    def _run(self, steps: int) -> float:
        import dataclasses
        from oracle import rks as R
        st = dataclasses.replace(self.st0, **self.base)
        t0 = time.perf_counter()
        R.extend(st, self.jbar + steps)
        return time.perf_counter() - t0

    def sample(self) -> dict:
        t1, t2 = self._run(1), self._run(1 + self.s)
        return {"seconds": t1 + t2, "per_product": max(t2 - t1, 0.0) / self.s}

    @staticmethod
    def cores() -> int:
        try:
            from threadpoolctl import threadpool_info
            return max((int(x.get("num_threads", 1)) for x in threadpool_info()), default=1)
        except Exception:
            return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()

    def estimate_ms(self, smp: dict, nmatvec: int) -> float:
        return nmatvec * smp["per_product"] * 1e3

    def describe(self, smp: dict, nmatvec: int) -> str:
        return (f"FP64 oracle (numpy/scipy) on the full problem: its Algorithm 2 from a {self.jbar}-column "
                f"decomposition by 1 and by {1 + self.s} steps ({smp['seconds']:.1f} s), "
                f"{smp['per_product'] * 1e3:.0f} ms per product with A at that basis size, scaled to the "
                f"{nmatvec} products of the solve (dense Schur steps not included)")


# Products with A that the benchmarked solve needs (mixed precision, measured
# with this solver on a GB300), used to scale the reference arm's samples.
REFERENCE_NMATVEC = {"convdiff3d_160": 20698, "convdiff2d_1000": 7536}


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
    P, u1 = _problem(args.workload, args.grid)
    sampler = OracleSampler(P, u1)
    nm = REFERENCE_NMATVEC[args.workload]
    vals, secs, last = [], [], None
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        smp = sampler.sample()
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            vals.append(sampler.estimate_ms(smp, nm))
            secs.append(dt)
            last = smp
    value_ms = statistics.mean(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value_ms, "unit": "ms",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": value_ms, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload], "n": P.A.n, "nnz": P.A.nnz, "k": P.k, "p": P.p,
                       "d": P.d, "zeta": P.zeta},
            "cpu_baseline": {"value": value_ms, "unit": "ms", "cores": sampler.cores(), "kind": "oracle",
                             "sample": sampler.describe(last, nm) + f"; {statistics.mean(secs):.1f} s of "
                             f"host time per step"},
            "e2e": {"value": value_ms, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _solve_once(rks, P, dev_arrays, stream, prec, keep, maxit, profile=False):
    """One solve of P on resident device inputs; returns (info, lam, res, rq, stats, ms)."""
    d_rowptr, d_colind, d_vals, d_u1 = dev_arrays
    with rks.Solver(P.A.n, d_rowptr, d_colind, d_vals, P.k, P.p, P.d, which=P.which, seed=P.omega_seed,
                    zeta=P.zeta, u1=d_u1, device=True, stream=stream, profile=profile, prec=prec, maxit=maxit,
                    keep=keep, **P.solver_opts()) as s:
        info = s.solve(allow_noconv=False)
        lam, _, res = s.eigpairs(want_vectors=False)
        rq = s.rayleigh()
        return info, lam, res, rq, s.stats(), info["t_solve_ms"]


def _pair_errors(lam, ref):
    """|l_i - l_ref| / |l_ref| for each of lam's values against the nearest
    reference value (both best first)."""
    import numpy as np
    return [float(np.min(np.abs(ref - l)) / abs(ref[int(np.argmin(np.abs(ref - l)))])) for l in lam]


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

    prec = args.prec or DEFAULT_PREC[args.workload]
    P, u1 = _problem(args.workload, args.grid)
    A = P.A
    keep = P.k if args.keep < 0 else args.keep
    stream = torch.cuda.current_stream(dev)
    # inputs resident in HBM before the timed region
    dev_arrays = (torch.from_numpy(A.rowptr).to(dev), torch.from_numpy(A.colind).to(dev),
                  torch.from_numpy(A.vals).to(dev), torch.from_numpy(u1).to(dev))
    d_rowptr, d_colind, d_vals, d_u1 = dev_arrays
    mk = lambda prof: rks.Solver(A.n, d_rowptr, d_colind, d_vals, P.k, P.p, P.d, which=P.which,
                                 seed=P.omega_seed, zeta=P.zeta, u1=d_u1, device=True,
                                 stream=stream.cuda_stream, profile=prof, prec=prec, maxit=args.maxit,
                                 max_restarts=args.max_restarts, keep=keep, ortho=args.ortho,
                                 aggressive=args.aggressive, **P.solver_opts())
    noconv_ok = args.max_restarts > 0
    X_dev = torch.empty((P.k + 2, A.n), dtype=torch.float64, device=dev)
    # one untimed solve with every kernel timed (the first warm-up): the
    # per-kernel breakdown and the dominant kernel; the timed solves then put
    # events around that kernel only
    with mk(True) as s_all:
        s_all.solve(allow_noconv=noconv_ok)
        breakdown = s_all.stats()
    dom = max((c for c in rks.KCLASSES if c != "other" and breakdown[c]["ms"] > 0),
              key=lambda c: breakdown[c]["ms"])
    solver = mk(rks.profile_mask(dom))

    def step():
        info = solver.solve(allow_noconv=noconv_ok)
        lam, _, res = solver.eigpairs(X_out=X_dev)
        rq = solver.rayleigh()
        return info, lam, res, rq

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(max(args.warmup - 1, 1)):
        step()
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    infos, agg, last = [], None, None
    with Clocks(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            info, lam, res, rq = step()
            infos.append(info)
            last = (lam, res, rq)
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
    rec = NCU_TRAFFIC.get((dom, prec, args.workload))
    if rec and rec.get("kernels_sha") == _kernel_hash():
        traffic = rec["ratio"] * bytes_per_launch
    path = ("spmv_sketch", "ls", "update_sketch", "finish")
    path_bytes = sum(breakdown[c]["bytes"] for c in path)
    path_ms = sum(breakdown[c]["ms"] for c in path)
    # the same aggregate split by the basis the launches worked on (the mixed
    # path's FP32 phase and its double-float phase)
    spmv_rgs_by_basis = {}
    b32 = sum(breakdown[c]["bytes_f32"] for c in path)
    m32 = sum(breakdown[c]["ms_f32"] for c in path)
    for name, b_, m_ in (("fp32", b32, m32), ("df", path_bytes - b32, path_ms - m32)):
        if m_ > 0 and b_ > 0:
            g = b_ / (m_ * 1e-3) / 1e9
            spmv_rgs_by_basis[name] = {"gbs": g, "frac": g / peaks["hbm_gbs"], "ms": m_}
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                "peak_source": peaks["source"],
                "bytes_per_launch": bytes_per_launch, "ms_per_launch": per_launch_ms,
                "flop_rate_gflops": d["flops"] / (d["ms"] * 1e-3) / 1e9,
                "flop_note": "algorithmic FLOP/s of the dominant kernel (multiply-adds counted as 2; "
                             "double-float work runs on the FP32 pipes)"}
    solver.close()

    # end to end through the C ABI with host (pinned) buffers, copies inside
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    h_rowptr, h_colind, h_vals, h_u1 = pin(A.rowptr), pin(A.colind), pin(A.vals), pin(u1)
    h_X = torch.empty((P.k + 2, A.n), dtype=torch.float64).pin_memory()
    e2e_times = []
    barrier()
    for _ in range(0 if args.no_e2e else max(1, min(args.steps, args.e2e_steps))):
        t0 = time.perf_counter()
        with rks.Solver(A.n, h_rowptr, h_colind, h_vals, P.k, P.p, P.d, which=P.which,
                        seed=P.omega_seed, zeta=P.zeta, u1=h_u1, stream=stream.cuda_stream,
                        prec=prec, maxit=args.maxit, keep=keep, ortho=args.ortho,
                        aggressive=args.aggressive, **P.solver_opts()) as s2:
            s2.solve(allow_noconv=False)
            nwx = s2.nwanted
            s2.eigpairs(X_out=h_X[:nwx])
        e2e_times.append((time.perf_counter() - t0) * 1e3)
    barrier()
    e2e_ms = statistics.mean(e2e_times) if e2e_times else None
    if e2e_ms is not None:
        e2e_ms = reduce_max_over_ranks([e2e_ms], dev, dist, world)[0]
    h2d = A.rowptr.nbytes + A.colind.nbytes + A.vals.nbytes + u1.nbytes
    nw = last[0].size
    d2h = 8 * A.n * nw + 3 * 8 * nw

    info = infos[-1]
    lam, res, rq = last
    line = {"metric": METRIC, "value": ms_step, "unit": "ms", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPES[prec],
            "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload], "n": A.n, "nnz": A.nnz, "k": P.k, "p": P.p,
                       "d": P.d, "zeta": P.zeta, "prec": prec, "keep": keep, "ortho": args.ortho,
                       "aggressive": bool(args.aggressive),
                       "parallelism": f"replicas{world}",
                       "l2": "inputs larger than L2 (basis of m+1 columns and A are several GB)"},
            "roofline": roofline,
            "spmv_rgs_gbs": path_bytes / (path_ms * 1e-3) / 1e9 if path_ms else None,
            "spmv_rgs_frac": (path_bytes / (path_ms * 1e-3) / 1e9 / peaks["hbm_gbs"]) if path_ms else None,
            "spmv_rgs_by_basis": spmv_rgs_by_basis,
            "e2e": {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": int(agg["launches_total"]),
            "clocks": clocks,
            "solve": {"restarts": info["restarts"], "nmatvec": info["nmatvec"],
                      "nlocked": info["nlocked"], "max_resid": info["max_resid"],
                      "max_est": info["max_est"], "host_dense_ms_per_step": agg["host_ms"] / args.steps,
                      "whitenings_per_step": agg["whitenings"] / args.steps,
                      "fp32_restarts": st["fp32_restarts"],
                      "mixed_phase2": ("none", "handover", "restart")[st["mixed_phase2"]],
                      "handover_rel": st["handover_rel"],
                      "max_rayleigh_vs_ritz": float(np.max(np.abs(rq - lam) / np.abs(lam))),
                      "kernel_ms_per_step": {c: breakdown[c]["ms"] for c in rks.KCLASSES},
                      "kernel_launches_per_step": {c: breakdown[c]["launches"] for c in rks.KCLASSES},
                      "kernel_ms_note": "one untimed solve with every kernel timed; the timed solves "
                                        "time only " + dom}}

    # the same configuration on the other GPU paths (one solve each), and the
    # per-eigenpair error of this run against the plain FP64 GPU path
    if rank == 0 and not args.no_extras:
        paths = {}
        for other in ("fp64", "df", "mixed"):
            if other == prec:
                continue
            oinfo, olam, ores, orq, _, oms = _solve_once(rks, P, dev_arrays, stream.cuda_stream, other, keep,
                                                         args.maxit)
            paths[other] = {"ms": oms, "restarts": oinfo["restarts"], "nmatvec": oinfo["nmatvec"],
                            "max_resid": oinfo["max_resid"]}
            if other == "fp64":
                errs = _pair_errors(lam, olam)
                rqerr = _pair_errors(rq, orq)
                line["eig_error_vs_fp64_gpu"] = {
                    "per_pair_rel": errs, "max": max(errs), "rayleigh_max": max(rqerr),
                    "note": ("|l - l_fp64| / |l_fp64| per wanted pair against the plain FP64 GPU solve of the "
                             "same problem; both have resid <= 1e-8 ||A||_1, which fixes l only to the "
                             "eigenvalue condition number times that")}
        line["paths"] = paths
        line["spmv_variants"] = _spmv_variants(rks)
        line["exp1_tridiag_1e6"] = _exp1(rks)
        line["batched_uneven256"] = _batched(rks)
        if args.workload == "convdiff3d_160":
            line["eig_error_vs_oracle_small"] = _small_oracle_errors(rks, prec)
            P2, u2 = _problem("convdiff2d_1000")
            arrs2 = (torch.from_numpy(P2.A.rowptr).to(dev), torch.from_numpy(P2.A.colind).to(dev),
                     torch.from_numpy(P2.A.vals).to(dev), torch.from_numpy(u2).to(dev))
            i2, _, _, _, _, ms2 = _solve_once(rks, P2, arrs2, stream.cuda_stream, "fp64", P2.k, args.maxit)
            line["convdiff2d_1000_fp64"] = {"ms": ms2, "restarts": i2["restarts"], "nmatvec": i2["nmatvec"],
                                            "max_resid": i2["max_resid"]}
            del arrs2
    if rank == 0 and not args.no_cpu_baseline:
        sampler = OracleSampler(P, u1)
        smp = sampler.sample()
        line["cpu_baseline"] = {
            "value": sampler.estimate_ms(smp, info["nmatvec"]), "unit": "ms", "cores": sampler.cores(),
            "kind": "oracle", "sample": sampler.describe(smp, info["nmatvec"])}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def _exp1(rks) -> dict:
    """The paper's first experiment at n = 1e6 (Table 1 exponential diagonal,
    N(0,1)/100 off-diagonals, LM, k = 40, m = 80, d = 160, zeta = 8,
    |b^T y|/|l| <= 1e-10): rKS against Krylov-Schur with CGS2 on the same
    kernels (double-float, keep = k), one solve each."""
    from paper_2508_05400_gb300 import inputs as I
    A = I.paper_tridiag(1_000_000, "exponential")
    out = {}
    for ortho in ("sketch", "cgs2"):
        with rks.Solver.from_csr(A, 40, 40, 160, which="LM", tol=1e-10, zeta=8, u1=I.start_vector(A.n, 1),
                                 keep=40, maxit=4000, ortho=ortho) as s:
            info = s.solve(allow_noconv=True)
        out["rks" if ortho == "sketch" else "ks_cgs2"] = {"ms": info["t_solve_ms"], "restarts": info["restarts"],
                                                          "nmatvec": info["nmatvec"], "status": info["status"]}
    out["speedup"] = out["ks_cgs2"]["ms"] / out["rks"]["ms"]
    return out


def _batched(rks) -> dict:
    """The batch of 256 uneven 2D convection-diffusion problems (sides
    U{70..450}, log-normal diffusivity, convection in [0, 30]^2, FP32 values;
    k = 8, p = 24, d = 64, residual <= 1e-8 verified in FP64):
      - persistent: one CUDA graph of persistent kernels (rks_solve_batched_dev:
        the whole of Algorithm 1 on the device, thick restart keep = 12, no
        locking, launch configuration autotuned at creation); CUDA-event time
        of the graph launch and host wall time of the call;
      - streams: one context per problem on its own stream, 16 host threads
        (rks_solve_batched, double-float, locking, keep = 8); host wall time."""
    from paper_2508_05400_gb300 import inputs as I
    probs = [I.uneven_convdiff2d_problem(i) for i in range(256)]
    P0 = probs[0]
    o = P0.solver_opts()
    out = {"sum_n": int(sum(P.A.n for P in probs))}
    t0 = time.perf_counter()
    with rks.DevBatch([P.A for P in probs], P0.k, P0.p, P0.d, which=P0.which, zeta=P0.zeta, tol=o["tol"],
                      conv="norm1", verify=o["verify"], maxit=4000, keep=12) as b:
        t_create = time.perf_counter() - t0
        t0 = time.perf_counter()
        infos = b.solve(allow_noconv=True)
        wall = time.perf_counter() - t0
        cfg = b.config()
        ph = b.phase_cycles()
    tot = sum(ph.values())
    # algorithmic bytes: per row and expansion step j the diagonal SpMV (D
    # values, x, w), the update ((j + 2) columns read, one written) and two
    # sketch-list reads (1.25 zeta uint16 entries each); per restart the
    # restart product (m + 1 columns read, ka + 1 written), ka = keep + 1
    m, zeta, D, ka = P0.k + P0.p, P0.zeta, 5, 13
    step = lambda j: 8 * (D + 2) + 8 * (j + 3) + 2 * 1.25 * zeta * 2
    first = sum(step(j) for j in range(m))
    per_restart = sum(step(j) for j in range(ka, m)) + 8 * (m + 1 + ka + 1)
    alg_bytes = sum(P.A.n * (first + i["restarts"] * per_restart) for P, i in zip(probs, infos))
    out["persistent_gbs"] = alg_bytes / (cfg["last_ms"] * 1e-3) / 1e9
    out["persistent"] = {"ms": cfg["last_ms"], "wall_ms": wall * 1e3, "create_s": t_create,
                         "config": {k: cfg[k] for k in ("GL", "nL", "GS", "nS")}, "tune_ms": cfg["tune_ms"],
                         "converged": int(sum(i["converged"] for i in infos)),
                         "max_resid": float(max(i["max_resid"] for i in infos)),
                         "restarts_median": float(statistics.median([i["restarts"] for i in infos])),
                         "phase_share": {k: round(v / max(tot, 1), 4) for k, v in ph.items()}}
    with rks.Batch([P.A for P in probs], P0.k, P0.p, P0.d, which=P0.which, zeta=P0.zeta, nthreads=16,
                   prec="df", keep=P0.k, maxit=4000, **o) as b:
        t0 = time.perf_counter()
        infos = b.solve(nthreads=16, allow_noconv=True)
        wall = time.perf_counter() - t0
    out["streams_df"] = {"ms": wall * 1e3, "converged": int(sum(i["converged"] for i in infos)),
                         "max_resid": float(max(i["max_resid"] for i in infos))}
    return out


def _spmv_variants(rks) -> dict:
    """Live GB/s of the SpMV+sketch on irregular matrices (algorithmic bytes:
    nnz (8 + 4) + 4 (n + 1) + 16 n per product, CUDA events around every
    launch of one restart of a double-float solve)."""
    from paper_2508_05400_gb300 import inputs as I
    out = {}
    for name, A in (("powerlaw_2e6", I.powerlaw_matrix(2_000_003)), ("wide_rows_1e6", I.wide_rows_matrix(1_000_003))):
        with rks.Solver.from_csr(A, 8, 24, 64, which="LM", tol=1e-12, zeta=8, profile=True, max_restarts=1) as s:
            s.solve()
            st = s.stats()["spmv_sketch"]
            out[name] = {"format": s.spmv_format, "n": A.n, "nnz": A.nnz,
                         "max_row": int((A.rowptr[1:] - A.rowptr[:-1]).max()),
                         "launches": st["launches"], "us_per_launch": 1e3 * st["ms"] / max(st["launches"], 1),
                         "gbs": st["bytes"] / max(st["ms"], 1e-9) / 1e6}
    return out


def _small_oracle_errors(rks, prec: str) -> dict:
    """Per-eigenpair error of this path against the FP64 oracle on the same
    operator family at 20^3 (n = 8000), where the oracle finishes in seconds."""
    import numpy as np
    from oracle import rks as R
    from paper_2508_05400_gb300 import inputs as I
    P = I.convdiff3d_problem(N=20, k=8, p=24, d=96)
    u1 = I.start_vector(P.A.n, 1)
    o = P.solver_opts()
    with rks.Solver.from_csr(P.A, P.k, P.p, P.d, which=P.which, zeta=P.zeta, u1=u1, prec=prec, keep=P.k, **o) as s:
        s.solve(allow_noconv=False)
        lam, _, res = s.eigpairs(want_vectors=False)
    ores = R.rks(P.A.to_scipy(), P.k, P.p, P.d, u1, zeta=P.zeta, seed=0, which=P.which, tol=o["tol"],
                 eta_lock=o["eta_lock"], conv="norm1", keep=P.k)
    errs = _pair_errors(lam[:P.k], ores.eigvals)
    return {"workload": "convdiff3d_20 (n=8000, k=8, p=24, d=96, same field/convection recipe)",
            "per_pair_rel": errs, "max": max(errs), "gpu_max_resid": float(res.max()),
            "oracle_max_resid": float(ores.resid.max())}


def run_batch_only(args) -> None:
    """The persistent batched solve alone on the first COUNT members of the
    batch of uneven 2D operators; one JSON line with its event time."""
    from paper_2508_05400_gb300 import build as B
    B.build()
    from paper_2508_05400_gb300 import inputs as I
    from paper_2508_05400_gb300 import rks
    probs = [I.uneven_convdiff2d_problem(i) for i in range(args.batch_only)]
    P0 = probs[0]
    o = P0.solver_opts()
    with rks.DevBatch([P.A for P in probs], P0.k, P0.p, P0.d, which=P0.which, zeta=P0.zeta, tol=o["tol"],
                      conv="norm1", verify=o["verify"], maxit=args.max_restarts or args.maxit, keep=12,
                      ctas=args.batch_ctas) as b:
        infos = b.solve(allow_noconv=True)
        cfg = b.config()
    print(json.dumps({"workload": "batch of uneven 2D convection-diffusion operators", "count": args.batch_only,
                      "sum_n": int(sum(P.A.n for P in probs)), "ms": cfg["last_ms"],
                      "config": {k: cfg[k] for k in ("GL", "nL", "GS", "nS")},
                      "converged": int(sum(i["converged"] for i in infos)),
                      "restarts": int(sum(i["restarts"] for i in infos))}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="convdiff3d_160", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the other precision paths and the per-eigenpair error records")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--e2e-steps", type=int, default=2, help="solves in the end-to-end leg (mean reported)")
    ap.add_argument("--maxit", type=int, default=4000, help="restart limit of each solve")
    ap.add_argument("--grid", type=int, default=0,
                    help="grid side in place of the workload's (smaller cases for profiling); 0: the workload's")
    ap.add_argument("--max-restarts", type=int, default=0,
                    help="stop every solve after this many restarts (profiling); 0: run to convergence")
    ap.add_argument("--ortho", default="sketch", choices=["sketch", "cgs2"],
                    help="sketch: randomized Gram-Schmidt (rKS); cgs2: the Krylov-Schur baseline "
                         "with Euclidean CGS2 (DF only)")
    ap.add_argument("--keep", type=int, default=-1,
                    help="active Schur vectors a restart keeps after locking (thick restart); "
                         "-1: k; 0: k - q as in Algorithm 1")
    ap.add_argument("--aggressive", action="store_true",
                    help="aggressive deflation: converged Schur blocks move to the front and lock")
    ap.add_argument("--prec", default=None, choices=["df", "fp64", "mixed"],
                    help="arithmetic of the n-dimensional work (see include/rks.h); default: the "
                         "workload's (mixed for the 3D workload)")
    ap.add_argument("--batch-only", type=int, default=0, metavar="COUNT",
                    help="only the persistent batched solve of the first COUNT uneven 2D operators "
                         "(profiling; --max-restarts caps the restarts, --batch-ctas fixes the cluster size)")
    ap.add_argument("--batch-ctas", type=int, default=0, help="CTAs per problem of --batch-only; 0: autotuned")
    ap.add_argument("--spmv-variants-only", action="store_true",
                    help="only the live GB/s of the irregular-row SpMV variants (profiling)")
    args = ap.parse_args()
    if args.spmv_variants_only:
        from paper_2508_05400_gb300 import build as B
        B.build()
        from paper_2508_05400_gb300 import rks
        print(json.dumps(_spmv_variants(rks)))
    elif args.batch_only:
        run_batch_only(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
