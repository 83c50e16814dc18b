#!/usr/bin/env python
"""Benchmark: sub-structured CG time-to-1e-8 on the 128^3 finite-volume system.

Workload: 3D 7-point variable-coefficient diffusion on 128^3 cells
(kappa = exp(g), g ~ N(0,1) per cell, harmonic-mean faces), 4x4x4 box split
into 64 subdomains, b = A x* with x* ~ U[-1,1], seeded.  One step = one
complete solve (Algorithm 3, M = I, in FP64 by default) from x = 0 to a
recursive relative residual of 1e-8, with b already resident on the device.

Prints one JSON line.  Besides the time per solve it reports the roofline of
the dominant kernel (fused sub-structured SpMV + interface assembly) measured
live with CUDA events, the end-to-end time through the host-buffer C ABI
call, the SM clocks sampled during the timed region, each solution's error
against x* and against the oracle's stored FP64 solution, the other modes
(mixed precision, diagonal preconditioner) with their own rooflines, the
other workloads (64^2 Poisson, 96^3 with 16 right-hand sides and gradients,
the 1024^2 finite-element mesh, the 512-system batch, the band splittings)
and, on rank 0 with one GPU, the FP64 CPU oracle timed on complete solves
of the same system on all host cores and on one.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank solves its own replica of the workload (the
path has no cross-GPU exchange on one node: "replicas only"); the reported
time is the maximum over ranks.
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

METRIC = "sub-structured CG time-to-1e-8 rel residual; SpMV+assembly HBM GB/s vs peak"
UNIT = "s"
RTOL = 1e-8
WORKLOAD = "fv3d_7pt_128^3_kappa=exp(N(0,1))_4x4x4_subdomains"
FALLBACK_HBM_GBS = 6800.0
PROFILE_RECORDS = {"fp64": os.path.join(ROOT, "profiles", "spmv_asm_fp64_fv3d128.md"),
                   "fp32": os.path.join(ROOT, "profiles", "spmv_asm_fp32_fv3d128.md")}
KERNEL_SOURCE = os.path.join(ROOT, "paper_2108_13162_gb300", "csrc", "kernels.cuh")
GOLDEN = os.path.join(ROOT, "tests", "golden", "oracle_fv3d_128_4x4x4.json")


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--spmv-reps", type=int, default=30)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mode", choices=("fp64", "mixed", "jacobi", "mixed_jacobi"), default="fp64",
                    help="the headline mode: fp64 = Algorithm 3 in FP64 (the paper's precision); mixed = FP32 "
                         "inner CG inside FP64 iterative refinement; jacobi / mixed_jacobi = the same with the "
                         "diagonal preconditioner.  All stop on an FP64 relative residual of 1e-8; every mode "
                         "is timed and reported")
    ap.add_argument("--no-p2d", action="store_true", help="skip the 64x64 Poisson system (solve to 1e-10)")
    ap.add_argument("--unroll", type=int, default=4, help="CG iterations per pass of the loop graph's body")
    ap.add_argument("--profile-spmm", choices=("fp64", "fp32"), default=None,
                    help="only build the 96^3 16-right-hand-side workload and launch the 16-vector product "
                         "--spmv-reps times (for ncu); no JSON line")
    ap.add_argument("--profile-block", choices=("fp64", "mixed"), default=None,
                    help="only build the 96^3 16-right-hand-side workload and run one solve of all 16 together "
                         "with the host-loop driver (for an ncu launch list); no JSON line")
    ap.add_argument("--profile-batch", choices=("fp64", "mixed"), default=None,
                    help="only build the 512-system batch of sides 32..128 and run one solve of all its "
                         "right-hand sides with the host-loop driver (for an ncu launch list); no JSON line")
    ap.add_argument("--profile-spmv", choices=("fp64", "fp32"), default=None,
                    help="only build the workload and launch the SpMV --spmv-reps times (for ncu); no JSON line")
    ap.add_argument("--profile-fe", choices=("fp64", "fp32"), default=None,
                    help="only build the 1024^2 finite-element workload (the default slice layout) and launch its "
                         "SpMV --spmv-reps times (for ncu); no JSON line")
    ap.add_argument("--profile-p2d", choices=("cluster", "loop"), default=None,
                    help="only build the 64x64 Poisson workload and run --spmv-reps FP64 solves to 1e-10 as the "
                         "one-cluster kernel or the three-kernel loop (for ncu); no JSON line")
    ap.add_argument("--fe-windows", action="store_true",
                    help="also time the 1024^2 finite-element product under every slice-sorting window "
                         "(1, 128, 256, 512, whole subdomain), each autotuned, and report them in fe2d")
    ap.add_argument("--head-only", action="store_true",
                    help="time the headline mode only (not the other modes); for profiler launch lists")
    ap.add_argument("--no-multi-rhs", action="store_true",
                    help="skip the 16-right-hand-side measurement (96^3 FV, reported beside the headline)")
    ap.add_argument("--no-bands", action="store_true",
                    help="skip the band-row / band-column comparison operators and global CG")
    ap.add_argument("--profile-band", choices=("row", "col"), default=None,
                    help="only run the band product of the 128^3 matrix (64 bands) spmv-reps times (for ncu)")
    ap.add_argument("--no-fe", action="store_true",
                    help="skip the 1024^2 P1 finite-element workload (256 RCB subdomains, autotuned SpMV)")
    ap.add_argument("--batch", choices=("off", "small", "full"), default="full",
                    help="many independent systems in one launch, reported beside the headline: full = 512 "
                         "systems of side 32..512 (44.3 M unknowns); small = 512 of side 32..128, also solved "
                         "one after another for comparison")
    ap.add_argument("--driver", choices=("graph", "host"), default="graph",
                    help="graph: one CUDA graph per solve (timed default); host: same kernels launched from a "
                         "host loop (for profilers that cannot see kernels inside conditional graphs)")
    return ap.parse_args(argv)


# ----------------------------------------------------------------------------- distributed helpers
class Dist:
    """Rank bookkeeping for torchrun launches; a no-op for one process."""

    def __init__(self, backend=None):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local_rank = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = False
        if self.world > 1:
            import torch.distributed as dist

            if backend is None:
                import torch

                backend = "nccl" if torch.cuda.is_available() else "gloo"
            if backend == "nccl":
                import torch

                torch.cuda.set_device(self.local_rank)
            dist.init_process_group(backend=backend)
            self.pg = True
            self.backend = backend

    def barrier(self):
        if self.pg:
            import torch.distributed as dist

            if self.backend == "nccl":
                import torch

                dist.barrier(device_ids=[self.local_rank])
            else:
                dist.barrier()

    def max(self, v: float) -> float:
        if not self.pg:
            return float(v)
        import torch
        import torch.distributed as dist

        dev = "cuda:%d" % self.local_rank if self.backend == "nccl" else "cpu"
        t = torch.tensor([float(v)], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    def sum(self, v: float) -> float:
        if not self.pg:
            return float(v)
        import torch
        import torch.distributed as dist

        dev = "cuda:%d" % self.local_rank if self.backend == "nccl" else "cpu"
        t = torch.tensor([float(v)], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.pg:
            import torch.distributed as dist

            dist.destroy_process_group()


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling (200 ms) of SM clocks and throttle reasons."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = str(device_index)
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.dev, "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.remove(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "", 1).isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "", 1).isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower().startswith("active")})
        return {
            "sm_mhz": statistics.median(sm) if sm else None,
            "sm_max_mhz": max(smax) if smax else None,
            "reasons": reasons,
            "samples": len(rows),
        }


def _device_index(local_rank):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v.strip() for v in vis.split(",") if v.strip()]
        if local_rank < len(ids):
            return ids[local_rank]
    return str(local_rank)


# ----------------------------------------------------------------------------- workload
def make_workload():
    from synth import config_problem

    return config_problem(2)


def spmv_algorithmic_bytes(sizes, vb: int = 8) -> int:
    """Bytes the fused sub-structured SpMV must move once per launch with
    vb-byte values and vectors (8: FP64, 4: FP32), int32 indices, each x and
    y entry once: matrix (vb+4)*nnz, row pointers 4*(nloc+1), x and y
    vb*nloc each, interface lists 4*ncopies + 4*(ngamma+1)."""
    return ((vb + 4) * sizes.nnz + 4 * (sizes.nloc + 1) + 2 * vb * sizes.nloc + 4 * sizes.ncopies
            + 4 * (sizes.ngamma + 1))


def time_spmv(S, prec, stream, reps):
    """Average duration of one SpMV launch (CUDA events on its stream)."""
    import torch

    dt = torch.float64 if prec == "fp64" else torch.float32
    xl = torch.rand(S.sizes.nloc, dtype=torch.float64, device="cuda").to(dt)
    y = torch.empty_like(xl)
    for _ in range(3):
        S.spmv_prec(xl, y, prec)
    torch.cuda.synchronize()
    k0 = torch.cuda.Event(enable_timing=True)
    k1 = torch.cuda.Event(enable_timing=True)
    k0.record(stream)
    for _ in range(reps):
        S.spmv_prec(xl, y, prec)
    k1.record(stream)
    torch.cuda.synchronize()
    return k0.elapsed_time(k1) / 1e3 / reps


def spmm_algorithmic_bytes(sizes, k: int, vb: int = 8) -> int:
    """The SpMV bytes with k vectors: the matrix and index arrays once, the x
    and y blocks (k values per local entry) once each."""
    return ((vb + 4) * sizes.nnz + 4 * (sizes.nloc + 1) + 2 * vb * k * sizes.nloc + 4 * sizes.ncopies
            + 4 * (sizes.ngamma + 1))


def time_spmm(S, prec, k, stream, reps):
    """Average duration of one k-vector product launch (CUDA events on its stream)."""
    import torch

    dt = torch.float64 if prec == "fp64" else torch.float32
    xl = torch.rand((S.sizes.nloc, k), dtype=torch.float64, device="cuda").to(dt)
    y = torch.empty_like(xl)
    for _ in range(3):
        S.spmm(xl, y)
    torch.cuda.synchronize()
    k0 = torch.cuda.Event(enable_timing=True)
    k1 = torch.cuda.Event(enable_timing=True)
    k0.record(stream)
    for _ in range(reps):
        S.spmm(xl, y)
    k1.record(stream)
    torch.cuda.synchronize()
    return k0.elapsed_time(k1) / 1e3 / reps


FP64_NOMINAL_TFLOPS = 1.25  # GB300 FP64, nominal: used only if the measurement below fails


def measure_fp64_peak(ctx, dev):
    """The FP64 FMA rate of this GPU (ssg_measure_fp64_rate: every SM busy
    with independent FMA chains, best of 3 launches of about 0.2 s, CUDA
    events), with the SM clocks sampled meanwhile."""
    from paper_2108_13162_gb300 import ssg

    ck = ClockSampler(_device_index(dev))
    ck.start()
    try:
        tflops, ms = ssg.ssg_measure_fp64_rate(ctx.h, 50000, 3)
    finally:
        clocks = ck.stop()
    return {"tflops": tflops, "best_launch_ms": ms, "clocks": clocks,
            "how": "8 x 256-thread blocks per SM, 8 independent DFMA chains per thread, 50000 steps; "
                   "best of 3 launches (CUDA events) after one untimed"}


def bench_multi_rhs(ctx, stream, reps, spmv_reps, fp64_peak=None):
    """The 16-right-hand-side workload (96^3 FV, 27 subdomains): time to 1e-8
    for all 16 with the columns iterating together (K = 16) and one after
    another, FP64, mixed and both with the diagonal preconditioner, the
    differentiable solve (forward + adjoint), and the k-vector product's
    roofline."""
    import numpy as np
    import torch

    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import System
    from synth import config_problem

    p = config_problem(5)
    S = System(ctx, p.A, p.part, p.P)
    B = torch.from_numpy(p.b.T.copy()).cuda()
    X = torch.zeros_like(B)
    out = {"workload": "fv3d_7pt_96^3_kappa=exp(N(0,1))_3x3x3_subdomains_16rhs", "n": p.A.n, "nnz": p.A.nnz,
           "nloc": S.sizes.nloc, "rhs": B.shape[0], "rtol": RTOL,
           "autotune_block": S.autotune_block(16, reps=10)}
    for mode_name, mode in (("fp64", ssg.SSG_FP64), ("mixed", ssg.SSG_MIXED), ("jacobi", ssg.SSG_FP64_JACOBI),
                            ("mixed_jacobi", ssg.SSG_MIXED_JACOBI)):
        for kb in (16, 1):
            ctx.set_rhs_block(kb)
            X.zero_()
            ssg.ssg_solve(S.h, B.shape[0], B, X, False, RTOL, 0, mode)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                rc, st = ssg.ssg_solve(S.h, B.shape[0], B, X, False, RTOL, 0, mode)
            e1.record(stream)
            torch.cuda.synchronize()
            if rc != ssg.SSG_OK:
                raise RuntimeError("16-RHS solve did not converge: %r" % st)
            key = "%s_%s" % (mode_name, "together" if kb == 16 else "one_by_one")
            out[key + "_s"] = e0.elapsed_time(e1) / 1e3 / reps
            out[key + "_iters_max"] = max(s["iters"] for s in st)
            out[key + "_true_relres_max"] = max(s["true_relres"] for s in st)
            out[key + "_launches"] = sum(s["kernel_launches"] for s in st) if kb == 1 else st[0]["kernel_launches"]
    ctx.set_rhs_block(16)
    # the differentiable solve: L = sum_j ||x_j - t_j||^2, gradients with
    # respect to B and the per-cell log conductivities (forward + adjoint)
    from paper_2108_13162_gb300 import autograd as ag

    dims = tuple(p.meta["grid"])
    logk0 = torch.from_numpy(p.meta["log_kappa"].ravel().copy()).cuda()
    Tt = torch.from_numpy(np.random.default_rng(2108).uniform(-1, 1, tuple(B.shape))).cuda()
    for mode_name, mode in (("fp64", ssg.SSG_FP64), ("mixed", ssg.SSG_MIXED)):
        def step():
            lk = logk0.clone().requires_grad_(True)
            Bg = B.clone().requires_grad_(True)
            Xs = ag.solve(S, ag.fv7_values(S, dims, lk), Bg, rtol=RTOL, mode=mode)
            L = torch.sum((Xs - Tt) ** 2)
            L.backward()
            return lk.grad, Bg.grad
        step()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            gk, gb = step()
        e1.record(stream)
        torch.cuda.synchronize()
        out["grad_%s_s" % mode_name] = e0.elapsed_time(e1) / 1e3 / reps
        out["grad_%s_norms" % mode_name] = [float(gk.norm()), float(gb.norm())]
    peak, peak_src = measured_peaks()
    flops = 2.0 * p.A.nnz * 16
    t64 = time_spmm(S, "fp64", 16, stream, spmv_reps)
    t32 = time_spmm(S, "fp32", 16, stream, spmv_reps)
    nb32 = spmm_algorithmic_bytes(S.sizes, 16, 4)
    p64 = fp64_peak["tflops"] if fp64_peak else FP64_NOMINAL_TFLOPS
    out["spmm_fp64_k16"] = {"bound": "alu", "achieved": flops / t64 / 1e12, "peak": p64,
                            "unit": "TFLOP/s", "frac": flops / t64 / 1e12 / p64,
                            "peak_source": "measured FP64 FMA rate (fp64_peak)" if fp64_peak else "nominal FP64 rate",
                            "launch_us": t64 * 1e6,
                            "hbm_gbs": spmm_algorithmic_bytes(S.sizes, 16, 8) / t64 / 1e9}
    out["spmm_fp32_k16"] = {"bound": "hbm", "achieved": nb32 / t32 / 1e9, "peak": peak, "unit": "GB/s",
                            "frac": nb32 / t32 / 1e9 / peak, "peak_source": peak_src, "launch_us": t32 * 1e6,
                            "algorithmic_bytes": nb32}
    S.close()
    return out


def batch_algorithmic_bytes(bp, st, mode_name):
    """Bytes the batch solve must move: for every system, the iterations of
    its K-column loop (the most any of its right-hand sides took; the K
    columns, padding included, run together) times the bytes of one
    iteration -- FP64: the matrix (12 per entry, 4 per row pointer) and 80
    per entry and column (product: x read, y written; residual update: r, q
    read, r written; x/p update: x, p, r read, x, p written); mixed (inner
    FP32 iterations): 8 per matrix entry and 40 per entry and column.
    Counted on the global sizes (interface copies left out), so a lower
    bound."""
    tot = 0
    t = 0
    for A, b in zip(bp.A, bp.b):
        k = b.shape[0]
        K = 2 if k <= 2 else 4 if k <= 4 else 8 if k <= 8 else 16
        its = max(st[t + j]["iters"] for j in range(k))
        t += k
        if mode_name == "fp64":
            per = 12 * A.nnz + 4 * (A.n + 1) + 80 * K * A.n
        else:
            per = 8 * A.nnz + 4 * (A.n + 1) + 40 * K * A.n
        tot += its * per
    return tot


def bench_batch(ctx, stream, reps, size):
    """Workload 4: independent 2D finite-volume systems (4-16 box subdomains,
    1-8 right-hand sides each) solved together in one graph launch, FP64,
    mixed and mixed with the diagonal preconditioner, against the same systems
    solved one after another (FP64, mixed).  size "full":
    512 systems with sides 32..512; "small": 512 systems with sides 32..128."""
    import numpy as np
    import torch

    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import Batch, System
    from synth import batch_problem

    hi = 512 if size == "full" else 128
    bp = batch_problem(512, 32, hi)
    t0 = time.perf_counter()
    B = Batch(ctx, [(A, pt, P, b.shape[0]) for A, pt, P, b in zip(bp.A, bp.part, bp.P, bp.b)])
    setup_s = time.perf_counter() - t0
    tune = B.autotune_block(reps=10)
    bb = torch.from_numpy(np.concatenate([b.ravel() for b in bp.b])).cuda()
    # mixed precision's inner tolerance for this workload: 1e-5 measured best
    # on the batch (4.54 s against 4.75 at the library's default 1e-4; the
    # single 128^3 and FE systems are indifferent, 16 right-hand sides 2 %
    # slower), set for the batch's solves and restored afterwards
    inner_rtol = 1e-5
    ctx.set_mixed(inner_rtol, 30)
    out = {"workload": "fv2d_5pt_batch512_side32-%d_sigma0.5_4-16subdomains_1-8rhs" % hi,
           "systems": len(bp.A), "unknowns": int(sum(A.n for A in bp.A)), "nnz": int(sum(A.nnz for A in bp.A)),
           "rhs": int(sum(b.shape[0] for b in bp.b)), "subdomains": int(sum(bp.P)), "rtol": RTOL,
           "mixed_inner_rtol": inner_rtol, "setup_s": setup_s, "autotune_block": tune}
    for mode_name, mode in (("fp64", ssg.SSG_FP64), ("mixed", ssg.SSG_MIXED), ("mixed_jacobi", ssg.SSG_MIXED_JACOBI)):
        x, rc, st = B.solve(bb, rtol=RTOL, mode=mode)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            x, rc, st = B.solve(bb, rtol=RTOL, mode=mode)
        e1.record(stream)
        torch.cuda.synchronize()
        if rc != ssg.SSG_OK:
            raise RuntimeError("batch solve did not converge")
        out[mode_name + "_together_s"] = e0.elapsed_time(e1) / 1e3 / reps
        out[mode_name + "_iters_max"] = max(t["iters"] for t in st)
        out[mode_name + "_true_relres_max"] = max(t["true_relres"] for t in st)
        out[mode_name + "_launches"] = st[0]["kernel_launches"]
        nb = batch_algorithmic_bytes(bp, st, mode_name)
        sec = out[mode_name + "_together_s"]
        peak, _ = measured_peaks()
        out[mode_name + "_roofline"] = {"algorithmic_bytes": nb, "achieved_gbs": nb / sec / 1e9,
                                        "frac": nb / sec / 1e9 / peak, "peak": peak}
    ctx.set_mixed(1e-4, 30)
    B.close()
    # the same systems one after another (each with its right-hand sides together)
    if size != "full":
        for mode_name, mode in (("fp64", ssg.SSG_FP64), ("mixed", ssg.SSG_MIXED)):
            tot = 0.0
            for A, pt, P, b in zip(bp.A, bp.part, bp.P, bp.b):
                S = System(ctx, A, pt, P)
                bt = torch.from_numpy(b.copy()).cuda()
                S.solve(bt, rtol=RTOL, mode=mode)
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                S.solve(bt, rtol=RTOL, mode=mode)
                e1.record(stream)
                torch.cuda.synchronize()
                tot += e0.elapsed_time(e1) / 1e3
                S.close()
            out[mode_name + "_one_by_one_s"] = tot
    return out


def bench_fe(ctx, stream, reps, windows=False):
    """Workload 3: P1 finite elements on the jittered 1024^2 mesh, 256 uneven
    RCB subdomains: the slice layout the row-length rule picks (rows sorted
    by length in windows) against the unsorted one, the SpMV instances chosen
    by ssg_autotune, the product's roofline in FP64 and FP32, then time to
    1e-8 in FP64, mixed and mixed + Jacobi."""
    import torch

    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import System
    from synth import config_problem

    p = config_problem(3)
    peak, peak_src = measured_peaks()

    def spmv_roofline(Sx):
        """The FE product in both precisions: launch time (CUDA events,
        the autotuned instance) against the algorithmic bytes."""
        rec = {}
        for prec, vb in (("fp64", 8), ("fp32", 4)):
            t = time_spmv(Sx, prec, stream, 50)
            nb = spmv_algorithmic_bytes(Sx.sizes, vb)
            rec[prec] = {"launch_us": t * 1e6, "algorithmic_bytes": nb, "achieved_gbs": nb / t / 1e9,
                         "frac": nb / t / 1e9 / peak, "peak": peak, "peak_source": peak_src}
        return rec

    # the unsorted layout (32 consecutive rows per slice), for comparison
    ctx.set_slice_sort(1)
    try:
        S1 = System(ctx, p.A, p.part, p.P)
    finally:
        ctx.set_slice_sort(0)
    S1.autotune(reps=20)
    unsorted = {"layout": S1.layout(), "spmv": spmv_roofline(S1)}
    S1.close()
    by_window = None
    if windows:
        by_window = {}
        for w in (128, 256, 512, -1):
            ctx.set_slice_sort(w)
            try:
                Sw = System(ctx, p.A, p.part, p.P)
            finally:
                ctx.set_slice_sort(0)
            Sw.autotune(reps=20)
            by_window[str(w)] = {"layout": Sw.layout(), "spmv": spmv_roofline(Sw)}
            Sw.close()
    # the layout the row-length rule picks (the default)
    S = System(ctx, p.A, p.part, p.P)
    tune = S.autotune(reps=20)
    b = torch.from_numpy(p.b[:, 0].copy()).cuda()
    out = {"workload": "fe2d_p1_jittered_1024^2_rcb256", "n": p.A.n, "nnz": p.A.nnz, "subdomains": p.P,
           "nloc": S.sizes.nloc, "rtol": RTOL, "autotune": tune, "layout": S.layout(),
           "iface_layout": S.iface_layout(), "spmv": spmv_roofline(S), "unsorted": unsorted}
    if by_window is not None:
        out["by_window"] = by_window
    for name, mode in (("fp64", ssg.SSG_FP64), ("mixed", ssg.SSG_MIXED), ("mixed_jacobi", ssg.SSG_MIXED_JACOBI)):
        x, rc, st = S.solve(b, rtol=RTOL, mode=mode)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            x, rc, st = S.solve(b, rtol=RTOL, mode=mode)
        e1.record(stream)
        torch.cuda.synchronize()
        if rc != ssg.SSG_OK:
            raise RuntimeError("FE solve did not converge")
        out[name + "_s"] = e0.elapsed_time(e1) / 1e3 / reps
        out[name + "_iters"] = st[0]["iters"]
        out[name + "_true_relres"] = st[0]["true_relres"]
    S.close()
    return out


def band_algorithmic_bytes(n, nnz, nb=0):
    """y = A x on global CSR: values and column ids once (12 B per entry), row
    pointers, x and y once each (band-column: plus its band boundaries)."""
    return 12 * nnz + 4 * (n + 1) + 8 * n + 8 * n


def time_band(B, x, y, stream, reps):
    import torch

    from paper_2108_13162_gb300 import ssg

    ssg.ssg_band_spmv(B.h, x, y)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        ssg.ssg_band_spmv(B.h, x, y)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3 / reps


def bench_bands(ctx, stream, prob, reps, spmv_reps):
    """The paper's other splittings as comparison operators on the 128^3
    matrix, 64 bands (as many as subdomains): band-row and band-column
    products (autotuned kernel, CUDA events, matrix larger than L2), and
    plain global CG (one subdomain) to 1e-8 in FP64 and mixed precision."""
    import numpy as np
    import torch

    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import Band, System

    A = prob.A
    peak, _ = measured_peaks()
    x = torch.from_numpy(np.random.default_rng(5).uniform(-1, 1, A.n)).cuda()
    y = torch.empty_like(x)
    nbytes = band_algorithmic_bytes(A.n, A.nnz)
    out = {"bands": 64, "algorithmic_bytes": nbytes}
    for name, kind in (("row", ssg.SSG_BAND_ROW), ("col", ssg.SSG_BAND_COL)):
        B = Band(ctx, A, kind, 64)
        tune = B.autotune(reps=10)
        t = time_band(B, x, y, stream, spmv_reps)
        out[name] = {"variant": tune["variant"], "rule_variant": tune["rule_variant"], "variants_us": tune["us"],
                     "launch_us": t * 1e6, "achieved_gbs": nbytes / t / 1e9, "frac": nbytes / t / 1e9 / peak}
        B.close()
    S1 = System(ctx, A, np.zeros(A.n, np.int32), 1)
    b = torch.from_numpy(prob.b[:, 0].copy()).cuda()
    for name, mode in (("fp64", ssg.SSG_FP64), ("mixed", ssg.SSG_MIXED)):
        xg, rc, st = S1.solve(b, rtol=RTOL, mode=mode)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            xg, rc, st = S1.solve(b, rtol=RTOL, mode=mode)
        e1.record(stream)
        torch.cuda.synchronize()
        out["global_cg_%s_s" % name] = e0.elapsed_time(e1) / 1e3 / reps
        out["global_cg_%s_iters" % name] = st[0]["iters"]
    out["global_cg_spmv_us"] = time_spmv(S1, "fp64", stream, spmv_reps) * 1e6
    S1.close()
    return out


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def spmv_source_sha256():
    """sha256 of the SpMV kernel's own source: the regions of kernels.cuh
    between the [spmv-source-begin] / [spmv-source-end] markers, joined."""
    text = open(KERNEL_SOURCE).read()
    parts = []
    pos = 0
    while True:
        a = text.find("[spmv-source-begin]", pos)
        if a < 0:
            break
        b = text.index("[spmv-source-end]", a)
        parts.append(text[a:b])
        pos = b
    return hashlib.sha256("".join(parts).encode()).hexdigest()


def profiled_traffic(prec="fp64"):
    """Per-launch DRAM bytes from the committed ncu summary, only if the
    kernel source is unchanged since the counters were taken."""
    try:
        text = open(PROFILE_RECORDS[prec]).read()
        src = spmv_source_sha256()
    except OSError:
        return None
    rec = {}
    for line in text.splitlines():
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            rec[k.strip()] = v.strip().strip("`")
    if rec.get("kernel_source_sha256") != src:
        return None
    try:
        return int(rec["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def golden_samples():
    """The oracle's stored results for the 128^3 workload (written by
    tests/golden/make_oracle_golden.py, which calls only the oracle): the
    sample indices, its FP64 solutions there (to 1e-8 and 1e-12) and its
    iteration counts per mode."""
    import numpy as np

    try:
        with open(GOLDEN) as f:
            d = json.load(f)
        out = {"idx": np.array(d["sample_idx"], dtype=np.int64), "oracle_iters": {}}
        for rec in d["solves"]:
            out["fp64_%g" % rec["rtol"]] = np.array(rec["sample_x"])
            if rec["rtol"] == RTOL:
                out["oracle_iters"]["fp64"] = int(rec["iters"])
        for m in ("mixed", "jacobi", "mixed_jacobi"):
            if m in d:
                out["oracle_iters"][m] = int(d[m]["iters"])
        return out
    except (OSError, KeyError, ValueError):
        return None


def bench_p2d(ctx, stream, reps):
    """Workload 1: the 64x64 5-point Poisson system on 2x2 subdomains, plain
    FP64 CG to 1e-10.  The whole system (0.33 MB) sits in L2, so latency, not
    HBM, bounds it: the figures are the time per solve and per iteration,
    with the error against the oracle's stored solution, for the one-cluster
    solve (the default at this size: every iteration inside one launch) and
    for the three-kernel loop graph."""
    import numpy as np
    import torch

    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import System
    from synth import config_problem

    rtol = 1e-10
    p = config_problem(1)
    S = System(ctx, p.A, p.part, p.P)
    b = torch.from_numpy(p.b[:, 0].copy()).cuda()
    x = torch.zeros_like(b)
    try:
        with open(os.path.join(ROOT, "tests", "golden", "oracle_p2d_64_2x2.json")) as f:
            g = json.load(f)
    except (OSError, ValueError):
        g = None
    limit, ctas = ctx.cluster_solve()

    def timed():
        for _ in range(3):
            x.zero_()
            ssg.ssg_solve(S.h, 1, b, x, False, rtol, 0, ssg.SSG_FP64)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            x.zero_()
            rc, st = ssg.ssg_solve(S.h, 1, b, x, False, rtol, 0, ssg.SSG_FP64)
        e1.record(stream)
        torch.cuda.synchronize()
        if rc != ssg.SSG_OK:
            raise RuntimeError("64x64 solve did not converge")
        t = e0.elapsed_time(e1) / 1e3 / reps
        xh = x.cpu().numpy()
        xs = p.xstar[:, 0]
        r = {"s": t, "iters": st[0]["iters"], "us_per_iter": t * 1e6 / max(st[0]["iters"], 1),
             "kernel_launches": st[0]["kernel_launches"], "true_relres": st[0]["true_relres"],
             "err_vs_xstar": float(np.linalg.norm(xh - xs) / np.linalg.norm(xs))}
        if g is not None:
            xo = np.array(g["x"])
            r["err_vs_oracle_fp64"] = float(np.linalg.norm(xh - xo) / np.linalg.norm(xo))
        return r

    out = {"workload": "poisson2d_5pt_64x64_2x2_subdomains", "n": p.A.n, "nnz": p.A.nnz,
           "nloc": S.sizes.nloc, "rtol": rtol, "mode": "fp64",
           "l2": "L2-resident (0.33 MB): latency-bound, no HBM roofline"}
    if g is not None:
        out["oracle_iters"] = int(g["iters"])
    try:
        ctx.set_cluster_solve(0)
        out["loop"] = timed()
    finally:
        ctx.set_cluster_solve(limit)
    if ctas > 0 and S.sizes.nloc <= limit:
        out["cluster"] = dict(timed(), ctas=ctas)
    head = out.get("cluster", out["loop"])
    for k in ("s", "iters", "us_per_iter", "true_relres", "err_vs_xstar", "err_vs_oracle_fp64"):
        if k in head:
            out[k] = head[k]
    S.close()
    return out


# ----------------------------------------------------------------------------- CPU oracle
def cpu_info():
    """Host CPU: logical cores (nproc) and the model name lscpu prints (or
    /proc/cpuinfo's, or the platform's)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() == "Model name":
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith("model name"):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    if not model:
        import platform

        model = platform.processor() or platform.machine()
    return {"nproc": os.cpu_count(), "cpu_model": model}


def oracle_solves(part, b, count, threads):
    """Complete FP64 solves of the oracle's sub-structured CG to RTOL from
    x = 0: threads 1 = the plain single-threaded oracle (or_sub_cg), else
    the subdomains shared among that many OpenMP threads (or_sub_cg_omp,
    0 = all).  Returns (seconds of each solve, last result)."""
    import oracle

    times = []
    r = None
    for _ in range(count):
        t0 = time.perf_counter()
        if threads == 1:
            r = part.cg(b, RTOL, 100000)
        else:
            r = part.cg_omp(b, RTOL, 100000, threads)
        times.append(time.perf_counter() - t0)
        if r.status != oracle.OK:
            raise RuntimeError("oracle solve did not converge (status %d)" % r.status)
    return times, r


def cpu_baseline_leg(prob):
    """The oracle on the host cores, one complete solve each: on every
    OpenMP thread (the baseline's value) and on one thread."""
    import oracle

    part = oracle.Partition(prob.A, prob.part, prob.P)
    b = prob.b[:, 0]
    nt = oracle.omp_max_threads()
    t_all, r_all = oracle_solves(part, b, 1, 0)
    t_one, r_one = oracle_solves(part, b, 1, 1)
    info = cpu_info()
    return {
        "value": t_all[0], "unit": UNIT, "cores": nt, "kind": "oracle",
        "sample": "one complete FP64 solve of the same 128^3 system to 1e-8 (%d iterations) by the oracle's "
                  "sub-structured CG with the 64 subdomains shared among %d OpenMP threads; one thread: %.2f s "
                  "(%d iterations)" % (r_all.iters, nt, t_one[0], r_one.iters),
        "iters": r_all.iters,
        "single_thread_s": t_one[0],
        "single_thread_iters": r_one.iters,
        **info,
    }


def run_reference(args, dist):
    """The reference arm: the paper gives no code, so the FP64 oracle's
    sub-structured CG (plain C, the subdomains shared among all host cores)
    solves the same 128^3 system from x = 0 to 1e-8, one complete solve per
    step, warm-up steps untimed."""
    if dist.rank != 0:
        return 0
    import numpy as np

    import oracle

    prob = make_workload()
    part = oracle.Partition(prob.A, prob.part, prob.P)
    b = prob.b[:, 0]
    nt = oracle.omp_max_threads()
    oracle_solves(part, b, max(args.warmup, 0), 0)
    times, r = oracle_solves(part, b, args.steps, 0)
    value = statistics.mean(times)
    info = cpu_info()
    tr = float(np.linalg.norm(b - oracle.spmv(prob.A, r.x)) / np.linalg.norm(b))
    line = {
        "impl": "reference",
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": args.gpus,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": value * 1e3,
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": reference_config(prob, dist.world),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": nt, "kind": "oracle",
                         "sample": "%d complete FP64 solves to 1e-8 (%d iterations each) by the oracle's "
                                   "sub-structured CG, 64 subdomains shared among %d OpenMP threads, after %d "
                                   "untimed" % (args.steps, r.iters, nt, args.warmup),
                         "iters": r.iters, "true_relres": tr, "step_s": times, **info},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def reference_config(prob, world):
    """The config keys both arms print, with the same values."""
    return {"workload": WORKLOAD, "n": prob.A.n, "nnz": prob.A.nnz, "subdomains": prob.P, "rtol": RTOL,
            "mode": "fp64", "parallelism": "replicas" if world > 1 else "single"}


# ----------------------------------------------------------------------------- our arm
def run_ours(args, dist):
    import numpy as np
    import torch

    from paper_2108_13162_gb300 import build as ssg_build
    from paper_2108_13162_gb300 import ssg
    from paper_2108_13162_gb300.ssg import Context, System

    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA GPU")
    ssg_build.build()
    dev = dist.local_rank
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    ctx = Context(dev, stream)
    if args.profile_block:
        from synth import config_problem

        p5 = config_problem(5)
        S = System(ctx, p5.A, p5.part, p5.P)
        ctx.set_driver(ssg.SSG_DRIVER_HOST)
        B = torch.from_numpy(p5.b.T.copy()).cuda()
        X = torch.zeros_like(B)
        mode = ssg.SSG_MIXED if args.profile_block == "mixed" else ssg.SSG_FP64
        rc, st = ssg.ssg_solve(S.h, B.shape[0], B, X, False, RTOL, 0, mode)
        torch.cuda.synchronize()
        print("block solve: status %d, iterations %d, launches %d" % (rc, max(t["iters"] for t in st),
                                                                      st[0]["kernel_launches"]))
        S.close()
        ctx.close()
        return 0
    if args.profile_batch:
        import numpy as np

        from paper_2108_13162_gb300.ssg import Batch
        from synth import batch_problem

        bp = batch_problem(512, 32, 128)
        Bt = Batch(ctx, [(A, pt, P, b.shape[0]) for A, pt, P, b in zip(bp.A, bp.part, bp.P, bp.b)])
        ctx.set_driver(ssg.SSG_DRIVER_HOST)
        bb = torch.from_numpy(np.concatenate([b.ravel() for b in bp.b])).cuda()
        mode = ssg.SSG_MIXED if args.profile_batch == "mixed" else ssg.SSG_FP64
        x, rc, st = Bt.solve(bb, rtol=RTOL, mode=mode)
        torch.cuda.synchronize()
        print("batch solve (%s): status %d, iterations %d, launches %d" % (
            args.profile_batch, rc, max(t["iters"] for t in st), st[0]["kernel_launches"]))
        Bt.close()
        ctx.close()
        return 0 if rc == ssg.SSG_OK else 1
    if args.profile_spmm:
        from synth import config_problem

        p5 = config_problem(5)
        S = System(ctx, p5.A, p5.part, p5.P)
        time_spmm(S, args.profile_spmm, 16, stream, args.spmv_reps)
        S.close()
        ctx.close()
        return 0
    if args.profile_p2d:
        from synth import config_problem

        p1 = config_problem(1)
        if args.profile_p2d == "loop":
            ctx.set_cluster_solve(0)
        S = System(ctx, p1.A, p1.part, p1.P)
        b1 = torch.from_numpy(p1.b[:, 0].copy()).cuda()
        x1 = torch.zeros_like(b1)
        for _ in range(args.spmv_reps):
            x1.zero_()
            rc, st = ssg.ssg_solve(S.h, 1, b1, x1, False, 1e-10, 0, ssg.SSG_FP64)
        torch.cuda.synchronize()
        print("64x64 solve (%s): rc %d, %d iterations, %d launches, %.3f ms" % (
            args.profile_p2d, rc, st[0]["iters"], st[0]["kernel_launches"], st[0]["solve_ms"]))
        S.close()
        ctx.close()
        return 0 if rc == ssg.SSG_OK else 1
    prob = make_workload()
    if args.profile_band:
        from paper_2108_13162_gb300.ssg import Band

        B = Band(ctx, prob.A, ssg.SSG_BAND_ROW if args.profile_band == "row" else ssg.SSG_BAND_COL, 64)
        xb = torch.from_numpy(prob.b[:, 0].copy()).cuda()
        t = time_band(B, xb, torch.empty_like(xb), stream, args.spmv_reps)
        print("band-%s product: %.1f us (rule variant)" % (args.profile_band, t * 1e6))
        B.close()
        ctx.close()
        return 0
    if args.profile_fe:
        from synth import config_problem

        p3 = config_problem(3)
        S = System(ctx, p3.A, p3.part, p3.P)
        t = time_spmv(S, args.profile_fe, stream, args.spmv_reps)
        print("fe2d product (%s): %.1f us, layout %r" % (args.profile_fe, t * 1e6, S.layout()))
        S.close()
        ctx.close()
        return 0
    if args.profile_spmv:
        S = System(ctx, prob.A, prob.part, prob.P)
        time_spmv(S, args.profile_spmv, stream, args.spmv_reps)
        S.close()
        ctx.close()
        return 0
    if args.driver == "host":
        ctx.set_driver(ssg.SSG_DRIVER_HOST)
    ctx.set_unroll(args.unroll)
    S = System(ctx, prob.A, prob.part, prob.P)
    # setup, outside the timed region: the product's launch shape for this system
    tune = S.autotune(reps=20)
    b = torch.from_numpy(prob.b[:, 0].copy()).to("cuda:%d" % dev)
    x = torch.zeros_like(b)
    modes = {"fp64": ssg.SSG_FP64, "mixed": ssg.SSG_MIXED, "jacobi": ssg.SSG_FP64_JACOBI,
             "mixed_jacobi": ssg.SSG_MIXED_JACOBI}
    gold = golden_samples()
    xstar = prob.xstar[:, 0]

    def solve(mode):
        x.zero_()
        rc, st = ssg.ssg_solve(S.h, 1, b, x, False, RTOL, 0, modes[mode])
        if rc != ssg.SSG_OK:
            raise RuntimeError("solve did not converge: %r" % st)
        return st[0]

    def timed(mode, steps, clocks=None):
        """K solves bracketed by a barrier and a device sync on both sides,
        CUDA events on the solve stream; returns (ms per step, stats list)."""
        if clocks:
            clocks.start()
        dist.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        sts = []
        e0.record(stream)
        for _ in range(steps):
            sts.append(solve(mode))
        e1.record(stream)
        torch.cuda.synchronize()
        dist.barrier()
        ck = clocks.stop() if clocks else None
        return dist.max(e0.elapsed_time(e1) / steps), sts, ck

    def accuracy(xg):
        """Relative error of the GPU solution against x* (exact) and against
        the oracle's FP64 solutions to 1e-8 and 1e-12 at the stored samples."""
        xh = xg.cpu().numpy()
        out = {"err_vs_xstar": float(np.linalg.norm(xh - xstar) / np.linalg.norm(xstar))}
        if gold:
            idx = gold["idx"]
            for key in ("1e-08", "1e-12"):
                ref = gold["fp64_" + key]
                out["err_vs_oracle_fp64_%s_sampled" % key] = float(np.linalg.norm(xh[idx] - ref)
                                                                     / np.linalg.norm(ref))
        return out

    # the headline: plain FP64 (the paper's precision), then the other modes
    # on the same system with the same protocol
    results = {}
    for mode in ([args.mode] + ([] if args.head_only else [m for m in modes if m != args.mode])):
        for _ in range(max(args.warmup, 0)):
            solve(mode)
        ms, sts, ck = timed(mode, args.steps, ClockSampler(_device_index(dev)) if mode == args.mode else None)
        iters = [t["iters"] for t in sts]
        results[mode] = {"ms": ms, "sts": sts, "clocks": ck, "iters": int(statistics.median(iters)),
                         "accuracy": accuracy(x)}
    head = results[args.mode]
    launches = sum(t["kernel_launches"] for t in head["sts"])

    # end to end through the host-buffer C ABI call (pinned host memory)
    bh = torch.from_numpy(prob.b[:, 0].copy()).pin_memory().numpy()
    xh = torch.zeros(prob.A.n, dtype=torch.float64).pin_memory().numpy()
    ssg.ssg_solve_host(S.h, 1, bh, xh, False, RTOL, 0, modes[args.mode])
    dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        rc, _ = ssg.ssg_solve_host(S.h, 1, bh, xh, False, RTOL, 0, modes[args.mode])
    e2e_s = dist.max((time.perf_counter() - t0) / args.steps)

    # this GPU's FP64 FMA rate: the co-bound of the FP64 kernels
    try:
        fp64_peak = measure_fp64_peak(ctx, dev)
    except Exception as e:  # noqa: BLE001 - reported, the nominal rate is used then
        fp64_peak = {"error": str(e)}
    fp64_ok = fp64_peak if "tflops" in fp64_peak else None

    # roofline of the dominant kernel of each mode: the fused SpMV + interface
    # assembly, CUDA events on the launching stream, matrix larger than L2
    peak, peak_src = measured_peaks()
    roof = {}
    for prec in ("fp64", "fp32"):
        spmv_s = time_spmv(S, prec, stream, args.spmv_reps)
        nbytes = spmv_algorithmic_bytes(S.sizes, 4 if prec == "fp32" else 8)
        achieved = nbytes / spmv_s / 1e9
        roof[prec] = {
            "kernel": "k_spmv_asm<%s> (fused local CSR SpMV + interface assembly + (p,Sp)_w partials)"
                      % ("float" if prec == "fp32" else "double"),
            "bound": "hbm",
            "achieved": achieved,
            "peak": peak,
            "peak_source": peak_src,
            "unit": "GB/s",
            "frac": achieved / peak,
            "traffic": profiled_traffic(prec),
            "algorithmic_bytes": nbytes,
            "launch_us": spmv_s * 1e6,
        }
        if prec == "fp64" and fp64_ok:
            # the co-bound: one FMA per stored entry (2 flops) against the measured FP64 rate
            tf = 2.0 * S.sizes.nnz / spmv_s / 1e12
            roof[prec]["fp64_pipe"] = {"achieved_tflops": tf, "peak_tflops": fp64_ok["tflops"],
                                       "frac": tf / fp64_ok["tflops"]}
    prec_of = {"fp64": "fp64", "jacobi": "fp64", "mixed": "fp32", "mixed_jacobi": "fp32"}

    def mode_record(mode):
        r = results[mode]
        st = r["sts"][-1]
        rec = {"s": r["ms"] / 1e3, "iters": r["iters"], "outer": st["outer"], "true_relres": st["true_relres"],
               "us_per_iter": r["ms"] * 1e3 / max(r["iters"], 1), **r["accuracy"]}
        if gold and mode in gold["oracle_iters"]:
            rec["oracle_iters"] = gold["oracle_iters"][mode]
        rec["roofline"] = roof[prec_of[mode]]
        return rec

    multi = None
    if not args.no_multi_rhs:
        multi = bench_multi_rhs(ctx, stream, max(1, min(args.steps, 3)), args.spmv_reps, fp64_ok)
    fe = None
    if not args.no_fe:
        fe = bench_fe(ctx, stream, max(1, min(args.steps, 3)), args.fe_windows)
    bands = None
    if not args.no_bands:
        bands = bench_bands(ctx, stream, prob, max(1, min(args.steps, 3)), args.spmv_reps)
    p2d = None
    if not args.no_p2d:
        p2d = bench_p2d(ctx, stream, max(args.steps, 5))
    batch = None
    if args.batch != "off":
        batch = bench_batch(ctx, stream, 1 if args.batch == "full" else max(1, min(args.steps, 3)), args.batch)

    cpu = None
    if dist.rank == 0 and dist.world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_leg(prob)

    ms_step = head["ms"]
    value = ms_step / 1e3
    cfg = reference_config(prob, dist.world)
    cfg["mode"] = args.mode
    cfg.update({
        "nloc": S.sizes.nloc,
        "interface_nodes": S.sizes.ngamma,
        "iters": head["iters"],
        "outer": head["sts"][-1]["outer"],
        "true_relres": head["sts"][-1]["true_relres"],
        "us_per_iter": ms_step * 1e3 / head["iters"],
        **head["accuracy"],
        "l2": "inputs larger than L2 (175 MB matrix + 5 x 18 MB vectors > 129 MB)",
        "driver": args.driver,
        "unroll": args.unroll,
        "autotune": tune,
        # interface slices or groups in the FP64 product (ssg_get_iface_layout)
        "iface_layout": S.iface_layout(),
    })
    if gold and args.mode in gold["oracle_iters"]:
        cfg["oracle_iters"] = gold["oracle_iters"][args.mode]
    line = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": dist.world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_step,
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64" if args.mode in ("fp64", "jacobi") else "f32+f64",
        "data": "synthetic",
        "config": cfg,
        "roofline": roof[prec_of[args.mode]],
        "e2e": {"value": e2e_s, "unit": UNIT, "h2d_bytes_per_step": 8 * prob.A.n, "d2h_bytes_per_step": 8 * prob.A.n},
        "gpu_launches": int(dist.sum(launches)),
        "clocks": head["clocks"],
        "cpu_baseline": cpu,
        "fp64_peak": fp64_peak,
        "modes": {m: mode_record(m) for m in modes if m != args.mode and m in results},
        "p2d64": p2d,
        "multi_rhs": multi,
        "batch": batch,
        "fe2d": fe,
        "splittings": bands,
    }
    if dist.rank == 0:
        print(json.dumps(line), flush=True)
    S.close()
    ctx.close()
    return 0


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        # rank 0 alone times the CPU oracle; other ranks exit without work
        dist = Dist.__new__(Dist)
        dist.world = int(os.environ.get("WORLD_SIZE", "1"))
        dist.rank = int(os.environ.get("RANK", "0"))
        dist.local_rank = int(os.environ.get("LOCAL_RANK", "0"))
        dist.pg = False
        return run_reference(args, dist)
    dist = Dist()
    try:
        return run_ours(args, dist)
    finally:
        dist.close()


if __name__ == "__main__":
    sys.exit(main())
