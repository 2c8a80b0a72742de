#!/usr/bin/env python
"""Benchmark of the variable-order fractional FE operator on GB300.

Metric: H^2 stiffness matvec DOF*RHS/s (with the CG time to tolerance).
Workload (default 'disk33k'): the 2D unit disk + annulus to R = 1.1, 96 rings
(34,027 vertices, 27,361 interior DoFs), s = 0.25 + 0.5(0.5 + 0.5 sin 2 pi x1
cos 2 pi x2), log a a seeded 16-mode Fourier field (sigma 0.5), s_bar = 0.9,
leaf size 64, admissibility lambda = 0.75, tensor Chebyshev order p = 8
(rank 64: an order at which the H^2 operator meets the matvec tolerance 1e-6
against the exact quadrature matrix on this disk, with a margin), FP64,
1 RHS, CG to 1e-10, f = 1.

One step = one pass of the whole hot path on device-resident inputs:
vfd_assemble (field values, coupling blocks, dense near blocks, singular
near field, density sweep, weighted mass) followed by vfd_solve (CG to
rtol).  value = n_dof * nrhs * (operator applications in the step) / step
time, i.e. matvec throughput delivered inside the full assemble + solve step;
ms_per_step is the time to a 1e-10 solution from the fields.

Outside the timed region the line also carries:
  "matvec_rel_err_vs_oracle"  sampled exact rows of A x (CPU oracle) against
                              the GPU apply, for this operator (rank 64) and
                              rank 16;
  "rank16_operator"           the same step with p = 4 (rank 16);
  "batched_mixed_precision"   64 seeded load vectors: the batched apply and
                              the mixed-precision solve to 1e-8 (TF32 / BF16
                              near panels, inner far field of rank 16, FP64
                              residuals of the rank-64 operator) against FP64
                              CG on all 64 columns on the same GPU;
  "batch_24_meshes"           24 squares and disks of 2k to 130k DoFs (rank
                              16), one batched solve vs per-mesh solves.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|fp32]
  python bench.py --impl reference ...     (the CPU oracle on a bounded sample)

Multi-GPU: replicas only (the method has no data-parallel exchange step at
one mesh); each rank solves its own replica, value sums the ranks, time is
the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "H^2 stiffness matvec DOF*RHS/s and CG time-to-tolerance (assemble + solve step)"
UNIT = "DOF*RHS/s"
FP64_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12   # GB300: 2 FP64 FMA per clock per SM at 2.07 GHz


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    p.add_argument("--workload", default="disk33k")
    p.add_argument("--precision", default="fp64", choices=["fp64", "fp32", "bf16"])
    p.add_argument("--nrhs", type=int, default=1, help="columns for --mode apply / solve")
    p.add_argument("--rtol", type=float, default=1e-10)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-batched", action="store_true", help="skip the 64-RHS mixed-precision leg")
    p.add_argument("--no-batch24", action="store_true", help="skip the 24-mesh batched leg")
    p.add_argument("--no-graded", action="store_true", help="skip the graded-exterior leg")
    p.add_argument("--no-ball", action="store_true", help="skip the 3D ball leg")
    p.add_argument("--no-grad", action="store_true", help="skip the gradient leg")
    p.add_argument("--mode", default="step", choices=["step", "apply", "solve"],
                   help="apply: assemble once, then --steps applies of --parts (bounded run for profilers)")
    p.add_argument("--parts", type=int, default=15, help="VFD_PART_* mask for --mode apply")
    p.add_argument("--precondition", type=int, default=0, help="VFD_PREC_* kind for --mode solve")
    p.add_argument("--near-config", type=int, default=-1,
                   help="--mode apply, low precision, 64-column multiples: pin the near-panel configuration")
    return p.parse_args()


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def replica_value(units, seconds, dist=None, device="cuda"):
    """Whole-job throughput of independent replicas (one per rank): the units
    all ranks processed divided by the slowest rank's time.  Returns (value,
    max seconds)."""
    if dist is None:
        return units / seconds, seconds
    import torch
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    s = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(s, op=dist.ReduceOp.MAX)
    return float(u.item()) / float(s.item()), float(s.item())


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        # the samples are summarised into the JSON line; the raw CSV goes to a
        # scratch directory (VFD_CLOCKS_DIR if set)
        d = os.environ.get("VFD_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(d, f"vfd_clocks_rank{gpu_index}_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        with open(self.path) as fh:
            return summarise_clocks(fh)


def summarise_clocks(lines):
    """Median SM clock, maximum SM clock and the throttle reasons seen active in
    nvidia-smi CSV lines of ClockSampler.Q (no header, no units)."""
    sm, smax, reasons = [], None, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in lines:
        f = [x.strip() for x in line.split(",")]
        if len(f) < 9:
            continue
        try:
            sm.append(float(f[1]))
            smax = float(f[2])
        except ValueError:
            continue
        for nm, v in zip(names, f[5:9]):
            if v.lower().startswith("active"):
                reasons.add(nm)
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
            "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------
# CPU oracle leg (bounded sample of the same workload)
# ----------------------------------------------------------------------------
def oracle_step_value(K=24, rtol=1e-10):
    """The oracle as it stands (dense FP64 assembly + plain CG) on a smaller
    disk of the same workload family; returns (value, seconds, n_dof, iters)."""
    import numpy as np

    import oracle
    import synth
    m = synth.disk_mesh(K, R=1.1, jitter=0.2, seed=2000 + K)
    s = synth.config2_s_field()
    k = synth.random_fourier_field(2001, 0.5)
    t0 = time.perf_counter()
    A = oracle.assemble(m, s, k, s_bar=0.9, n_sing=3)
    F = oracle.load(m, np.ones(m.n_vert))
    U, it = oracle.cg(A.A, F, rtol)
    t = time.perf_counter() - t0
    return A.N * (it + 1) / t, t, A.N, it


def reference_arm(args):
    rank, world, _ = _dist()
    if rank != 0:
        return
    import oracle
    K = 20
    for _ in range(args.warmup):
        oracle_step_value(K, args.rtol)
    vals, secs, n, its = [], [], 0, []
    for _ in range(args.steps):
        v, t, n, it = oracle_step_value(K, args.rtol)
        vals.append(v)
        secs.append(t)
        its.append(it)
    tot = sum(secs)
    value = n * sum(i + 1 for i in its) / tot
    cores = oracle.num_threads()
    sample = f"disk K={K} ({n} DoFs): dense FP64 oracle assembly + CG to {args.rtol:g}, per step"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": args.workload, "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------
def main():
    args = _args()
    if args.impl == "reference":
        return reference_arm(args)
    import numpy as np
    import torch

    import synth
    from paper_2302_02863_gb300 import vfd

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    vfd.load()
    m, s, k, prm = synth.workload(args.workload)
    prec = {"fp64": vfd.VFD_FP64, "fp32": vfd.VFD_FP32, "bf16": vfd.VFD_BF16}[args.precision]
    mesh = vfd.vfd_mesh(m.d, m.coords, m.cells, m.cell_is_interior, leaf_m=prm["leaf"], cheb_p=prm["p"],
                        lam=prm["lam"], rho_lambda=prm["lam"], tail_mode=prm["tail"], tail_R=prm["R"],
                        inner_p=prm.get("inner_p", 0))
    info = mesh.info
    n = mesh.n_dof
    if args.mode in ("apply", "solve"):
        return apply_mode(args, mesh, s, k, prm, prec, torch, vfd)
    stream = torch.cuda.current_stream()
    F = torch.zeros(n, dtype=torch.float64, device="cuda")
    vfd.vfd_load(mesh, torch.ones(m.n_vert, dtype=torch.float64, device="cuda"), F)
    U = torch.zeros_like(F)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2

    def step(timed=False):
        op = vfd.vfd_assemble(mesh, s, k, prm["s_bar"], precision=prec,
                              flags=vfd.VFD_ASSEMBLE_TIMED if timed else 0)
        U.zero_()
        st, it, rel = vfd.vfd_solve(op, F, U, rtol=args.rtol, max_it=100000)
        return op, st, int(it[0]), float(rel[0])

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    times, iters, rels, phases = [], [], [], []
    for _ in range(args.steps):
        flush.zero_()                        # L2 flush between timed steps (not timed)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        op, st, it, rel = step(timed=True)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) / 1000.0)
        iters.append(it)
        rels.append(rel)
        phases.append(vfd.vfd_op_timings(op))
        del op
    clk = clocks.stop()
    tot = sum(times)
    n_apply = sum(i + 2 for i in iters)          # CG iterations + initial and final residual
    value, tot = replica_value(n * n_apply, tot, dist, "cuda")

    # ---- e2e: the same step through the C ABI with HOST buffers (copies timed)
    Fh = F.cpu().numpy().copy()
    Uh = np.zeros(n)
    for _ in range(2):
        op = vfd.vfd_assemble(mesh, s, k, prm["s_bar"], precision=prec)
        Uh[:] = 0
        vfd.vfd_solve(op, Fh, Uh, rtol=args.rtol, max_it=100000, stream=0)
        del op
    torch.cuda.synchronize()
    e2e_t, e2e_apply = 0.0, 0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        op = vfd.vfd_assemble(mesh, s, k, prm["s_bar"], precision=prec, stream=0)
        Uh[:] = 0
        st, it, rel = vfd.vfd_solve(op, Fh, Uh, rtol=args.rtol, max_it=100000, stream=0)
        e2e_t += time.perf_counter() - t0
        e2e_apply += int(it[0]) + 2
        del op
    e2e_value = world * n * e2e_apply / e2e_t

    # ---- dominant-kernel roofline, measured live on the launching stream
    op = vfd.vfd_assemble(mesh, s, k, prm["s_bar"], precision=prec, flags=vfd.VFD_ASSEMBLE_TIMED)
    ph = {key: statistics.mean(p[key] for p in phases) for key in phases[0]}
    X = torch.randn(n, dtype=torch.float64, device="cuda")
    Y = torch.empty_like(X)
    parts_near = vfd.VFD_PART_B | vfd.VFD_PART_M | vfd.VFD_PART_KNEAR   # one kernel: fused leaf/near/CSR rows
    for _ in range(5):
        vfd.vfd_apply_parts(op, parts_near, X, Y)
    R = 50
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record(stream)
    for _ in range(R):
        vfd.vfd_apply_parts(op, parts_near, X, Y)
    ev[1].record(stream)
    torch.cuda.synchronize()
    t_leaf = ev[0].elapsed_time(ev[1]) / R / 1000.0
    ev[0].record(stream)
    for _ in range(R):
        vfd.vfd_apply(op, X, Y)
    ev[1].record(stream)
    torch.cuda.synchronize()
    t_apply = ev[0].elapsed_time(ev[1]) / R / 1000.0
    wbytes = 8 if prec == vfd.VFD_FP64 else 4
    leaf_bytes = info["near_entries"] * wbytes + info["nnz"] * 12 + (n + 1) * 4 + 2 * n * 8
    leaf_flops = 2.0 * (info["near_entries"] + info["nnz"])
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    if prec == vfd.VFD_FP64:
        # FP64 FMA rate bounds this kernel on GB300 (1 FMA per 8 bytes of the
        # streamed matrix > 1.25 TFLOP/s / 6.8 TB/s); nominal FP64 peak
        roof = {"bound": "alu", "achieved": leaf_flops / t_leaf / 1e12, "peak": FP64_TFLOPS, "unit": "TFLOP/s",
                "frac": leaf_flops / t_leaf / 1e12 / FP64_TFLOPS, "traffic": None,
                "kernel": "k_near_csr<double,double> (near panels + B+M CSR rows)",
                "peak_source": "152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz",
                "hbm_frac": leaf_bytes / t_leaf / 1e9 / hbm}
    else:
        roof = {"bound": "hbm", "achieved": leaf_bytes / t_leaf / 1e9, "peak": hbm, "unit": "GB/s",
                "frac": leaf_bytes / t_leaf / 1e9 / hbm, "traffic": None,
                "kernel": "k_near_csr<float,float> (near panels + B+M CSR rows)", "peak_source": "MEASURED_PEAKS.json hbm_gbs"}
    roof["algorithmic_bytes"] = leaf_bytes
    roof["launch_us"] = t_leaf * 1e6
    roof["traffic"] = _traffic_from_profile(args.workload, args.precision)
    roof_apply = roof
    # the assembly's two largest kernels: FP64-pipe bound (their DRAM traffic is
    # negligible); throughput in kernel evaluations per second from the live
    # phase timings (mean over the timed assemblies)
    asm_k = {}
    for name, key, ev in (("k_singular2d", "singular", "sing_points"), ("k_near_build", "near", "near_point_pairs")):
        if info.get(ev) and ph.get(key):
            asm_k[name] = {"bound": "alu (FP64 pipe)", "unit": "Geval/s", "evals": info[ev], "ms": round(ph[key], 3),
                           "achieved": info[ev] / (ph[key] / 1e3) / 1e9}
    # the step's largest kernel (launch list share) is the near-block build: an
    # FP64-ALU roofline in kernel evaluations per second, peak = the FP64 issue
    # rate of the part (152 SMs x 2 FP64 instructions/clk x 2.07 GHz = 0.629e12/s,
    # which the measured FMA rate matches) divided by the FP64 instructions of one
    # evaluation as implemented (2D: r^2 4, exponent 3, table-driven log 11, exp
    # 12 = 30; the leaf contractions come on top)
    if prec == vfd.VFD_FP64 and "k_near_build" in asm_k:
        peak_ev = FP64_TFLOPS / 2 * 1e12 / 30 / 1e9
        nb = asm_k["k_near_build"]
        roof = {"bound": "alu", "kernel": "k_near_build (dense inadmissible leaf blocks, Sec. 5.2)",
                "achieved": nb["achieved"], "peak": peak_ev, "unit": "Geval/s", "frac": nb["achieved"] / peak_ev,
                "traffic": _profile_value("k_near_build", args.workload, args.precision, "dram_bytes_per_launch"),
                "fp64_pipe_active_ncu": _profile_value("k_near_build", args.workload, args.precision,
                                                       "fp64_pipe_active"),
                "evals_per_launch": nb["evals"], "fp64_inst_per_eval": 30, "launch_ms": nb["ms"],
                "peak_source": "FP64 issue rate from unit counts and clock (0.629e12/s) / 30 FP64 instructions"}

    # apply: far projections, node sums, coupling, row kernel, far expansion
    apply_kernels = 5 if info["far_blocks"] > 0 else 1
    mean_it = statistics.mean(iters)
    replays = math.ceil(mean_it / 8)
    per_solve = apply_kernels + 4 + replays * 8 * (apply_kernels + 3) + apply_kernels + 2
    per_assemble = 4 + 1 + 2 + 2 + 1 + 1 + 1 + (4 if prec == vfd.VFD_FP32 else 0)
    gpu_launches = args.steps * (per_assemble + per_solve)

    # ---- the same step with rank 16 (p = 4): throughput and error of the lower order
    mesh16 = vfd.vfd_mesh(m.d, m.coords, m.cells, m.cell_is_interior, leaf_m=prm["leaf"], cheb_p=4,
                          lam=prm["lam"], rho_lambda=prm["lam"], tail_mode=prm["tail"], tail_R=prm["R"])
    r16 = rank16_leg(mesh16, s, k, prm, F, args, vfd, torch, flush, stream)

    # ---- matvec error: every row against the exact-mode operator (every block
    # near, direct density: the GPU's evaluation of the quadrature matrix
    # itself), and sampled rows of all three against the oracle's exact rows
    # (CPU leg)
    mesh_x = vfd.vfd_mesh(m.d, m.coords, m.cells, m.cell_is_interior, leaf_m=prm["leaf"], lam=0.0, rho_lambda=0.0,
                          tail_mode=prm["tail"], tail_R=prm["R"])
    rows = sampled_rows_gpu({"operator": mesh, "rank16": mesh16, "exact_mode": mesh_x}, m, s, k, prm, prec, vfd,
                            torch)
    del mesh_x

    grad = None if args.no_grad else gradient_leg(m, k, prm, torch, vfd)
    recomp = recompress_leg(m, s, k, prm, F, torch, vfd) if prec == vfd.VFD_FP64 else None
    if recomp is not None and not args.no_batched:
        recomp["mixed_64rhs_pcg"] = recompress_mixed_leg(m, s, k, prm, torch, vfd)
    prec_leg = precond_leg(mesh, s, k, prm, F, torch, vfd) if prec == vfd.VFD_FP64 else None
    graded = None if args.no_graded else graded_leg(torch, vfd)
    ball = None if args.no_ball else ball_leg(torch, vfd)

    batched = None
    if not args.no_batched:
        batched = batched_leg(mesh, s, k, prm, torch, vfd, hbm=hbm)
    batch24 = None
    if not args.no_batch24:
        batch24 = batch24_leg(torch, vfd, hbm=hbm)

    cpu, mv_err = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu, mv_err = cpu_leg(args, m, s, k, prm, rows, n)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000 * tot / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == vfd.VFD_FP64 else "f64+f32",
            "data": "synthetic",
            "config": {"workload": args.workload, "n_dof": n, "nrhs": 1, "precision": args.precision,
                       "rtol": args.rtol, "leaf": prm["leaf"], "rank": info["rank"], "lambda": prm["lam"],
                       "matvec_tolerance": 1e-6, "l2": "flushed between timed steps (256 MB write)",
                       "parallelism": f"replicas x{world}"},
            "matvec_rel_err_vs_oracle": mv_err,
            "cg_iters": iters[0], "relres": rels[0],
            "assemble_ms": ph["total"], "phases_ms": {k2: round(v2, 3) for k2, v2 in ph.items()},
            "solve_ms": 1000 * tot / args.steps - ph["total"], "apply_us": t_apply * 1e6,
            "apply_dof_rhs_per_s": n / t_apply,
            "roofline": roof, "roofline_apply": roof_apply, "assembly_kernels": asm_k, "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 2 * n * 8, "d2h_bytes_per_step": n * 8},
            "gpu_launches": gpu_launches, "clocks": clk, "mesh": info, "rank16_operator": r16,
            "graded_exterior": graded, "ball_3d": ball, "batched_mixed_precision": batched,
            "batch_24_meshes": batch24, "gradient": grad, "preconditioner": prec_leg, "recompression": recomp,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def graded_leg(torch, vfd, mc=128, grade=1.5, rtol=1e-10):
    """The square of Sec. 7.2 at T_6 (mc = 128, 16,129 DoFs): quasi-uniform
    exterior (131,072 cells) against a graded exterior (cells growing by the
    factor `grade` away from the interface): mesh sizes, assembly phases, CG
    solve to rtol with f = 1, and the relative difference of the solutions
    (s = 0.7, log kappa = 0; rank 16, lambda 0.75)."""
    import numpy as np

    import synth
    s, k = synth.const_field(0.7), synth.const_field(0.0)
    out = {"mc": mc, "grade": grade, "fields": "s = 0.7, kappa = 1"}
    sols = {}
    for name, m in (("uniform", synth.square_mesh(mc)), ("graded", synth.square_mesh_graded(mc, grade))):
        mesh = vfd.vfd_mesh(2, m.coords, m.cells, m.cell_is_interior)
        info = mesh.info
        n = mesh.n_dof
        F = torch.zeros(n, dtype=torch.float64, device="cuda")
        vfd.vfd_load(mesh, torch.ones(m.n_vert, dtype=torch.float64, device="cuda"), F)
        vfd.vfd_assemble(mesh, s, k, 0.9)   # warm-up
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        op = vfd.vfd_assemble(mesh, s, k, 0.9, flags=vfd.VFD_ASSEMBLE_TIMED)
        U = torch.zeros_like(F)
        st, it, rel = vfd.vfd_solve(op, F, U, rtol=rtol, max_it=100000)
        e1.record()
        torch.cuda.synchronize()
        ph = vfd.vfd_op_timings(op)
        dof, _ = vfd.vfd_mesh_dofs(mesh)
        inner = np.abs(m.coords).max(axis=1) < 1.0 - 1e-9
        order = np.lexsort((m.coords[inner, 0], m.coords[inner, 1]))
        u = np.zeros(m.n_vert)
        sel = dof >= 0
        u[sel] = U.cpu().numpy()[dof[sel]]
        sols[name] = u[inner][order]
        out[name] = {"cells": info["n_cell"], "n_q": info["n_q"], "n_dof": n, "rho_near_pairs": info["rho_near_pairs"],
                     "assemble_ms": round(ph["total"], 2), "density_ms": round(ph["density"], 2),
                     "singular_ms": round(ph["singular"], 2), "step_ms": e0.elapsed_time(e1), "cg_iters": int(it[0])}
    out["solution_rel_diff"] = float(np.linalg.norm(sols["graded"] - sols["uniform"]) /
                                     np.linalg.norm(sols["uniform"]))
    out["step_speedup"] = out["uniform"]["step_ms"] / out["graded"]["step_ms"]
    return out


def ball_leg(torch, vfd, n=40, nrhs=16):
    """The 3D configuration on a smaller ball: the Kuhn-grid ball with n^3 cubes
    (n = 40: spacing 0.055, 22,321 DoFs; the full configuration has n = 88),
    Gaussian-bump order and 3D Fourier log kappa, leaf 64, p = 4 (rank 64),
    lambda 0.75.  B is not included: the paper gives no singular rules for
    tetrahedron pairs (reading R20), so the operator is K + M.  FP64 assembly,
    apply and CG (f = 1, to 1e-8); 16 seeded right-hand sides solved to 1e-8
    with FP32 / TF32 coupling and FP64 residuals against FP64 CG."""
    import synth
    m, s, k, prm = synth.ball_workload(n)
    t0 = time.perf_counter()
    mesh = vfd.vfd_mesh(3, m.coords, m.cells, m.cell_is_interior, leaf_m=prm["leaf"], cheb_p=prm["p"],
                        lam=prm["lam"], rho_lambda=prm["lam"])
    t_setup = time.perf_counter() - t0
    info = mesh.info
    N = mesh.n_dof
    op = vfd.vfd_assemble(mesh, s, k, prm["s_bar"], flags=vfd.VFD_ASSEMBLE_TIMED)
    ph = vfd.vfd_op_timings(op)
    X = torch.randn(N, dtype=torch.float64, device="cuda")
    Y = torch.empty_like(X)
    for _ in range(3):
        vfd.vfd_apply(op, X, Y)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(10):
        vfd.vfd_apply(op, X, Y)
    e1.record()
    torch.cuda.synchronize()
    ta = e0.elapsed_time(e1) / 10 / 1000.0
    F = torch.zeros(N, dtype=torch.float64, device="cuda")
    vfd.vfd_load(mesh, torch.ones(m.n_vert, dtype=torch.float64, device="cuda"), F)
    U = torch.zeros_like(F)
    e0.record()
    st, it, rel = vfd.vfd_solve(op, F, U, rtol=1e-8, max_it=100000)
    e1.record()
    torch.cuda.synchronize()
    out = {"workload": f"Kuhn ball n={n}", "n_dof": N, "cells": info["n_cell"], "rank": info["rank"],
           "note": "B not included (no tetrahedron-pair singular rules): operator K + M",
           "mesh_setup_s_host": t_setup, "assemble_ms": round(ph["total"], 1),
           "phases_ms": {kk: round(v, 1) for kk, v in ph.items()}, "near_point_pairs": info["near_point_pairs"],
           "apply_ms": ta * 1e3, "apply_dof_rhs_per_s": N / ta, "cg_iters": int(it[0]),
           "solve_ms": e0.elapsed_time(e1), "status": int(st)}
    g = torch.Generator(device="cuda").manual_seed(5000)
    Fb = torch.randn(nrhs, N, dtype=torch.float64, device="cuda", generator=g)
    U64 = torch.zeros_like(Fb)
    e0.record()
    vfd.vfd_solve(op, Fb, U64, rtol=1e-8, max_it=100000)
    e1.record()
    torch.cuda.synchronize()
    t64 = e0.elapsed_time(e1)
    op32 = vfd.vfd_assemble(mesh, s, k, prm["s_bar"], precision=vfd.VFD_FP32)
    U = torch.zeros_like(Fb)
    vfd.vfd_solve(op32, Fb, U, rtol=1e-8, max_it=100000)   # warm-up (tuning, capture)
    U.zero_()
    e0.record()
    st, it, rel = vfd.vfd_solve(op32, Fb, U, rtol=1e-8, max_it=100000)
    e1.record()
    torch.cuda.synchronize()
    out["mixed_16rhs"] = {"nrhs": nrhs, "fp64_cg_ms": t64, "mixed_ms": e0.elapsed_time(e1), "status": int(st),
                          "inner_iters": int(it[0]), "relres_max": float(rel.max()),
                          "solution_rel_err_vs_fp64_cg": (torch.linalg.norm(U - U64, dim=1) /
                                                          torch.linalg.norm(U64, dim=1)).max().item()}
    return out


def rank16_leg(mesh16, s, k, prm, F, args, vfd, torch, flush, stream, steps=3):
    """The headline step on the rank-16 (p = 4) operator of the same disk."""
    def step():
        op = vfd.vfd_assemble(mesh16, s, k, prm["s_bar"])
        U = torch.zeros_like(F)
        st, it, rel = vfd.vfd_solve(op, F, U, rtol=args.rtol, max_it=100000)
        return int(it[0])
    step()
    ts, its = [], []
    for _ in range(steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        its.append(step())
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1) / 1000.0)
    n = mesh16.n_dof
    return {"rank": mesh16.info["rank"], "ms_per_step": 1000 * statistics.mean(ts), "cg_iters": its[0],
            "value": n * sum(i + 2 for i in its) / sum(ts), "unit": UNIT}


def sampled_rows_gpu(meshes, m, s, k, prm, prec, vfd, torch, nrows=24, seed=2024):
    """A x on the GPU for a seeded x at nrows seeded interior vertices, per
    operator; the vertices and x are in vertex order so the CPU leg can
    compare with the oracle's exact rows."""
    import numpy as np
    rng = np.random.default_rng(seed)
    x_v = rng.standard_normal(m.n_vert)          # x by vertex (only DoF vertices matter)
    out = {"x_vertex": x_v}
    full = {}
    for name, mesh in meshes.items():
        dof, n = vfd.vfd_mesh_dofs(mesh)
        sel = np.nonzero(dof >= 0)[0]
        if "verts" not in out:
            out["verts"] = rng.choice(sel, nrows, replace=False)
        xg = np.zeros(n)
        xg[dof[sel]] = x_v[sel]
        op = vfd.vfd_assemble(mesh, s, k, prm["s_bar"])
        X = torch.tensor(xg, device="cuda")
        Y = torch.empty_like(X)
        vfd.vfd_apply(op, X, Y)
        torch.cuda.synchronize()
        y = Y.cpu().numpy()
        out[name] = y[dof[out["verts"]]]
        yv = np.zeros(m.n_vert)
        yv[sel] = y[dof[sel]]
        full[name] = yv
        del op
    ref = full.get("exact_mode")
    if ref is not None:
        out["all_rows_vs_exact_mode"] = {nm: float(np.linalg.norm(full[nm] - ref) / np.linalg.norm(ref))
                                         for nm in full if nm != "exact_mode"}
    return out


def cpu_leg(args, m, s, k, prm, rows, n):
    """The oracle on the host cores: (1) the dense FP64 step (assembly + plain
    CG) on disks of 16, 20 and 24 rings (the bounded sample), all threads,
    and the 16-ring disk single-threaded; the step time fitted as a power of
    the DoF count and extrapolated to the benchmark disk (labelled
    extrapolated); (2) the exact rows of A x at the sampled vertices of the
    benchmark disk, against the GPU operators' rows."""
    import numpy as np

    import oracle
    cores = oracle.num_threads()
    pts = []
    for K in (16, 20, 24):
        v, t, ns, it = oracle_step_value(K, args.rtol)
        pts.append((ns, t, it))
    oracle.set_threads(1)
    v1, t1, n1, it1 = oracle_step_value(16, args.rtol)
    oracle.set_threads(cores)
    Ns = np.log([p[0] for p in pts])
    Ts = np.log([p[1] for p in pts])
    b, a = np.polyfit(Ns, Ts, 1)
    t_ext = float(np.exp(a + b * np.log(n)))
    n24, t24, it24 = pts[-1]
    cpu = {"value": n24 * (it24 + 1) / t24, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"disks of 16/20/24 rings ({', '.join(str(p[0]) for p in pts)} DoFs, same fields): dense FP64 "
                     f"oracle assembly + plain CG to {args.rtol:g}; value from the 24-ring step ({t24:.1f} s)",
           "step_s": {str(p[0]): round(p[1], 3) for p in pts},
           "single_thread": {"n_dof": n1, "step_s": round(t1, 3), "value": n1 * (it1 + 1) / t1},
           "extrapolated": {"n_dof": n, "step_s": t_ext, "fit": f"t ~ N^{b:.2f}",
                            "note": "extrapolated from the fit, not measured"}}
    # matvec parity on sampled exact rows
    dof_o, N = oracle.dofs(m)
    xo = np.zeros(N)
    sel = dof_o >= 0
    xo[dof_o[sel]] = rows["x_vertex"][sel]
    y_or = oracle.apply_rows(m, s, k, xo, dof_o[rows["verts"]], s_bar=prm["s_bar"], n_sing=3, tail=prm["tail"],
                             R=prm["R"])
    err = {"rows": int(len(rows["verts"])),
           "definition": "seeded N(0,1) x; all_rows_vs_exact_mode = ||A x - A_exact x||_2 / ||A_exact x||_2 over "
                         "every row, A_exact the GPU operator without low-rank blocks (itself checked here on the "
                         "sampled rows); per operator over the sampled rows i: rel2 = ||(Ax)_s - (Ax)_s,oracle||_2 / "
                         "||(Ax)_s,oracle||_2, relmax = max |(Ax)_i - (Ax)_i,oracle| / max |(Ax)_i,oracle|",
           "all_rows_vs_exact_mode": rows.get("all_rows_vs_exact_mode")}
    for name in ("operator", "rank16", "exact_mode"):
        d = rows[name] - y_or
        err[name] = {"rel2": float(np.linalg.norm(d) / np.linalg.norm(y_or)),
                     "relmax": float(np.abs(d).max() / np.abs(y_or).max())}
    return cpu, err


def batched_leg(mesh, s, k, prm, torch, vfd, nrhs=64, rtol=1e-8, hbm=6800.0):
    """The mixed-precision batched path against the plain FP64 path on the same
    operator: 64 seeded N(0,1) load vectors; the batched apply (device-resident
    FP64 column-major X, as the C ABI takes it) and the mixed-precision solve
    to rtol (TF32 and BF16 near panels, the inner far field at the mesh's
    inner order, FP64 residuals of the full operator); FP64 CG on all 64
    columns (column by column) on the same GPU."""
    n = mesh.n_dof
    g = torch.Generator(device="cuda").manual_seed(3000)
    F = torch.randn(nrhs, n, dtype=torch.float64, device="cuda", generator=g)
    X = torch.randn(nrhs, n, dtype=torch.float64, device="cuda", generator=g)
    Y = torch.empty_like(X)
    info = mesh.info
    out = {"nrhs": nrhs, "rtol": rtol, "rhs": "seeded N(0,1)", "rank": info["rank"],
           "inner_rank": info["inner_rank"]}

    def ev_time(fn, reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps / 1000.0

    op64 = vfd.vfd_assemble(mesh, s, k, prm["s_bar"], precision=vfd.VFD_FP64)
    vfd.vfd_apply(op64, X, Y)
    Y64 = Y.clone()
    U64 = torch.zeros_like(F)
    torch.cuda.synchronize()
    t64 = ev_time(lambda: vfd.vfd_solve(op64, F, U64.zero_(), rtol=rtol, max_it=100000), 1)
    st, it64, rel64 = vfd.vfd_solve(op64, F, U64.zero_(), rtol=rtol, max_it=100000)
    ta64 = ev_time(lambda: vfd.vfd_apply(op64, X, Y), 3)
    out["fp64"] = {"apply_us": ta64 * 1e6, "apply_dof_rhs_per_s": n * nrhs / ta64, "solve_ms": 1000 * t64,
                   "cg_iters_mean": float(sum(it64) / len(it64)), "cols_timed": nrhs, "status": int(st)}
    # the same with the two-level preconditioner (setup timed separately)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    vfd.vfd_precondition(op64)
    torch.cuda.synchronize()
    tsu64 = time.perf_counter() - t0
    Up = torch.zeros_like(F)
    vfd.vfd_solve(op64, F[:1], Up[:1], rtol=rtol, max_it=100000)   # graph capture
    tp64 = ev_time(lambda: vfd.vfd_solve(op64, F, Up.zero_(), rtol=rtol, max_it=100000), 1)
    st, itp, _ = vfd.vfd_solve(op64, F, Up.zero_(), rtol=rtol, max_it=100000)
    out["fp64_pcg"] = {"setup_s": tsu64, "solve_ms": 1000 * tp64, "cg_iters_mean": float(sum(itp) / len(itp)),
                       "status": int(st),
                       "solution_rel_err_vs_fp64_cg": (torch.linalg.norm(Up - U64, dim=1) /
                                                       torch.linalg.norm(U64, dim=1)).max().item()}
    for name, prec, wbytes in (("tf32", vfd.VFD_FP32, 4), ("bf16", vfd.VFD_BF16, 2)):
        op = vfd.vfd_assemble(mesh, s, k, prm["s_bar"], precision=prec)
        for _ in range(3):
            vfd.vfd_apply(op, X, Y)
        ta = ev_time(lambda: vfd.vfd_apply(op, X, Y), 20)
        err_apply = (torch.linalg.norm(Y - Y64, dim=1) / torch.linalg.norm(Y64, dim=1)).max().item()
        U = torch.zeros_like(F)
        vfd.vfd_solve(op, F, U, rtol=rtol, max_it=100000)   # warm-up (graph capture)
        U.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        st, it, rel = vfd.vfd_solve(op, F, U, rtol=rtol, max_it=100000)
        e1.record()
        torch.cuda.synchronize()
        ts = e0.elapsed_time(e1) / 1000.0
        err_sol = (torch.linalg.norm(U - U64, dim=1) / torch.linalg.norm(U64, dim=1)).max().item()
        # preconditioned (two-level, FP32 inverses in the batched iteration)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        vfd.vfd_precondition(op)
        torch.cuda.synchronize()
        tsu = time.perf_counter() - t0
        Up = torch.zeros_like(F)
        vfd.vfd_solve(op, F, Up, rtol=rtol, max_it=100000)   # warm-up (graph capture)
        Up.zero_()
        torch.cuda.synchronize()
        e0.record()
        stp, itp, relp = vfd.vfd_solve(op, F, Up, rtol=rtol, max_it=100000)
        e1.record()
        torch.cuda.synchronize()
        tsp = e0.elapsed_time(e1) / 1000.0
        pcg = {"setup_s": tsu, "solve_ms": tsp * 1000, "status": int(stp), "inner_iters": int(itp[0]),
               "ms_per_inner_iter": tsp * 1000 / max(1, int(itp[0])), "relres_max": float(relp.max()),
               "solution_rel_err_vs_fp64_cg": (torch.linalg.norm(Up - U64, dim=1) /
                                               torch.linalg.norm(U64, dim=1)).max().item(),
               "speedup_vs_fp64_cg": t64 / tsp, "speedup_vs_fp64_pcg": tp64 / tsp}
        vfd.vfd_precondition(op, vfd.VFD_PREC_NONE)
        bt = vfd.vfd_batch_create([op])
        vfd.vfd_batch_apply(bt, [X], [Y])
        chosen, cand_us = vfd.vfd_batch_tuning(bt)
        del bt
        # the tuned near phase alone (its time from the tuner, warm L2): panel entries
        # once from HBM (unpadded count), x in and y out once, and the B + M rows
        # (CSR values and columns) where they are not folded into the panels (BF16)
        t_near = min(u for u in cand_us if u > 0) * 1e-6
        near_bytes = info["near_entries"] * wbytes + 2 * n * nrhs * 4 + \
            (info["nnz"] * 8 + (n + 1) * 4 if prec == vfd.VFD_BF16 else n * 4)
        out[name] = {"apply_us": ta * 1e6, "apply_dof_rhs_per_s": n * nrhs / ta,
                     "near_kernel_tuned": {"stage_cols": chosen[0], "stages": chosen[1], "split": chosen[2],
                                           "warps": chosen[3], "acc_sets": chosen[4], "tcgen05": chosen[5]},
                     "apply_rel_err_vs_fp64": err_apply, "solve_ms": ts * 1000, "status": int(st),
                     "inner_iters": int(it[0]), "ms_per_inner_iter": ts * 1000 / max(1, int(it[0])),
                     "relres_max": float(rel.max()), "solution_rel_err_vs_fp64_cg": err_sol,
                     "speedup_vs_fp64_solve": t64 / ts, "preconditioned": pcg,
                     "near_kernel_roofline": {"bound": "hbm", "launch_us": t_near * 1e6,
                                              "algorithmic_bytes": near_bytes,
                                              "achieved_gbs": near_bytes / t_near / 1e9, "peak_gbs": hbm,
                                              "frac": near_bytes / t_near / 1e9 / hbm,
                                              "peak_source": "MEASURED_PEAKS.json hbm_gbs"}}
        del op
    del op64
    return out


def batch24_leg(torch, vfd, nrhs=64, rtol=1e-8, hbm=6800.0):
    """Many meshes at once: the 24 squares and disks of synth.batch_workload
    (2k to 130k DoFs, 773,540 in all, each with its own fields), 64 seeded
    N(0,1) load vectors per mesh, one batched refinement solve to rtol over
    all meshes (TF32 and BF16 near panels), and the batch apply throughput;
    against the same per-mesh batched solves run one mesh after another."""
    from concurrent.futures import ThreadPoolExecutor

    import synth
    W = synth.batch_workload()
    t0 = time.perf_counter()

    def mk(w):
        m = w[0]
        return vfd.vfd_mesh(2, m.coords, m.cells, m.cell_is_interior, leaf_m=64, cheb_p=4, lam=0.75,
                            rho_lambda=0.75)

    with ThreadPoolExecutor(16) as ex:
        meshes = list(ex.map(mk, W))
    t_setup = time.perf_counter() - t0
    ntot = sum(mm.n_dof for mm in meshes)
    out = {"meshes": len(meshes), "n_dof_total": ntot, "n_dof_min": min(mm.n_dof for mm in meshes),
           "n_dof_max": max(mm.n_dof for mm in meshes), "nrhs": nrhs, "rtol": rtol,
           "mesh_setup_s_host": t_setup, "rhs": "seeded N(0,1)"}
    g = torch.Generator(device="cuda").manual_seed(4000)
    Fs = [torch.randn(nrhs, mm.n_dof, dtype=torch.float64, device="cuda", generator=g) for mm in meshes]
    for name, prec in (("tf32", vfd.VFD_FP32), ("bf16", vfd.VFD_BF16)):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ops = [vfd.vfd_assemble(mesh, w[1], w[2], 0.9, precision=prec) for mesh, w in zip(meshes, W)]
        e1.record()
        torch.cuda.synchronize()
        t_asm = e0.elapsed_time(e1) / 1000.0
        batch = vfd.vfd_batch_create(ops)
        Ys = [torch.empty_like(f) for f in Fs]
        for _ in range(2):
            vfd.vfd_batch_apply(batch, Fs, Ys)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(5):
            vfd.vfd_batch_apply(batch, Fs, Ys)
        e1.record()
        torch.cuda.synchronize()
        ta = e0.elapsed_time(e1) / 5 / 1000.0
        Us = [torch.zeros_like(f) for f in Fs]
        e0.record()
        st, it, rel = vfd.vfd_batch_solve(batch, Fs, Us, rtol=rtol, max_it=200000)
        e1.record()
        torch.cuda.synchronize()
        ts = e0.elapsed_time(e1) / 1000.0
        Us2 = [torch.zeros_like(f) for f in Fs]
        e0.record()
        for op, F, U in zip(ops, Fs, Us2):
            vfd.vfd_solve(op, F, U, rtol=rtol, max_it=200000)
        e1.record()
        torch.cuda.synchronize()
        tseq = e0.elapsed_time(e1) / 1000.0
        chosen, _ = vfd.vfd_batch_tuning(batch)
        # preconditioned: every operator gets the two-level preconditioner
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for op in ops:
            vfd.vfd_precondition(op)
        torch.cuda.synchronize()
        tsu = time.perf_counter() - t0
        Us3 = [torch.zeros_like(f) for f in Fs]
        e0.record()
        stp, itp, relp = vfd.vfd_batch_solve(batch, Fs, Us3, rtol=rtol, max_it=200000)
        e1.record()
        torch.cuda.synchronize()
        tsp = e0.elapsed_time(e1) / 1000.0
        Us4 = [torch.zeros_like(f) for f in Fs]
        e0.record()
        for op, F, U in zip(ops, Fs, Us4):
            vfd.vfd_solve(op, F, U, rtol=rtol, max_it=200000)
        e1.record()
        torch.cuda.synchronize()
        tseqp = e0.elapsed_time(e1) / 1000.0
        pcg = {"setup_s": tsu, "solve_s": tsp, "status": int(stp), "inner_iters_max": int(itp.max()),
               "relres_max": float(relp.max()), "solved_dof_rhs_per_s": ntot * nrhs / tsp,
               "sequential_per_mesh_solves_s": tseqp}
        out[name] = {"assemble_s": t_asm, "apply_ms": ta * 1000, "apply_dof_rhs_per_s": ntot * nrhs / ta,
                     "near_kernel_tuned": {"stage_cols": chosen[0], "stages": chosen[1], "split": chosen[2],
                                           "warps": chosen[3], "acc_sets": chosen[4], "tcgen05": chosen[5]},
                     "solve_s": ts, "status": int(st), "inner_iters_max": int(it.max()),
                     "relres_max": float(rel.max()), "solved_dof_rhs_per_s": ntot * nrhs / ts,
                     "sequential_per_mesh_solves_s": tseq, "preconditioned": pcg}
        del batch, ops
    return out


def _vertex_fields(k, x):
    """P1 (vertex) values of the benchmark fields: the disk's s(x) and its
    Fourier log-kappa rows (input generation only)."""
    import numpy as np

    s_n = 0.25 + 0.5 * (0.5 + 0.5 * np.sin(2 * math.pi * x[:, 0]) * np.cos(2 * math.pi * x[:, 1]))
    lk = np.full(len(x), float(k.c0))
    for row in np.asarray(k.fourier, dtype=float).reshape(-1, 5):
        lk += row[3] * np.cos(math.pi * (x @ row[:2]) + row[4])
    return s_n, lk


def gradient_leg(m, k, prm, torch, vfd, n_dir=4, h=1e-6, rtol=1e-12):
    """The differentiation workload on the benchmark disk and operator (H^2,
    rank 64) with P1 s and log kappa: loss ||u - u_obs||^2 in the lumped mass
    norm, u_obs from a seeded reference s field.  Times vfd_grad alone and the
    autograd forward (assembly + solve) and backward (adjoint solve + vfd_grad),
    and checks the gradient against central differences along n_dir seeded
    directions (the full 20-direction check is a GPU test)."""
    import numpy as np

    import synth
    from paper_2302_02863_gb300 import inverse
    from paper_2302_02863_gb300.autograd import solve as vsolve

    x = m.coords
    s_n, lk_n = _vertex_fields(k, x)
    s_ref = np.clip(s_n + 0.05 * np.sin(3.0 * x[:, 0] + 1.0) * np.cos(2.0 * x[:, 1]), 0.1, 0.85)
    mesh = vfd.vfd_mesh(m.d, m.coords, m.cells, m.cell_is_interior, leaf_m=prm["leaf"], cheb_p=prm["p"],
                        lam=prm["lam"], rho_lambda=prm["lam"], tail_mode=prm["tail"], tail_R=prm["R"])
    dev = "cuda"
    t0 = time.perf_counter()
    op = vfd.vfd_assemble(mesh, synth.nodal_field(s_n), synth.nodal_field(lk_n), prm["s_bar"])
    torch.cuda.synchronize()
    first_assemble_s = time.perf_counter() - t0          # includes the nodes' nearest-point location
    F = torch.zeros(mesh.n_dof, dtype=torch.float64, device=dev)
    vfd.vfd_load(mesh, torch.ones(m.n_vert, dtype=torch.float64, device=dev), F)
    m_l = inverse.lumped_mass(mesh, m.n_vert, dev)
    lk_t = torch.tensor(lk_n, device=dev)
    with torch.no_grad():
        u_obs = vsolve(torch.tensor(s_ref, device=dev), lk_t, F, mesh, prm["s_bar"], rtol)
    # vfd_grad alone (U the solution, Lam a solve for a seeded right-hand side)
    U = torch.zeros_like(F)
    vfd.vfd_solve(op, F, U, rtol=rtol, max_it=100000)
    g = torch.Generator(device=dev).manual_seed(9)
    Lam = torch.randn(mesh.n_dof, dtype=torch.float64, device=dev, generator=g)
    gs = torch.empty(m.n_vert, dtype=torch.float64, device=dev)
    gk = torch.empty_like(gs)
    stream = torch.cuda.current_stream()
    vfd.vfd_grad(op, U, Lam, gs, gk)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record(stream)
    for _ in range(3):
        vfd.vfd_grad(op, U, Lam, gs, gk)
    ev[1].record(stream)
    torch.cuda.synchronize()
    grad_ms = ev[0].elapsed_time(ev[1]) / 3

    def J(sv, lv):
        e = vsolve(sv, lv, F, mesh, prm["s_bar"], rtol) - u_obs
        return (m_l * e * e).sum()

    s_t = torch.tensor(s_n, device=dev, requires_grad=True)
    l_t = torch.tensor(lk_n, device=dev, requires_grad=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    loss = J(s_t, l_t)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    loss.backward()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    rng = np.random.default_rng(4)
    worst = 0.0
    with torch.no_grad():
        for _ in range(n_dir):
            vs = torch.tensor(rng.standard_normal(m.n_vert), device=dev)
            vl = torch.tensor(rng.standard_normal(m.n_vert), device=dev)
            fd = (J(s_t + h * vs, l_t + h * vl) - J(s_t - h * vs, l_t - h * vl)).item() / (2 * h)
            ad = ((s_t.grad * vs).sum() + (l_t.grad * vl).sum()).item()
            worst = max(worst, abs(ad - fd) / abs(fd))
    return {"workload": "benchmark disk, P1 s and log kappa, H^2 rank 64", "n_vert": m.n_vert,
            "n_dof": mesh.n_dof, "vfd_grad_ms": round(grad_ms, 3), "forward_s": round(t1 - t0, 4),
            "backward_s": round(t2 - t1, 4), "first_assemble_s_incl_node_location": round(first_assemble_s, 3),
            "fd_directions": n_dir, "fd_h": h, "fd_max_rel_gap": worst, "loss": loss.item()}


def precond_leg(mesh, s, k, prm, F, torch, vfd, rtol=1e-10):
    """Plain CG against the two-level preconditioned CG (leaf blocks + the
    leaf-constant coarse space) on the benchmark operator, one right-hand side."""
    out = {}
    op = vfd.vfd_assemble(mesh, s, k, prm["s_bar"])
    for name in ("cg", "pcg"):
        if name == "pcg":
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            vfd.vfd_precondition(op)
            torch.cuda.synchronize()
            out["setup_s"] = round(time.perf_counter() - t0, 4)
        U = torch.zeros_like(F)
        vfd.vfd_solve(op, F, U, rtol=rtol, max_it=100000)        # warm (graph capture)
        U.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, it, rel = vfd.vfd_solve(op, F, U, rtol=rtol, max_it=100000)
        torch.cuda.synchronize()
        out[name] = {"iters": int(it[0]), "solve_ms": round(1000 * (time.perf_counter() - t0), 3),
                     "relres": float(rel[0])}
        if name == "cg":
            U_cg = U.clone()
        else:
            out["solution_rel_diff"] = (torch.linalg.norm(U - U_cg) / torch.linalg.norm(U_cg)).item()
    out["rtol"] = rtol
    return out


def recompress_leg(m, s, k, prm, F, torch, vfd, tol=1e-6, rtol=1e-10):
    """The benchmark operator with the algebraic recompression of its far field
    (recompress_tol = tol): per-level ranks, assembly and FP64 apply time, FP64
    CG, and the matvec gap to the interpolation operator it was cut from
    (every row, seeded x) -- next to the same figures without recompression."""
    def mk(t):
        return vfd.vfd_mesh(m.d, m.coords, m.cells, m.cell_is_interior, leaf_m=prm["leaf"], cheb_p=prm["p"],
                            lam=prm["lam"], rho_lambda=prm["lam"], tail_mode=prm["tail"], tail_R=prm["R"],
                            recompress_tol=t)

    stream = torch.cuda.current_stream()
    out = {"tol": tol}
    g = torch.Generator(device="cuda").manual_seed(12)
    X = torch.randn(mk(0.0).n_dof, dtype=torch.float64, device="cuda", generator=g)
    Ys = {}
    for name, t in (("interpolation", 0.0), ("recompressed", tol)):
        mesh = mk(t)
        for _ in range(2):
            op = vfd.vfd_assemble(mesh, s, k, prm["s_bar"], flags=vfd.VFD_ASSEMBLE_TIMED)
        ph = vfd.vfd_op_timings(op)
        Y = torch.empty_like(X)
        for _ in range(5):
            vfd.vfd_apply(op, X, Y)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(stream)
        for _ in range(50):
            vfd.vfd_apply(op, X, Y)
        ev[1].record(stream)
        torch.cuda.synchronize()
        apply_us = ev[0].elapsed_time(ev[1]) * 1000 / 50
        Ys[name] = Y.clone()
        U = torch.zeros_like(F)
        vfd.vfd_solve(op, F, U, rtol=rtol, max_it=100000)   # warm-up (graph capture)
        U.zero_()
        torch.cuda.synchronize()
        ev[0].record(stream)
        st, it, rel = vfd.vfd_solve(op, F, U, rtol=rtol, max_it=100000)
        ev[1].record(stream)
        torch.cuda.synchronize()
        out[name] = {"far_ranks": vfd.vfd_op_far_ranks(op), "assemble_ms": ph["total"],
                     "coupling_phase_ms": ph["coupling"], "apply_us": apply_us, "cg_iters": int(it[0]),
                     "cg_ms": ev[0].elapsed_time(ev[1])}
        out[name]["step_ms"] = out[name]["assemble_ms"] + out[name]["cg_ms"]
        del op
    out["matvec_rel_gap"] = (torch.linalg.norm(Ys["recompressed"] - Ys["interpolation"]) /
                             torch.linalg.norm(Ys["interpolation"])).item()
    return out


def recompress_mixed_leg(m, s, k, prm, torch, vfd, tols=(0.0, 1e-10, 1e-8), nrhs=64, rtol=1e-8):
    """The 64-RHS BF16 preconditioned mixed-precision solve on the benchmark
    disk when the FP64 operator of its reliable updates carries a recompressed
    far field (recompress_tol = each of tols; 0 = the interpolation operator):
    per-level ranks, the FP64 64-column apply, the solve time and iterations,
    the matvec gap of the FP64 operator and the solution gap, both to the
    interpolation operator's."""
    def mk(t):
        return vfd.vfd_mesh(m.d, m.coords, m.cells, m.cell_is_interior, leaf_m=prm["leaf"], cheb_p=prm["p"],
                            lam=prm["lam"], rho_lambda=prm["lam"], tail_mode=prm["tail"], tail_R=prm["R"],
                            inner_p=prm.get("inner_p", 0), recompress_tol=t)

    stream = torch.cuda.current_stream()
    g = torch.Generator(device="cuda").manual_seed(13)
    out = {"nrhs": nrhs, "rtol": rtol, "precision": "bf16 inner, FP64 residuals", "preconditioner": "two-level"}
    ref = {}
    for t in tols:
        try:
            mesh = mk(t)
            if "F" not in ref:
                ref["F"] = torch.randn(nrhs, mesh.n_dof, dtype=torch.float64, device="cuda", generator=g)
            F = ref["F"]
            op64 = vfd.vfd_assemble(mesh, s, k, prm["s_bar"])
            Y = torch.empty_like(F)
            for _ in range(2):
                vfd.vfd_apply(op64, F, Y)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ev[0].record(stream)
            vfd.vfd_apply(op64, F, Y)
            ev[1].record(stream)
            torch.cuda.synchronize()
            apply_ms = ev[0].elapsed_time(ev[1])
            del op64
            op = vfd.vfd_assemble(mesh, s, k, prm["s_bar"], precision=vfd.VFD_BF16)
            vfd.vfd_precondition(op)
            U = torch.zeros_like(F)
            vfd.vfd_solve(op, F, U, rtol=rtol, max_it=20000)   # warm-up (graph capture)
            U.zero_()
            torch.cuda.synchronize()
            ev[0].record(stream)
            st, it, rel = vfd.vfd_solve(op, F, U, rtol=rtol, max_it=20000)
            ev[1].record(stream)
            torch.cuda.synchronize()
            row = {"far_ranks": vfd.vfd_op_far_ranks(op), "fp64_apply_64_ms": apply_ms,
                   "solve_ms": ev[0].elapsed_time(ev[1]), "inner_iters": int(it.max()), "status": int(st),
                   "relres_max": float(rel.max())}
            if t == 0.0:
                ref["Y"], ref["U"] = Y.clone(), U.clone()
            else:
                row["matvec_rel_gap"] = (torch.linalg.norm(Y - ref["Y"]) / torch.linalg.norm(ref["Y"])).item()
                row["solution_rel_gap"] = (torch.linalg.norm(U - ref["U"], dim=1) /
                                           torch.linalg.norm(ref["U"], dim=1)).max().item()
            out["interpolation" if t == 0.0 else f"recompressed_{t:g}"] = row
            del op
        except Exception as exc:   # a failing variant is reported, the other legs still run
            out[f"tol_{t:g}"] = {"error": str(exc)}
    return out


def apply_mode(args, mesh, s, k, prm, prec, torch, vfd):
    """Bounded runs for profilers: one assembly, then --warmup + --steps applies
    (--parts, --nrhs columns; low precision with nrhs % 64 == 0 takes the
    batched tensor-core path), or with --mode solve one solve of --nrhs seeded
    N(0,1) columns to --rtol."""
    op = vfd.vfd_assemble(mesh, s, k, prm["s_bar"], precision=prec)
    g = torch.Generator(device="cuda").manual_seed(11)
    shape = (mesh.n_dof,) if args.nrhs == 1 else (args.nrhs, mesh.n_dof)
    X = torch.randn(*shape, dtype=torch.float64, device="cuda", generator=g)
    Y = torch.zeros_like(X)
    if args.mode == "solve":
        if args.precondition:
            vfd.vfd_precondition(op, args.precondition)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        st, it, rel = vfd.vfd_solve(op, X, Y, rtol=args.rtol, max_it=200000)
        e1.record()
        torch.cuda.synchronize()
        print(json.dumps({"mode": "solve", "precision": args.precision, "nrhs": args.nrhs, "status": int(st),
                          "precondition": args.precondition,
                          "iters": int(it[0]), "relres_max": float(rel.max()),
                          "ms": e0.elapsed_time(e1)}), flush=True)
        return
    run = lambda: vfd.vfd_apply_parts(op, args.parts, X, Y)   # noqa: E731
    if args.near_config >= 0:
        batch = vfd.vfd_batch_create([op])
        vfd.vfd_batch_set_config(batch, args.near_config)
        run = lambda: vfd.vfd_batch_apply(batch, [X], [Y])   # noqa: E731
    for _ in range(args.warmup):
        run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        run()
    e1.record()
    torch.cuda.synchronize()
    print(json.dumps({"mode": "apply", "parts": args.parts, "precision": args.precision, "nrhs": args.nrhs,
                      "near_config": args.near_config,
                      "us_per_apply": 1000 * e0.elapsed_time(e1) / args.steps}), flush=True)


def _profile_value(kernel, workload, precision, key):
    """A figure from the committed ncu summary of a kernel (else null)."""
    p = os.path.join(ROOT, "profiles", f"{kernel}_{workload}_{precision}.json")
    try:
        return json.load(open(p)).get(key)
    except Exception:
        return None


def _traffic_from_profile(workload, precision):
    """DRAM bytes per launch of the roofline kernel from the committed ncu
    summary, if one exists for this workload and precision (else null)."""
    p = os.path.join(ROOT, "profiles", f"k_near_csr_{workload}_{precision}.json")
    try:
        return json.load(open(p)).get("dram_bytes_per_launch")
    except Exception:
        return None


if __name__ == "__main__":
    main()
