#!/usr/bin/env python
"""Time-to-solution of the sixth-order compact Helmholtz solve on one GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
    python bench.py --ops R            # operator and preconditioner only (kernel profiling)
    python bench.py --oracle-full      # the oracle's complete FP64 GMRES(30) solve, timed once

A step is one complete solve of the large mixed-face problem: n = 256 interior points per
side (256 x 258 x 258 = 17,040,384 complex unknowns), k = 80, Dirichlet x faces, Neumann y
faces, Sommerfeld-like z faces, right side the compact assembly of 8 Gaussian sources with
unit-modulus random phases, solved from u = 0 to ||F - A u|| / ||F|| <= 1e-8 (FP64 true
residual) by FP64 refinement around FP32 FGMRES(30) with BF16-split tensor-core
transforms.  `value` is the device time per solve with F resident in HBM; `e2e` adds the
host->device copy of F and the device->host copy of u (pinned buffers) to every step.
The per-phase times, the roofline of the kernel with the most device time and the launch
count come from a repeat of the timed solves with the library's phase events on.
Beside it: the same solve with an FP32 Krylov basis, with the learned second stage (AUTO),
the plain FP64 GMRES(30) solve, GMRES(20) against the stationary SKS iteration on the
128 x 130 x 130, k = 40 mixed workload, the 64-problem batched workload, and the CPU
oracle's time-to-solution from a bounded sample of its own functions at the full size.

With N > 1 (torchrun) every rank solves its own replica (independent right sides, no
collective on the data path); the timed region is bracketed by barriers and the slowest
rank's time is reported ("replicas": the method itself does not shard here).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import helm6_inputs as inputs  # noqa: E402

WORKLOAD = "mixed_n256_k80"
METRIC = "time to rel-res 1e-8 at 256^3 k=80 (mixed FP32/BF16 + FP64 refinement)"


def metric_for(workload):
    """The metric of the default workload, and the same wording for any other."""
    if workload == WORKLOAD:
        return METRIC
    cfg = inputs.WORKLOADS[workload]
    k = cfg["k"]
    kk = f"{k.real:g}{k.imag:+g}i" if isinstance(k, complex) and k.imag else f"{complex(k).real:g}"
    tol = f"{cfg['tol']:.0e}".replace("e-0", "e-")
    return (f"time to rel-res {tol} at {cfg['n']}^3 k={kk} faces {cfg['faces']} "
            "(mixed FP32/BF16 + FP64 refinement)")
# The oracle's complete FP64 GMRES(30) solve of a workload from u = 0 to its tolerance,
# measured once on the GPU machine's host cores by `bench.py --oracle-full` (seconds, iterations,
# cycles, threads).  The iteration and cycle counts size the bounded sample's projection.
ORACLE_FULL = {
    # GB300 machine, 16 Arm host cores: 587.1 s from u = 0 to 9.81e-9, 182 iterations, 7 cycles
    "mixed_n256_k80": {"seconds": 587.1, "iters": 182, "cycles": 7, "relres": 9.81e-9, "cores": 16},
}

# Library phases and the kernel each one launches (the four transform phases are one kernel).
KERNEL_OF = {
    "stencil": "stencil4_kernel",
    "xform_x_fwd": "xform_tc_kernel",
    "xform_y_fwd": "xform_tc_kernel",
    "ztri": "ztri_lines_kernel<8>",
    "xform_y_inv": "xform_tc_kernel",
    "xform_x_inv": "xform_tc_kernel",
    "gs_dot": "dcgs_dot_kernel<float,{p},{tv}{dch}>",
    "gs_update": "dcgs_update_kernel<float,{p},{tv}{uch}>",
    "resid64": "stencil_kernel<double,1>",
}

# DRAM bytes (ncu dram__bytes_read.sum + dram__bytes_write.sum) per launch and unknown of a
# kernel, from a capture of the kernel as it is now built (a kernel absent here was changed
# since its last capture: traffic null).
# Captured on the 256 x 258 x 258 grid with `bench.py --ops 3` (mixed precision, tensor-core
# transforms): the x/y transform writes partly stay in the 129 MB L2 for the next kernel, so its
# DRAM bytes fall below the 16 B per unknown it reads and writes; the z lines read their input,
# the pivot table twice (once per sweep) and their own forward results back.
NCU_DRAM_BYTES_PER_UNKNOWN = {
    "xform_tc_kernel": 12.736,
    "ztri_lines_kernel<8>": 40.786,
    "stencil4_kernel": 13.844,
}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), "measured"
    except Exception:
        return 6800.0, 1900.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.fh = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.flush()
        self.fh.seek(0)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.fh.read().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        os.unlink(self.fh.name)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_problem(cfg, seed):
    import oracle as O
    prob = O.Problem(cfg["n"], cfg["k"], cfg["faces"])
    return O, prob, inputs.complex_normal(seed, prob.shape)


def oracle_unit_costs(O, prob, x):
    """Seconds of the oracle's own work units at the full size on the host cores: the
    preconditioner's set-up, one application of A_p^-1 and of A, and one modified
    Gram-Schmidt projection as its GMRES does it (a dot product with one basis vector and
    the update of w against it)."""
    t0 = time.perf_counter()
    M = O.Preconditioner(prob)
    t1 = time.perf_counter()
    z = M(x)
    t2 = time.perf_counter()
    w = O.apply_A(prob, z)
    t3 = time.perf_counter()
    from oracle.helm6_oracle import _dot
    hij = _dot(x, w)
    w = w - hij * x
    t4 = time.perf_counter()
    del z, w
    return dict(setup=t1 - t0, precond=t2 - t1, apply_A=t3 - t2, proj=t4 - t3)


def oracle_projection(u, iters, restart):
    """Time-to-solution of the oracle's restarted GMRES(restart) taking `iters` iterations
    (cycles of `restart` columns, the last one shorter), from its unit costs: set-up, the
    initial residual, per iteration one A_p^-1 and one A plus j + 1 projections at column j,
    per cycle the combination V y (one projection per column), A_p^-1 of it and the true
    residual."""
    cycles = max(1, -(-iters // restart))
    lens = [restart] * (cycles - 1) + [iters - restart * (cycles - 1)]
    proj = sum(L * (L + 1) // 2 + L for L in lens)
    s = (u["setup"] + u["apply_A"] + iters * (u["precond"] + u["apply_A"])
         + cycles * (u["precond"] + u["apply_A"]) + proj * u["proj"])
    return 1e3 * s, cycles


def oracle_counts(workload, fallback_iters=None):
    """(iterations, source) of the oracle's complete solve of this workload."""
    full = ORACLE_FULL.get(workload)
    if full:
        return full["iters"], "the oracle's complete solve of this workload (bench.py --oracle-full)"
    if fallback_iters:
        return fallback_iters, "the GPU's FP64 GMRES(30) iteration count of this run (oracle not run in full)"
    return None, None


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


# ---- replicas over ranks (N > 1: one independent problem per rank, no data-path collective) ----

def replica_seeds(rank):
    """Seeds of rank `rank`'s replica: its Gaussian sources and its noise field."""
    return 1000 + rank, 2000 + rank


def sync_all(dist, cuda=True):
    """Device synchronisation, then a barrier over the ranks (when there are several)."""
    if cuda:
        import torch
        torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()


def reduce_max(x, dist):
    """Largest value of x over the ranks (the slowest rank's time)."""
    if dist is None:
        return x
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_reference(args, cfg, rank, world):
    """--impl reference: the CPU oracle timed on the host cores (rank 0 only).  Each step
    times a bounded sample of the oracle's own functions at the full size (set-up, one
    A_p^-1, one A, one Gram-Schmidt projection); the value is the time-to-solution those
    unit costs give for the iterations of the oracle's complete solve."""
    if rank != 0:
        return
    O, prob, x = oracle_problem(cfg, 12345)
    for _ in range(args.warmup):
        oracle_unit_costs(O, prob, x)
    iters, src = oracle_counts(args.workload)
    if iters is None:
        print(json.dumps({"impl": "reference", "unavailable": "no complete oracle solve recorded for "
                          f"{args.workload} (bench.py --oracle-full)"}), flush=True)
        return
    step_s, vals = [], []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        u = oracle_unit_costs(O, prob, x)
        step_s.append(time.perf_counter() - t0)
        vals.append(oracle_projection(u, iters, cfg["restart"])[0])
    v = float(np.mean(vals))
    step_ms = 1e3 * float(np.mean(step_s))
    sample = (f"oracle (numpy/LAPACK FP64) at the full {cfg['n']}^3 size, per step: preconditioner set-up, one "
              f"A_p^-1, one A and one Gram-Schmidt projection ({step_ms / 1e3:.2f} s); value = those unit costs "
              f"x the work of GMRES({cfg['restart']}) in {iters} iterations ({src})")
    line = {"impl": "reference", "metric": metric_for(args.workload), "value": v, "unit": "ms", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "n": cfg["n"], "k": str(cfg["k"]), "faces": cfg["faces"]},
            "cpu_baseline": {"kind": "oracle", "cores": cpu_cores(), "sample": sample, "value": v,
                             "unit": "ms"},
            "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "oracle_full": ORACLE_FULL.get(args.workload)}
    print(json.dumps(line), flush=True)


def run_oracle_full(args, cfg):
    """--oracle-full: the oracle's complete FP64 GMRES solve of the workload from u = 0 to
    its tolerance, on the host cores, timed once (minutes at 256^3)."""
    import oracle as O
    n, k, faces = cfg["n"], cfg["k"], cfg["faces"]
    prob = O.Problem(n, k, faces)
    src = inputs.gaussian_sources(replica_seeds(0)[0], n, cfg.get("nsrc", 8))
    noise = None
    if cfg.get("noise", 0.0) > 0:
        noise = cfg["noise"] * inputs.complex_normal(replica_seeds(0)[1], prob.shape)
    F = O.rhs(prob, O.sources.gaussians(src), noise=noise)
    t0 = time.perf_counter()
    M = O.Preconditioner(prob)
    U, info = O.gmres(lambda v: O.apply_A(prob, v), M, F, tol=cfg["tol"], restart=cfg["restart"],
                      maxit=args.oracle_maxit)
    t1 = time.perf_counter()
    full = {"workload": args.workload, "seconds": t1 - t0, "iters": info["iters"],
            "cycles": max(1, -(-info["iters"] // cfg["restart"])), "relres": info["relres"],
            "converged": info["converged"], "cores": cpu_cores()}
    print(json.dumps({"oracle_full": full}), flush=True)
    del U
    u = oracle_unit_costs(O, prob, inputs.complex_normal(12345, prob.shape))
    proj, _ = oracle_projection(u, info["iters"], cfg["restart"])
    full.update(unit_costs_s=u, projection_from_unit_costs_s=proj / 1e3)
    print(json.dumps({"oracle_full": full}), flush=True)


def run_ops(args, cfg):
    """--ops R: R applications each of the operator and of the preconditioner at the
    workload's size (--ops-precision, --ops-transform), device-timed per application; for
    kernel profiling."""
    import torch
    from paper_1212_1397_gb300 import build
    from paper_1212_1397_gb300 import helm6 as H
    build.build()
    H.load()
    torch.cuda.set_device(0)
    prec = H.FP64 if args.ops_precision == "fp64" else H.MIXED
    with H.Solver(cfg["n"], cfg["k"], cfg["faces"], precision=prec, method=H.SKS,
                  transform=args.ops_transform) as s:
        x = torch.from_numpy(inputs.complex_normal(5, s.shape)).cuda()
        y, z = s.apply_A(x), s.apply_Pinv(x)
        torch.cuda.synchronize()
        out = {}
        s.profile(True)
        for name, fn in (("apply_A", lambda: s.apply_A(x, y)), ("apply_Pinv", lambda: s.apply_Pinv(x, z))):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(args.ops):
                fn()
            e1.record()
            torch.cuda.synchronize()
            out[name + "_ms"] = e0.elapsed_time(e1) / args.ops
        prof = s.profile_read()["phases"]
        s.profile(False)
        # device time per call of each kernel phase (CUDA events around the launches)
        out["phase_us"] = {k: 1e3 * v["ms"] / v["count"] for k, v in prof.items() if v["count"] > 0}
        out.update(workload=args.workload, dims=list(s.dims), reps=args.ops, precision=args.ops_precision,
                   transforms="/".join(s.transforms),
                   max_abs_Ax=float(y.abs().max()), max_abs_Pinv_x=float(z.abs().max()))
    print(json.dumps({"ops": out}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(inputs.WORKLOADS))
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP64 GMRES solve")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-learned", action="store_true", help="skip the mixed + learned-stage solve")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-problem batched workload")
    ap.add_argument("--basis", default="auto", choices=["auto", "f32", "f16"],
                    help="storage of the inner solve's Krylov basis (auto: the library default)")
    ap.add_argument("--no-f32", action="store_true", help="skip the FP32-basis solve")
    ap.add_argument("--no-sks", action="store_true", help="skip the GMRES(20) vs SKS comparison")
    ap.add_argument("--eager", action="store_true",
                    help="host-driven headline solve instead of one graph launch (for ncu, which cannot "
                         "profile kernel nodes of graphs with conditional nodes)")
    ap.add_argument("--ops", type=int, default=0, help="only apply A and A_p^-1 this many times each")
    ap.add_argument("--ops-precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--ops-transform", default="auto", choices=["auto", "dense", "fft"])
    ap.add_argument("--oracle-full", action="store_true", help="only the oracle's complete solve, timed once")
    ap.add_argument("--oracle-maxit", type=int, default=2000)
    args = ap.parse_args()
    cfg = dict(inputs.WORKLOADS[args.workload])
    if args.oracle_full:
        run_oracle_full(args, cfg)
        return
    if args.ops > 0:
        run_ops(args, cfg)
        return

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, cfg, rank, world)
        return

    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)

    from paper_1212_1397_gb300 import build
    from paper_1212_1397_gb300 import helm6 as H
    if rank == 0:
        build.build()
    if dist:
        dist.barrier()
    H.load()

    n, k, faces = cfg["n"], cfg["k"], cfg["faces"]
    restart, tol = cfg["restart"], cfg["tol"]
    stream = torch.cuda.current_stream()
    basis = {"auto": H.BASIS_AUTO, "f32": H.BASIS_F32, "f16": H.BASIS_F16}[args.basis]
    # the headline solve runs as one CUDA graph launch with its convergence decided on the
    # device (use_graphs = 2; results identical to the host-driven path)
    solver = H.Solver(n, k, faces, precision=H.MIXED, method=H.FGMRES, max_restart=restart,
                      stream=stream, basis=basis, use_graphs=0 if args.eager else 2)
    N = solver.shape[0] * solver.shape[1] * solver.shape[2]
    src_seed, noise_seed = replica_seeds(rank)
    src = inputs.gaussian_sources(src_seed, n, cfg.get("nsrc", 8))
    noise = None
    if cfg.get("noise", 0.0) > 0:
        noise = torch.from_numpy(cfg["noise"] * inputs.complex_normal(noise_seed, solver.shape)).cuda()
    F = solver.rhs_gaussians(src, noise=noise)
    u = solver.empty()

    # ---- warm-up ----
    st = None
    for _ in range(args.warmup):
        u.zero_()
        _, st = solver.solve(F, u, tol=tol, restart=restart, maxit=1000)

    # ---- timed region: device-resident F ----
    clocks = ClockSampler(local)
    sync_all(dist)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stats = []
    ev0.record(stream)
    for _ in range(args.steps):
        u.zero_()
        _, st = solver.solve(F, u, tol=tol, restart=restart, maxit=1000)
        stats.append(st)
    ev1.record(stream)
    sync_all(dist)
    clk = clocks.stop()
    ms = reduce_max(ev0.elapsed_time(ev1) / args.steps, dist)

    # ---- e2e: host buffers through the same public API, right after the device-resident
    # solves (the same conditions; the profiled repeat below comes after both) ----
    F_host = F.cpu().pin_memory()
    u_host = torch.empty_like(F_host).pin_memory()
    u_dev = solver.empty()
    F_dev = solver.empty()
    F_dev.copy_(F_host, non_blocking=True)  # one untimed pass over the fresh buffers
    u_dev.zero_()
    solver.solve(F_dev, u_dev, tol=tol, restart=restart, maxit=1000)
    u_host.copy_(u_dev, non_blocking=True)
    sync_all(dist)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        F_dev.copy_(F_host, non_blocking=True)
        u_dev.zero_()
        solver.solve(F_dev, u_dev, tol=tol, restart=restart, maxit=1000)
        u_host.copy_(u_dev, non_blocking=True)
    e1.record(stream)
    sync_all(dist)
    e2e_ms = reduce_max(e0.elapsed_time(e1) / args.steps, dist)

    # ---- the same solves again, host-driven, with the library's per-phase events on (the
    # graph path records no phases; the events stay out of the timed region above) ----
    with H.Solver(n, k, faces, precision=H.MIXED, method=H.FGMRES, max_restart=restart,
                  stream=stream, basis=basis) as psolver:
        psolver.profile(True)
        for _ in range(args.steps):
            u.zero_()
            _, st = psolver.solve(F, u, tol=tol, restart=restart, maxit=1000)
        torch.cuda.synchronize()
        prof = psolver.profile_read()
        psolver.profile(False)

    # ---- mixed + learned second stage (AUTO: one probe cycle, then the better) ----
    learned = None
    if not args.no_learned:
        from paper_1212_1397_gb300 import weights_path
        wfile = weights_path("stage2_kh031.npz")
        if os.path.exists(wfile):
            w = np.load(wfile)
            solver.set_cnn(w["theta"], float(w["out_scale"]), H.CNN_AUTO)
            u.zero_()
            solver.solve(F, u, tol=tol, restart=restart, maxit=1000)  # warm-up
            u.zero_()
            sync_all(dist)
            l0, l1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            l0.record(stream)
            _, stl = solver.solve(F, u, tol=tol, restart=restart, maxit=1000)
            l1.record(stream)
            sync_all(dist)
            learned = {"ms": reduce_max(l0.elapsed_time(l1), dist), "iters": stl["iters"], "outer": stl["outer"],
                       "learned_cycles": stl["cnn_cycles"], "relres": stl["relres"], "status": stl["status"],
                       "mode": "auto", "weights": os.path.basename(wfile)}
            solver.set_cnn(w["theta"], 1.0, H.CNN_OFF)

    def timed_solve(slv, FF, uu, tol_, restart_, maxit_):
        slv.solve(FF, uu.zero_(), tol=tol_, restart=restart_, maxit=maxit_)  # warm-up
        uu.zero_()
        sync_all(dist)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        _, st_ = slv.solve(FF, uu, tol=tol_, restart=restart_, maxit=maxit_)
        b.record(stream)
        sync_all(dist)
        return reduce_max(a.elapsed_time(b), dist), st_

    # ---- the same mixed solve with the Krylov basis in FP32 ----
    f32leg = None
    if not args.no_f32 and solver.basis == H.BASIS_F16:
        with H.Solver(n, k, faces, precision=H.MIXED, method=H.FGMRES, max_restart=restart, stream=stream,
                      basis=H.BASIS_F32, use_graphs=2) as s32:
            u32 = s32.empty()
            ms32, st32 = timed_solve(s32, F, u32, tol, restart, 1000)
            f32leg = {"ms": ms32, "iters": st32["iters"], "outer": st32["outer"], "relres": st32["relres"],
                      "status": st32["status"], "basis": "f32"}
            del u32

    # ---- GMRES(20) against the stationary SKS iteration (Algorithm 1), mixed workload 128^3 ----
    sks_leg = None
    if not args.no_sks:
        c2 = inputs.WORKLOADS["mixed_n128_k40"]
        src2 = inputs.gaussian_sources(src_seed, c2["n"], c2["nsrc"])
        sks_leg = {"workload": "mixed_n128_k40", "n": c2["n"], "k": str(c2["k"]), "faces": c2["faces"],
                   "tol": c2["tol"]}
        for name, meth, maxit in (("gmres20", H.FGMRES, 3000), ("sks", H.SKS, 3000)):
            with H.Solver(c2["n"], c2["k"], c2["faces"], precision=H.MIXED, method=meth, max_restart=c2["restart"],
                          stream=stream, use_graphs=2) as s2:
                eta = torch.from_numpy(c2["noise"] * inputs.complex_normal(noise_seed, s2.shape)).cuda()
                F2 = s2.rhs_gaussians(src2, noise=eta)
                u2 = s2.empty()
                ms2, st2 = timed_solve(s2, F2, u2, c2["tol"], c2["restart"], maxit)
                sks_leg[name] = {"ms": ms2, "iters": st2["iters"], "outer": st2["outer"],
                                 "relres": st2["relres"], "status": st2["status"]}
                del F2, u2, eta

    # ---- plain FP64 GMRES(30) of the same problem ----
    plain = None
    if not args.no_plain:
        u_mixed = u.clone()
        solver64 = H.Solver(n, k, faces, precision=H.FP64, method=H.GMRES, max_restart=restart,
                            stream=stream)
        u64 = solver64.empty()
        solver64.solve(F, u64, tol=tol, restart=restart, maxit=1000)  # warm-up
        u64.zero_()
        sync_all(dist)
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        _, st64 = solver64.solve(F, u64, tol=tol, restart=restart, maxit=1000)
        p1.record(stream)
        sync_all(dist)
        diff = float(torch.linalg.vector_norm(u_mixed - u64) / torch.linalg.vector_norm(u64))
        plain = {"ms": reduce_max(p0.elapsed_time(p1), dist), "iters": st64["iters"],
                 "relres": st64["relres"], "status": st64["status"],
                 "mixed_vs_fp64_rel_l2": diff, "transforms": "/".join(solver64.transforms)}
        plain["ms_per_iter"] = plain["ms"] / max(1, st64["iters"])
        solver64.close()
        # the same solver with the dense m x m transforms, over its first 10 iterations
        solverd = H.Solver(n, k, faces, precision=H.FP64, method=H.GMRES, max_restart=restart,
                           stream=stream, transform="dense")
        u64.zero_()
        solverd.solve(F, u64, tol=tol, restart=restart, maxit=2)  # warm-up
        u64.zero_()
        sync_all(dist)
        p0.record(stream)
        _, std = solverd.solve(F, u64, tol=tol, restart=restart, maxit=10)
        p1.record(stream)
        sync_all(dist)
        plain["dense_ms_per_iter"] = reduce_max(p0.elapsed_time(p1), dist) / max(1, std["iters"])
        solverd.close()
        del u64

    # ---- batched workload: 64 heterogeneous problems, tuned grids and schedule ----
    batch = None
    if not args.no_batch:
        from paper_1212_1397_gb300 import batch as B
        tfile = os.path.join(ROOT, "paper_1212_1397_gb300", "tuning", "batch_gb300.json")
        tun = B.load_tuning(tfile)
        sch = tun["schedule"]
        for graphs, key in ((2, "one_launch"), (1, "host_threads")):
            items = B.make_batch(inputs.batch_problems(0, 64), tun, graphs=graphs)
            try:
                for _ in range(max(1, args.warmup)):
                    B.run_batch(items, sch["nthreads"], sch["order"])  # first run builds the graphs
                runs = [B.run_batch(items, sch["nthreads"], sch["order"]) for _ in range(max(1, args.steps))]
                wall, bstats = sorted(runs, key=lambda r: r[0])[len(runs) // 2]
                res = B.summary(items, wall, bstats)
                res.update({"runs": len(runs), "wall_s_all": [r[0] for r in runs]})
            finally:
                B.close_batch(items)
            if batch is None:
                batch = dict(res)
                batch.update({"metric": "solves/s, 64 problems n in {48..160}, Re k in [5,60], rel-res 1e-8",
                              "mode": "one graph launch for the whole batch, device-driven convergence",
                              "tuning": os.path.basename(tfile) if os.path.exists(tfile) else "defaults"})
            else:
                batch[key] = dict(res, schedule=sch)

    # ---- roofline of the kernel with the most device time (live per-phase events) ----
    hbm, bf16, peak_src = peaks()
    phases = prof["phases"]
    f16 = solver.basis == H.BASIS_F16
    # an FP16 basis on a grid of 8k points: 8 points per thread, the reduction pass compiled
    # for 1 to 6 vectors per warp group (by the step's count), the update 4 vectors at a time
    p8 = f16 and N % 8 == 0
    kernel_of = {ph: name.format(p=8 if p8 else 4 if f16 and N % 4 == 0 else 2, tv="__half" if f16 else "float",
                                 dch=",1..6" if p8 else ",8", uch=",4" if p8 else ",8")
                 for ph, name in KERNEL_OF.items()}
    single = [p for p in phases if p in kernel_of and phases[p]["count"] > 0]
    per_kernel = {}
    for p in single:
        kk_ = per_kernel.setdefault(kernel_of[p], {"ms": 0.0, "bytes": 0.0, "launches": 0, "phases": []})
        kk_["ms"] += phases[p]["ms"]
        kk_["bytes"] += phases[p]["bytes"]
        kk_["launches"] += phases[p]["count"]
        kk_["phases"].append(p)
    dom = max(per_kernel, key=lambda kn: per_kernel[kn]["ms"])
    dk = per_kernel[dom]
    per_launch_ms = dk["ms"] / max(dk["launches"], 1)
    alg_bytes = dk["bytes"] / max(dk["launches"], 1)   # algorithmic bytes per launch (mean)
    achieved = dk["bytes"] / (dk["ms"] * 1e-3) / 1e9
    tpu = NCU_DRAM_BYTES_PER_UNKNOWN.get(dom)
    roof = {"bound": "hbm", "kernel": dom, "phases": dk["phases"], "achieved": achieved, "peak": hbm,
            "unit": "GB/s", "frac": achieved / hbm, "peak_source": peak_src,
            "traffic": tpu * N if tpu else None,
            "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum per launch of this kernel "
                               "as built now, per unknown, times this workload's unknowns") if tpu else None,
            "per_launch_ms": per_launch_ms,
            "alg_bytes_per_launch": alg_bytes,
            "launches_per_step": dk["launches"] / args.steps,
            "kernel_ms_per_step": {kn: v["ms"] / args.steps for kn, v in per_kernel.items()},
            "phase_frac": {p: (phases[p]["bytes"] / (phases[p]["ms"] * 1e-3) / 1e9) / hbm
                           for p in single}}

    # ---- CPU oracle baseline (rank 0, N = 1): bounded sample of its own functions ----
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        iters, isrc = oracle_counts(args.workload, plain["iters"] if plain else None)
        if iters is not None:
            O, oprob, ox = oracle_problem(cfg, 12345)
            reps = 3
            t0 = time.perf_counter()
            us = [oracle_unit_costs(O, oprob, ox) for _ in range(reps)]
            samp_s = time.perf_counter() - t0
            u_med = {key: float(np.median([u_[key] for u_ in us])) for key in us[0]}
            est, cyc = oracle_projection(u_med, iters, restart)
            cpu = {"value": est, "unit": "ms", "cores": cpu_cores(), "kind": "oracle",
                   "sample": (f"oracle (numpy/LAPACK FP64) at the full size, {reps} x (set-up, one A_p^-1, one A, "
                              f"one Gram-Schmidt projection), {samp_s:.1f} s; value = median unit costs x the work "
                              f"of GMRES({restart}) in {iters} iterations, {cyc} cycles ({isrc})"),
                   "unit_costs_s": u_med, "oracle_full": ORACLE_FULL.get(args.workload)}
            del O, oprob, ox

    if rank == 0:
        last = stats[-1]
        line = {
            "metric": metric_for(args.workload), "value": ms, "unit": "ms", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+bf16/f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "n": n, "k": str(k), "faces": faces,
                       "unknowns": N, "restart": restart, "tol": tol,
                       "sources": len(src), "l2": "inputs larger than L2 (17M-unknown vectors)",
                       "basis": {H.BASIS_F16: "f16", H.BASIS_F32: "f32"}.get(solver.basis, "fp64"),
                       "launch": ("host-driven (--eager)" if args.eager else
                                  "one CUDA graph per solve, convergence decided on the device (use_graphs=2)"),
                       "parallelism": "replicas" if world > 1 else "single"},
            "iters": last["iters"], "outer": last["outer"], "relres": last["relres"],
            "status": last["status"],
            "plain_fp64": plain,
            "mixed_learned": learned,
            "mixed_f32_basis": f32leg,
            "gmres_vs_sks": sks_leg,
            "batch64": batch,
            "e2e": {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": 16 * N,
                    "d2h_bytes_per_step": 16 * N},
            "roofline": roof,
            "phases_ms_per_step": {p: phases[p]["ms"] / args.steps for p in phases},
            # kernels the library ran in the timed solves: counted on the host-driven repeat of
            # the same solves (the graph executes the same kernels plus its one-thread
            # control kernels)
            "gpu_launches": prof["launches"],
            "clocks": clk,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    solver.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
