#!/usr/bin/env python
"""Time-to-solution of the sixth-order compact Helmholtz solve on one GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

A step is one complete solve of the large mixed-face problem: n = 256 interior points per
side (256 x 258 x 258 = 17,040,384 complex unknowns), k = 80, Dirichlet x faces, Neumann y
faces, Sommerfeld-like z faces, right side the compact assembly of 8 Gaussian sources with
unit-modulus random phases, solved from u = 0 to ||F - A u|| / ||F|| <= 1e-8 (FP64 true
residual) by FP64 refinement around FP32 FGMRES(30) with BF16-split tensor-core / FP32
transforms.  `value` is the device time per solve with F resident in HBM; `e2e` adds the
host->device copy of F and the device->host copy of u (pinned buffers) to every step.
The per-phase times, the roofline of the dominant kernel and the launch count come from a
repeat of the timed solves with the library's phase events on (the events stay out of the
timed region: recording them serialises the transform's side stream).
The plain FP64 GMRES(30) solve of the same problem is timed beside it, and the CPU oracle
on a bounded sample gives `cpu_baseline`.

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
# FP64 GMRES(30) iterations of this workload to 1e-8 (plain GPU path; the oracle runs the
# same algorithm), used to scale the oracle's per-iteration sample to a time-to-solution.
FP64_ITERS_NOMINAL = 175

# Library phases that are one kernel each (the roofline is reported for the slowest).
KERNEL_OF = {
    "stencil": "stencil_kernel<float,0>",
    "xform_x_fwd": "xform_tc_kernel (x forward)",
    "xform_y_fwd": "xform_tc_kernel (y forward)",
    "ztri": "ztri_apply_kernel<float>",
    "xform_y_inv": "xform_tc_kernel (y inverse)",
    "xform_x_inv": "xform_tc_kernel (x inverse)",
    "gs_dot": "dcgs_dot_kernel<float,{p},{tv}>",
    "gs_update": "dcgs_update_kernel<float,{p},{tv}>",
    "resid64": "stencil_kernel<double,1>",
}

# ncu DRAM bytes (read + write) per launch of a kernel over that launch's algorithmic bytes,
# from the capture at the bench size summarised in profiles/dram_dcgs_dot_f16_n256.md
# (bytes-weighted over launches with 0-4 and 28-30 basis vectors; absent: not captured since
# the kernel last changed).
NCU_TRAFFIC_RATIO = {"dcgs_dot_kernel<float,4,__half>": 1.045}


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


def oracle_sample(cfg, iters_scale):
    """CPU oracle on a bounded sample: preconditioner set-up plus one preconditioned matvec
    (A_p^{-1} then A, the work of one GMRES iteration) at the full size, scaled to a
    time-to-solution by the FP64 GMRES iteration count."""
    import oracle as O
    prob = O.Problem(cfg["n"], cfg["k"], cfg["faces"])
    x = inputs.complex_normal(12345, prob.shape)
    t0 = time.perf_counter()
    M = O.Preconditioner(prob)
    t1 = time.perf_counter()
    y = O.apply_A(prob, M(x))
    t2 = time.perf_counter()
    del y
    per_iter = t2 - t1
    est_ms = 1e3 * ((t1 - t0) + per_iter * iters_scale)
    return est_ms, per_iter


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
    """--impl reference: the CPU oracle timed on the host cores (rank 0 only)."""
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_sample(cfg, FP64_ITERS_NOMINAL)
    vals = []
    for _ in range(args.steps):
        ms, per_iter = oracle_sample(cfg, FP64_ITERS_NOMINAL)
        vals.append(ms)
    v = float(np.mean(vals))
    sample = (f"oracle (numpy/LAPACK FP64) at the full 256^3 size: preconditioner set-up + one "
              f"A(A_p^-1 x) per step ({per_iter:.2f} s), scaled by {FP64_ITERS_NOMINAL} GMRES iterations")
    line = {"impl": "reference", "metric": metric_for(args.workload), "value": v, "unit": "ms", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "n": cfg["n"], "k": str(cfg["k"]), "faces": cfg["faces"]},
            "cpu_baseline": {"kind": "oracle", "cores": cpu_cores(), "sample": sample, "value": v,
                             "unit": "ms"},
            "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


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
    args = ap.parse_args()
    cfg = dict(inputs.WORKLOADS[args.workload])

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
    solver = H.Solver(n, k, faces, precision=H.MIXED, method=H.FGMRES, max_restart=restart,
                      stream=stream, basis=basis)
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

    # ---- the same solves again with the library's per-phase events on (their records
    # serialise the side-stream work, so they stay out of the timed region above) ----
    solver.profile(True)
    for _ in range(args.steps):
        u.zero_()
        _, st = solver.solve(F, u, tol=tol, restart=restart, maxit=1000)
    torch.cuda.synchronize()
    prof = solver.profile_read()
    solver.profile(False)

    # ---- e2e: host buffers through the same public API ----
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
                 "mixed_vs_fp64_rel_l2": diff}
        solver64.close()
        del u64

    # ---- batched workload: 64 heterogeneous problems, tuned grids and schedule ----
    batch = None
    if not args.no_batch:
        from paper_1212_1397_gb300 import batch as B
        tfile = os.path.join(ROOT, "paper_1212_1397_gb300", "tuning", "batch_gb300.json")
        tun = B.load_tuning(tfile)
        items = B.make_batch(inputs.batch_problems(0, 64), tun)
        try:
            sch = tun["schedule"]
            for _ in range(max(1, args.warmup)):
                B.run_batch(items, sch["nthreads"], sch["order"])  # first run captures the graphs
            runs = [B.run_batch(items, sch["nthreads"], sch["order"]) for _ in range(max(1, args.steps))]
            wall, bstats = sorted(runs, key=lambda r: r[0])[len(runs) // 2]
            batch = B.summary(items, wall, bstats)
            batch.update({"metric": "solves/s, 64 problems n in {48..160}, Re k in [5,60], rel-res 1e-8",
                          "runs": len(runs), "wall_s_all": [r[0] for r in runs],
                          "tuning": os.path.basename(tfile) if os.path.exists(tfile) else "defaults",
                          "schedule": sch})
        finally:
            B.close_batch(items)

    # ---- roofline of the dominant kernel (live per-phase events) ----
    hbm, bf16, peak_src = peaks()
    phases = prof["phases"]
    f16 = solver.basis == H.BASIS_F16
    kernel_of = {ph: name.format(p=4 if f16 and N % 4 == 0 else 2, tv="__half" if f16 else "float")
                 for ph, name in KERNEL_OF.items()}
    single = [p for p in phases if p in kernel_of and phases[p]["count"] > 0]
    dom = max(single, key=lambda p: phases[p]["ms"])
    cnt = max(phases[dom]["count"], 1)
    per_launch_ms = phases[dom]["ms"] / cnt
    alg_bytes = phases[dom]["bytes"] / cnt        # algorithmic bytes per launch (mean)
    achieved = phases[dom]["bytes"] / (phases[dom]["ms"] * 1e-3) / 1e9
    roof = {"bound": "hbm", "kernel": kernel_of[dom], "phase": dom, "achieved": achieved, "peak": hbm,
            "unit": "GB/s", "frac": achieved / hbm, "peak_source": peak_src,
            "traffic": (NCU_TRAFFIC_RATIO[kernel_of[dom]] * alg_bytes if kernel_of[dom] in NCU_TRAFFIC_RATIO
                        else None),
            "traffic_source": ("ncu dram bytes at the bench size (profiles/dram_dcgs_dot_f16_n256.md): "
                               "traffic / algorithmic bytes of the captured launches x this run's mean "
                               "algorithmic bytes per launch" if kernel_of[dom] in NCU_TRAFFIC_RATIO else None),
            "per_launch_ms": per_launch_ms,
            "alg_bytes_per_launch": alg_bytes,
            "phase_frac": {p: (phases[p]["bytes"] / (phases[p]["ms"] * 1e-3) / 1e9) / hbm
                           for p in single}}

    # ---- CPU oracle baseline (rank 0, N = 1) ----
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        iters = plain["iters"] if plain else FP64_ITERS_NOMINAL
        est, per_iter = oracle_sample(cfg, iters)
        cpu = {"value": est, "unit": "ms", "cores": cpu_cores(), "kind": "oracle",
               "sample": f"oracle (numpy/LAPACK FP64) preconditioner set-up + one A(A_p^-1 x) at "
                         f"the full size ({per_iter:.2f} s), scaled by the {iters} FP64 GMRES "
                         f"iterations this workload takes"}

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
                       "parallelism": "replicas" if world > 1 else "single"},
            "iters": last["iters"], "outer": last["outer"], "relres": last["relres"],
            "status": last["status"],
            "plain_fp64": plain,
            "mixed_learned": learned,
            "batch64": batch,
            "e2e": {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": 16 * N,
                    "d2h_bytes_per_step": 16 * N},
            "roofline": roof,
            "phases_ms_per_step": {p: phases[p]["ms"] / args.steps for p in phases},
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
