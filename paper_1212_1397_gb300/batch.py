"""Batched solves of many independent problems, and the autotuner that picks their grids
and schedule.

    python -m paper_1212_1397_gb300.batch tune --out tuning.json   # on the GPU
    python -m paper_1212_1397_gb300.batch run [--tuning tuning.json]

The batched workload (helm6_inputs.batch_problems) is 64 problems with n in
{48, 64, 96, 128, 160}, Re k in [5, 60], Im k = 0.01 Re k and random faces (Sommerfeld-like
on z only), each with one Gaussian source, solved by mixed FGMRES(30) to 1e-8 (at most 300
iterations).  Every problem keeps its own context (workspace resident in HBM, its own CUDA
stream created by the library).  With graphs=2 (the default) each context runs device-driven
solves and helm6_solve_batch launches the whole batch as ONE CUDA graph (every problem's
solve a branch, every convergence decision on the device); with graphs=1 the Arnoldi steps
are captured as CUDA graphs and replayed, and helm6_solve_batch runs the problems on a pool
of host threads.

The autotuner measures, per problem size, the thread-block counts of the Gram-Schmidt
reduction and update passes (the grids of the two kernels that read the Krylov basis),
timing 4 same-size problems solved concurrently for one 30-step cycle each; then, on the
real batch, the number of host threads (problems in flight) and the order in which they
are taken (as drawn, or largest first).  The result is a JSON cache that `run` and
bench.py read.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

import helm6_inputs as inputs
from . import helm6 as H

RESTART, TOL, MAXIT = 30, 1e-8, 300


def _torch():
    import torch
    return torch


def default_tuning():
    return {"blocks": {}, "schedule": {"nthreads": 8, "order": "largest_first"}}


def make_batch(problems, tuning=None, graphs=2):
    """One context per problem (own stream, graphs, tuned grids), its right side and a zero
    initial guess.  Returns a list of dicts."""
    torch = _torch()
    tuning = tuning or default_tuning()
    items = []
    for p in problems:
        blk = tuning["blocks"].get(str(p["n"]), {})
        s = H.Solver(p["n"], p["k"], p["faces"], precision=H.MIXED, method=H.FGMRES, max_restart=RESTART,
                     own_stream=True, use_graphs=graphs, dot_blocks=blk.get("dot_blocks", 0),
                     update_blocks=blk.get("update_blocks", 0))
        F = s.rhs_gaussians(inputs.gaussian_sources(p["src_seed"], p["n"], 1, margin_h=4))
        items.append(dict(problem=p, solver=s, F=F, u=s.empty(), N=int(np.prod(s.shape))))
    torch.cuda.synchronize()
    return items


def close_batch(items):
    for it in items:
        it["solver"].close()


def run_batch(items, nthreads, order="largest_first", tol=TOL, maxit=MAXIT):
    """Solve every problem from u = 0; returns (wall seconds, stats per item in item order)."""
    torch = _torch()
    idx = list(range(len(items)))
    if order == "largest_first":
        idx.sort(key=lambda i: -items[i]["N"])
    for it in items:
        it["u"].zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rc, stats = H.solve_batch([items[i]["solver"] for i in idx], [items[i]["F"] for i in idx],
                              [items[i]["u"] for i in idx], tol=tol, restart=RESTART, maxit=maxit,
                              nthreads=nthreads)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    out = [None] * len(items)
    for j, i in enumerate(idx):
        out[i] = stats[j]
    return wall, out


def summary(items, wall, stats):
    per = np.array([st["t_total_ms"] for st in stats])
    return dict(solves=len(stats), wall_s=wall, solves_per_s=len(stats) / wall,
                p50_ms=float(np.percentile(per, 50)), p99_ms=float(np.percentile(per, 99)),
                converged=sum(st["status"] == "OK" for st in stats),
                iters_total=int(sum(st["iters"] for st in stats)),
                unknowns_total=int(sum(it["N"] for it in items)))


def tune(sizes=inputs.BATCH_SIZES, problems=None, log=print):
    torch = _torch()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    cands = [(d, u) for d in (sms // 2, sms, 2 * sms) for u in (sms, 2 * sms, 4 * sms, 8 * sms)]
    res = default_tuning()
    for n in sizes:
        k = 0.31 * (n + 1)  # about 20 points per wavelength
        best = None
        for d, u in cands:
            probs = [dict(n=n, k=complex(k, 0.01 * k), faces="DDNNSS", src_seed=7 + i) for i in range(4)]
            items = make_batch(probs, {"blocks": {str(n): {"dot_blocks": d, "update_blocks": u}}}, graphs=1)
            try:
                run_batch(items, 4, "as_drawn", tol=1e-14, maxit=RESTART)  # captures the graphs
                t = min(run_batch(items, 4, "as_drawn", tol=1e-14, maxit=RESTART)[0] for _ in range(3))
            finally:
                close_batch(items)
            log(f"tune n={n} dot_blocks={d} update_blocks={u}: {t * 1e3:.2f} ms")
            if best is None or t < best[0]:
                best = (t, d, u)
        res["blocks"][str(n)] = {"dot_blocks": best[1], "update_blocks": best[2], "ms_4x30": best[0] * 1e3}
    problems = problems or inputs.batch_problems(0, 64)
    items = make_batch(problems, res)
    try:
        run_batch(items, 8)  # graph capture
        best = None
        for nt in (4, 8, 16, 32):
            for order in ("as_drawn", "largest_first"):
                wall, _ = run_batch(items, nt, order)
                log(f"tune schedule nthreads={nt} order={order}: {wall * 1e3:.1f} ms")
                if best is None or wall < best[0]:
                    best = (wall, nt, order)
    finally:
        close_batch(items)
    res["schedule"] = {"nthreads": best[1], "order": best[2], "batch_ms": best[0] * 1e3}
    return res


def load_tuning(path):
    if path:
        try:
            with open(path) as f:
                return json.load(f)
        except OSError:
            pass
    return default_tuning()


def main(argv=None):
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    t = sub.add_parser("tune")
    t.add_argument("--out", required=True)
    r = sub.add_parser("run")
    r.add_argument("--tuning", default=None)
    r.add_argument("--reps", type=int, default=3)
    a = ap.parse_args(argv)
    if a.cmd == "tune":
        res = tune()
        with open(a.out, "w") as f:
            json.dump(res, f, indent=1)
        print(json.dumps(res))
    else:
        tun = load_tuning(a.tuning)
        items = make_batch(inputs.batch_problems(0, 64), tun)
        try:
            sch = tun["schedule"]
            run_batch(items, sch["nthreads"], sch["order"])
            for _ in range(a.reps):
                wall, stats = run_batch(items, sch["nthreads"], sch["order"])
                print(json.dumps(summary(items, wall, stats)))
        finally:
            close_batch(items)


if __name__ == "__main__":
    main()
