"""Training data, training and evaluation of the learned second preconditioner stage.

    python -m paper_1212_1397_gb300.learned train --out W.npz   # harvest, train on the GPU
    python -m paper_1212_1397_gb300.learned eval --weights W.npz  # iterations with/without

The stage is z = A_p^-1 u + c s N(t/s) with t = u - A A_p^-1 u and s = rms(t) (see
include/helm6.h).  N is trained as a local approximate inverse of the sixth-order
operator on what the direct preconditioner leaves: for residuals r = F - A U_k of the
solver's own iterates U_k,

    r~ = r - A A_p^-1 r   (so that the exact correction e~ solves A e~ = r~),

normalised by the root mean square s of r~ over the whole field (the normalisation the
solver applies) and cropped into 32^3 patches X, the loss is mean |A_h N(X) - X|^2 over
each patch's interior (A_h the interior 27-point operator), and c = 1.  Regressing e~
directly does not generalise: e~ = A^-1 r~ is dominated by near-resonant global modes
that a network of receptive field 9^3 cannot see.  Patches come from the library's
mixed-precision GMRES runs on the mixed-face workloads (Dirichlet x, Neumann y,
Sommerfeld-like z) at about 20 points per wavelength (kh = 0.31).  Everything runs
through the C-ABI: the solver, A and A_p^-1 for the pairs, and the network's forward,
backward and Adam kernels for training; torch only holds the tensors and cuts the crops.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

import helm6_inputs as inputs
from . import helm6 as H
from . import weights_path

PATCH = 32


def _torch():
    import torch
    return torch


def problem_rhs(solver, n, seed, nsrc, noise):
    """Compact right side of nsrc seed-placed Gaussian sources plus `noise` times circular
    complex normal noise (seed + 7919), on the solver's grid."""
    torch = _torch()
    src = inputs.gaussian_sources(seed, n, nsrc)
    nz = None
    if noise > 0:
        nz = torch.from_numpy(noise * inputs.complex_normal(seed + 7919, solver.shape)).cuda()
    return solver.rhs_gaussians(src, noise=nz)


def harvest(n, k, faces, seeds, nsrc, noise, cycles=6, restart=30, log=print):
    """Full-field r~ = r - A A_p^-1 r (complex128 CUDA tensors) for the residuals r of
    `cycles` successive refinement steps of the mixed FGMRES(restart) solver per seed."""
    fields = []
    mixed = H.Solver(n, k, faces, precision=H.MIXED, method=H.FGMRES, max_restart=restart)
    f64 = H.Solver(n, k, faces, precision=H.FP64, method=H.GMRES, max_restart=1)
    try:
        for seed in seeds:
            F = problem_rhs(mixed, n, seed, nsrc, noise)
            U = mixed.empty()
            for _ in range(cycles):
                U, st = mixed.solve(F, U, tol=1e-12, restart=restart, maxit=restart)
                r = F - f64.apply_A(U)
                fields.append(r - f64.apply_A(f64.apply_Pinv(r)))
            log(f"harvest n={n} k={k} seed={seed}: {len(fields)} fields, last relres {st['relres']:.2e}")
    finally:
        mixed.close()
        f64.close()
    return fields


def _rms(t):
    return float(t.abs().pow(2).mean().sqrt())


def make_patches(fields, count, seed):
    """Random 32^3 crops of r~/rms(r~) as a float32 CUDA tensor [count, 32, 32, 32, 2]."""
    torch = _torch()
    srt = [_rms(f) for f in fields]
    X = torch.empty((count, PATCH, PATCH, PATCH, 2), dtype=torch.float32, device="cuda")
    u = inputs.uniform01(seed, 4 * count)
    for i in range(count):
        j = int(u[4 * i] * len(fields)) % len(fields)
        f = fields[j]
        mz, my, mx = f.shape
        z0 = int(u[4 * i + 1] * (mz - PATCH + 1))
        y0 = int(u[4 * i + 2] * (my - PATCH + 1))
        x0 = int(u[4 * i + 3] * (mx - PATCH + 1))
        cr = f[z0:z0 + PATCH, y0:y0 + PATCH, x0:x0 + PATCH] / srt[j]
        X[i] = torch.stack([cr.real, cr.imag], dim=-1).float()
    return X


def init_theta(seed):
    """Weights N(0, 1/(27 c_in)) from the shared normal draws, biases zero."""
    z = inputs.standard_normal(seed, H.CNN_NPARAMS)
    th = np.zeros(H.CNN_NPARAMS)
    o = 0
    for ci, co in zip((2, 16, 16, 16), (16, 16, 16, 2)):
        nw = 27 * ci * co
        th[o:o + nw] = z[o:o + nw] / math.sqrt(27.0 * ci)
        o += nw + co
    return th.astype(np.float32)


def train(X, Xv, k, h, steps=3000, batch=32, lr=2e-3, seed=5, log=print):
    """Adam with cosine decay of the learning rate on the residual-form loss; returns
    (theta, history).  Losses are reported relative to that of N = 0."""
    torch = _torch()
    th0 = init_theta(seed)
    hist = []
    u = inputs.uniform01(seed + 1, steps * batch)
    idx_all = torch.from_numpy((u * X.shape[0]).astype(np.int64) % X.shape[0]).cuda()
    zero = np.zeros(H.CNN_NPARAMS, dtype=np.float32)
    t0 = time.time()
    nv = (Xv.shape[0] // batch) * batch
    with H.Trainer(batch, PATCH, PATCH, PATCH, th0) as tr, \
            H.Trainer(batch, PATCH, PATCH, PATCH, zero) as tr0:
        tr.set_residual_loss(k, h)
        tr0.set_residual_loss(k, h)

        def val_loss(t):
            tot = 0.0
            for i in range(0, nv, batch):
                xb = Xv[i:i + batch].contiguous()
                tot += t.gradient(xb, xb)[0]
            return tot / max(1, nv // batch)
        base = val_loss(tr0)
        v0 = val_loss(tr)
        hist.append(dict(step=0, val=v0 / base))
        log(f"train: val loss relative to N = 0 at init {v0 / base:.4f}")
        for st in range(steps):
            lr_t = 0.5 * lr * (1.0 + math.cos(math.pi * st / steps))
            idx = idx_all[st * batch:(st + 1) * batch]
            xb = X[idx].contiguous()
            want = (st + 1) % 250 == 0 or st == steps - 1
            loss = tr.step(xb, xb, lr_t, want_loss=want)
            if want:
                l0 = tr0.gradient(xb, xb)[0]
                v = val_loss(tr)
                hist.append(dict(step=st + 1, train=loss / l0, val=v / base, lr=lr_t, sec=time.time() - t0))
                log(f"train: step {st + 1} train {loss / l0:.4f} val {v / base:.4f} ({time.time() - t0:.1f} s)")
        theta = tr.params()
    return theta, hist


def evaluate(theta, out_scale, n, k, faces, seeds, nsrc, noise, restart=30, tol=1e-8, log=print,
             modes=("plain", "on", "auto")):
    """Iterations and solve time to `tol` of mixed FGMRES(restart) without the learned
    stage, with it on every cycle, and in AUTO mode, per seed (second of two solves)."""
    torch = _torch()
    res = []
    s = H.Solver(n, k, faces, precision=H.MIXED, method=H.FGMRES, max_restart=restart)
    try:
        for seed in seeds:
            F = problem_rhs(s, n, seed, nsrc, noise)
            row = dict(seed=seed)
            sols = {}
            for mode in modes:
                if mode == "plain":
                    s.set_cnn(theta, out_scale, H.CNN_OFF)
                else:
                    s.set_cnn(theta, out_scale, H.CNN_ON if mode == "on" else H.CNN_AUTO)
                for rep in range(2):
                    u, st = s.solve(F, tol=tol, restart=restart, maxit=3000)
                torch.cuda.synchronize()
                row[mode] = dict(iters=st["iters"], ms=st["t_total_ms"], relres=st["relres"],
                                 status=st["status"], cnn_cycles=st["cnn_cycles"])
                sols[mode] = u
            for mode in modes:
                if mode != "plain":
                    row[mode]["rel_diff_vs_plain"] = float((sols[mode] - sols["plain"]).norm()
                                                           / sols["plain"].norm())
            res.append(row)
            log(json.dumps(row))
    finally:
        s.close()
    return res


def time_steps(steps=50, warmup=5, batch=32, seed=5):
    """Device time of one training step (forward, residual-form loss, backward, Adam) on
    seeded random patches, CUDA events around `steps` steps after `warmup`."""
    torch = _torch()
    x = torch.from_numpy(inputs.complex_normal(seed, (batch, PATCH, PATCH, PATCH)).view(np.float64)
                         .reshape(batch, PATCH, PATCH, PATCH, 2).astype(np.float32)).cuda()
    with H.Trainer(batch, PATCH, PATCH, PATCH, init_theta(seed)) as tr:
        tr.set_residual_loss(40.0, 1.0 / 129)
        for _ in range(warmup):
            tr.step(x, x, 1e-3, want_loss=False)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            tr.step(x, x, 1e-3, want_loss=False)
        e1.record()
        torch.cuda.synchronize()
    return e0.elapsed_time(e1) / max(1, steps)


def time_stage(n=256, reps=5, seed=5):
    """Device time of one application of the direct preconditioner and of the two-stage
    preconditioner (with the stored weights) on a seeded random field of the n^3 mixed-face
    workload (k = 80 n / 256), CUDA events over `reps` applications after two."""
    torch = _torch()
    w = np.load(weights_path("stage2_kh031.npz"))
    out = {}
    with H.Solver(n, 80.0 * n / 256, "DDNNSS", precision=H.MIXED, method=H.FGMRES) as s:
        s.set_cnn(w["theta"], float(w["out_scale"]), H.CNN_ON)
        u = torch.from_numpy(inputs.complex_normal(seed, s.shape)).cuda()
        for name, f in (("apply_Pinv_ms", s.apply_Pinv), ("apply_stage2_ms", s.apply_stage2)):
            for _ in range(2):
                f(u)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                f(u)
            e1.record()
            torch.cuda.synchronize()
            out[name] = e0.elapsed_time(e1) / reps
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    t = sub.add_parser("train")
    t.add_argument("--out", required=True)
    t.add_argument("--patches", type=int, default=20000)
    t.add_argument("--steps", type=int, default=3000)
    t.add_argument("--batch", type=int, default=32)
    t.add_argument("--lr", type=float, default=2e-3)
    t.add_argument("--seeds128", type=int, default=16)
    t.add_argument("--seeds256", type=int, default=3)
    t.add_argument("--eval", action="store_true")
    e = sub.add_parser("eval")
    e.add_argument("--weights", required=True)
    e.add_argument("--seeds", type=int, default=5)
    e.add_argument("--n", type=int, default=192)
    tg = sub.add_parser("time-stage")
    tg.add_argument("--n", type=int, default=256)
    tg.add_argument("--reps", type=int, default=5)
    ts = sub.add_parser("time-step")
    ts.add_argument("--steps", type=int, default=50)
    ts.add_argument("--batch", type=int, default=32)
    a = ap.parse_args(argv)
    if a.cmd == "time-stage":
        print(json.dumps(dict(n=a.n, **time_stage(a.n, a.reps))))
    elif a.cmd == "time-step":
        ms = time_steps(a.steps, batch=a.batch)
        print(json.dumps(dict(ms_per_train_step=ms, batch=a.batch, patch=PATCH, steps=a.steps)))
    elif a.cmd == "train":
        t0 = time.time()
        fields = harvest(128, 40.0, "DDNNSS", range(100, 100 + a.seeds128), nsrc=1, noise=1e-3)
        fields += harvest(256, 80.0, "DDNNSS", range(100, 100 + a.seeds256), nsrc=8, noise=0.0)
        X = make_patches(fields, a.patches, seed=11)
        del fields
        # validation: the learned-stage workload's own problem class, held-out seeds
        vfields = harvest(192, 60.0, "DDNNSS", range(900, 902), nsrc=1, noise=1e-3, cycles=4)
        Xv = make_patches(vfields, 512, seed=12)
        del vfields
        th_harvest = time.time() - t0
        kt, ht = 40.0, 1.0 / 129  # kh = 0.31, the training workloads' resolution
        theta, hist = train(X, Xv, kt, ht, steps=a.steps, batch=a.batch, lr=a.lr)
        c = 1.0
        np.savez(a.out, theta=theta, out_scale=np.float64(c), val=np.array([h["val"] for h in hist]),
                 harvest_sec=np.float64(th_harvest), train_sec=np.float64(hist[-1].get("sec", 0.0)),
                 patches=np.int64(a.patches), steps=np.int64(a.steps), kh=np.float64(kt * ht))
        print(json.dumps(dict(out=a.out, out_scale=c, val_final=hist[-1]["val"], harvest_sec=th_harvest,
                              train_sec=hist[-1].get("sec"))))
        if a.eval:
            evaluate(theta, c, 192, 60.0, "DDNNSS", range(1000, 1002), nsrc=1, noise=1e-3)
    else:
        w = np.load(a.weights)
        evaluate(w["theta"], float(w["out_scale"]), a.n, 60.0 * a.n / 192, "DDNNSS",
                 range(1000, 1000 + a.seeds), nsrc=1, noise=1e-3)


if __name__ == "__main__":
    main()
