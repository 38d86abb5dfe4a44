"""Repeated applications of the operator and the preconditioner, for kernel profiling.

    python -m paper_1212_1397_gb300.profile_ops [--n 256] [--k 80] [--faces DDNNSS]
                                                [--precision mixed|fp64] [--reps 3]

Builds a context with the SKS method (which holds no Krylov basis, so the device footprint
is a few fields) and applies helm6_apply_A and helm6_apply_Pinv `reps` times each to a
seeded random complex field.  A profiler pointed at this command sees the stencil and the
preconditioner's kernels at the chosen size without the rest of a solve.
"""
from __future__ import annotations

import argparse

import helm6_inputs as inputs
from . import build, helm6 as H


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--k", type=float, default=80.0)
    ap.add_argument("--faces", default="DDNNSS")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--reps", type=int, default=3)
    a = ap.parse_args(argv)
    import torch
    build.build()
    prec = H.MIXED if a.precision == "mixed" else H.FP64
    with H.Solver(a.n, a.k, a.faces, precision=prec, method=H.SKS) as s:
        x = torch.from_numpy(inputs.complex_normal(5, s.shape)).cuda()
        for _ in range(a.reps):
            y = s.apply_A(x)
        for _ in range(a.reps):
            z = s.apply_Pinv(x)
        torch.cuda.synchronize()
        print(f"applied A and A_p^-1 {a.reps} times at {s.dims}: max |Ax| {float(y.abs().max()):.4g}, "
              f"max |A_p^-1 x| {float(z.abs().max()):.4g}")


if __name__ == "__main__":
    main()
