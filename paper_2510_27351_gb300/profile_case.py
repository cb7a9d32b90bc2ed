"""Run a few solves of one configuration, for profilers (ncu) and quick timing.

    python -m paper_2510_27351_gb300.profile_case --n 8388608 --dtype f64 --s 32 --reps 3
    python -m paper_2510_27351_gb300.profile_case --batched 4096 --dtype refine
    python -m paper_2510_27351_gb300.profile_case --adjoint 1024 --n 8192

Inputs are the benchmark distribution (workloads.single / workloads.batched,
seed 0).  Prints per-kernel event times of the last solve and the mean time
per solve.
"""
from __future__ import annotations

import argparse
import os
import sys

import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import paper_2510_27351_gb300 as tdp  # noqa: E402
import workloads as W  # noqa: E402

CODES = {"f64": tdp.F64, "f32": tdp.F32, "refine": tdp.F32_REFINE}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=1 << 23)
    ap.add_argument("--batched", type=int, default=0, help="log-uniform batch of this many systems instead")
    ap.add_argument("--adjoint", type=int, default=0, help="adjoint of this many systems of --n rows instead")
    ap.add_argument("--dtype", choices=sorted(CODES), default="f64")
    ap.add_argument("--s", type=int, default=0)
    ap.add_argument("--iters", type=int, default=1)
    ap.add_argument("--reps", type=int, default=3)
    args = ap.parse_args()
    code = CODES[args.dtype]
    if args.adjoint:
        S = W.uniform_batch(args.adjoint, args.n, seed=0)
    elif args.batched:
        S = W.batched(args.batched, 64, 65536, seed=0)
    else:
        S = W.single(args.n, seed=0)
    dt = torch.float32 if code == tdp.F32 else torch.float64
    a, b, c, d = (torch.from_numpy(getattr(S, k)).to("cuda", dt) for k in "abcd")
    x = torch.empty_like(d)
    it = args.iters if code == tdp.F32_REFINE else 0
    if args.adjoint:
        off = torch.from_numpy(S.offsets).cuda()
        tdp.tdp_solve_batched(off, S.batch, S.n, a, b, c, d, x, 0, code, it)
        g = torch.from_numpy(W.loss_weights(S.n, seed=0)).to("cuda", dt)
        grads = [torch.empty_like(x) for _ in range(4)]
        fn = lambda: tdp.tdp_solve_backward(off, S.batch, S.n, a, b, c, x, g, *grads, args.s, code)
    elif args.batched:
        off = torch.from_numpy(S.offsets).cuda()
        fn = lambda: tdp.tdp_solve_batched(off, S.batch, S.n, a, b, c, d, x, args.s, code, it)
    else:
        fn = lambda: tdp.tdp_solve(a, b, c, d, x, S.n, args.s, code, it)
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    tdp.tdp_profile_enable(True)
    fn()
    prof = tdp.tdp_profile_summary()
    tdp.tdp_profile_enable(False)
    err = float((x.double().cpu() - torch.from_numpy(S.xstar)).abs().max() / abs(S.xstar).max())
    if args.adjoint:  # <g, x> = <lambda, d> (L = g^T A^-1 d)
        lam = grads[3].double()
        err = float(abs(torch.dot(g.double(), x.double()) - torch.dot(lam, d.double())) /
                    abs(torch.dot(g.double(), x.double())))
    what = "duality_rel_err" if args.adjoint else "rel_err_vs_xstar"
    print(f"n={S.n} batch={S.batch} dtype={args.dtype} ms/solve={e0.elapsed_time(e1) / args.reps:.4f} "
          f"{what}={err:.3e}")
    for k, (cnt, ms) in prof.items():
        print(f"  {k:22s} launches={cnt:3d} ms={ms:.4f}")


if __name__ == "__main__":
    main()
