"""Run one kind of library call repeatedly on a seeded workload, for kernel timing and profiling.

    python -m paper_2511_05233_gb300.kernel_driver --n 64 --order 1 --chem tradeoff --op jvp --reps 5

Prints the mean device time per call (CUDA events on the library's stream).  --op jvp_fused times
dg_jvp_fused: FP64 with --precision fp64, the FP32 product of the mixed Krylov loop with mixed.
"""
from __future__ import annotations

import argparse
import json

import numpy as np


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--order", type=int, default=1)
    ap.add_argument("--chem", default="tradeoff")
    ap.add_argument("--porosity", type=float, default=0.5)
    ap.add_argument("--corr", type=float, default=4.0, help="correlation length of the structure, voxels")
    ap.add_argument("--seed", type=int, default=3, help="structure seed")
    ap.add_argument("--noise-seed", type=int, default=4)
    ap.add_argument("--op", default="jvp",
                    help="residual, jvp, jvp_fused or step; several separated by commas run one after the other "
                         "on the same context")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--no-warm", action="store_true", help="no untimed call first (launch lists of exactly reps calls)")
    a = ap.parse_args()
    import torch

    from . import dgls, inputs

    phase = inputs.make_structure(a.n, a.porosity, a.corr, a.seed)
    chem = dgls.TRADEOFF if a.chem == "tradeoff" else dgls.REDUCED3
    prm = dgls.default_params(chem, a.order, eps_struct=1 - a.porosity,
                              precision=dgls.MIXED if a.precision == "mixed" else dgls.FP64)
    ctx = dgls.Context(phase, 1e-6, prm)
    N = ctx.n_dof
    z0 = ctx.new_state()
    ctx.equilibrium_state(z0)
    noise = torch.from_numpy(inputs.uniform_noise(N, a.noise_seed)).cuda()
    nl = 6 if a.chem == "tradeoff" else 3
    z = z0.clone()
    z[: ctx.offsets[nl]] *= 1.0 + 0.01 * noise[: ctx.offsets[nl]]
    v = torch.from_numpy(inputs.normal_noise(N, 5)).cuda() * (z.abs() + 1e-3)
    out = torch.empty_like(z)
    v32, o32 = v.float(), torch.empty(N, dtype=torch.float32, device="cuda")
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    ops = a.op.split(",")
    for op in ops:
        if op not in ("residual", "jvp", "jvp_fused", "step"):
            raise SystemExit(f"unknown op {op}")

    def call(op):
        if op == "residual":
            ctx.residual(z, z0, 1e-3, 1e-3, out)
        elif op == "jvp":
            ctx.jvp(z, 1e-3, 1e-3, v, out)
        elif op == "jvp_fused":
            if a.precision == "mixed":
                ctx.jvp_fused(z, 1e-3, 1e-3, v32, o32)
            else:
                ctx.jvp_fused(z, 1e-3, 1e-3, v, out)
        else:
            ctx.step(z, out, 0.0, 1e-3, check=False)

    for op in ops:
        if not a.no_warm:
            call(op)
        torch.cuda.synchronize()
        e0.record(st)
        for _ in range(a.reps):
            call(op)
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / a.reps
        res = o32 if op == "jvp_fused" and a.precision == "mixed" else out
        print(json.dumps({"op": op, "n": a.n, "order": a.order, "chem": a.chem, "precision": a.precision,
                          "n_dof": N, "ms_per_call": ms, "gdof_per_s": N / (ms / 1e3) / 1e9,
                          "finite": bool(np.isfinite(res.cpu().numpy()).all())}), flush=True)


if __name__ == "__main__":
    main()
