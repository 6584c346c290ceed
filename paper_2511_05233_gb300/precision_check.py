"""Distance of the mixed-precision Newton-Krylov path from the FP64 path on one discharge.

The mixed path runs the GMRES matvecs (FP32 Jacobian-vector products), the Krylov basis and the
cell-block-Jacobi preconditioner in FP32, inside an FP64 Newton iteration whose residual,
convergence test, time-step control and ledger stay FP64.  This tool runs the same galvanostatic
discharge (naive controller, Sec. 2.8 / Fig. 4) through an FP64 context and then through a mixed
context on the same structure and initial state (one context at a time, so that both fit in HBM at
large grids) and reports, per output, the largest relative difference of the mixed path from the
FP64 path: the cell-voltage curve U_cell(t) (Eq. A1), the accepted step sizes, the final state by
kind of unknown (concentrations, solid fractions, potentials) and the conservation ledger.

    python -m paper_2511_05233_gb300.precision_check --n 192 --porosity 0.7 --corr-len 8 --f-C 1.0 --steps 6
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np


def run(n, porosity, corr_len, f_C, steps, order, seed, h, dt0):
    import torch

    from . import dgls, inputs

    phase = None
    for s in range(seed, seed + 50):
        ph = inputs.make_structure(n, porosity, corr_len, s)
        if np.any(ph[:, :, 0] == inputs.STRUCT):
            phase = ph
            break
    out = {}
    for name, prec in (("fp64", dgls.FP64), ("mixed", dgls.MIXED)):
        prm = dgls.default_params(dgls.TRADEOFF, order, f_C=f_C, eps_struct=1.0 - porosity, precision=prec)
        ctx = dgls.Context(phase, h, prm)
        z = ctx.new_state()
        ctx.equilibrium_state(z)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = ctx.discharge(z, controller=dgls.NAIVE, dt0=dt0, max_steps=steps)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        lay = list(zip(ctx.offsets, ctx.lengths))
        nl = 6
        kinds = {"conc": range(0, nl), "eps": range(nl, ctx.n_fields - 2),
                 "pot": range(ctx.n_fields - 2, ctx.n_fields)}
        zh = z.cpu().numpy()
        out[name] = {"curve": res, "state": {k: np.concatenate([zh[lay[f][0]:lay[f][0] + lay[f][1]] for f in fs])
                                             for k, fs in kinds.items()},
                     "ledger": np.asarray(ctx.ledger(z)), "wall_s": wall, "n_dof": ctx.n_dof,
                     "workspace_bytes": ctx.workspace_bytes()}
        ctx.close()
        del z
        torch.cuda.empty_cache()
    a, b = out["fp64"], out["mixed"]
    ca, cb = a["curve"], b["curve"]
    m = min(len(ca["t"]), len(cb["t"]))

    def rel(x, y):
        x, y = np.asarray(x, dtype=np.float64), np.asarray(y, dtype=np.float64)
        scale = np.abs(x).max() if x.size else 0.0
        return float(np.abs(y - x).max() / scale) if scale > 0 else 0.0

    return {
        "workload": f"{n}^3 voxel grid, DG{order}, Tradeoff Chemistry, Gaussian random-field structure porosity "
                    f"{porosity}, correlation length {corr_len} voxels, {f_C}C, naive controller from dt={dt0} s, "
                    f"{steps} accepted steps from the Tab. 6 equilibrium state",
        "n_dof": a["n_dof"],
        "steps_fp64": len(ca["t"]), "steps_mixed": len(cb["t"]),
        "same_step_sequence": bool(len(ca["dt"]) == len(cb["dt"]) and np.array_equal(ca["dt"], cb["dt"])),
        "status": {"fp64": ca["status"], "mixed": cb["status"]},
        "max_rel_diff": {
            "U_cell": rel(ca["U_cell"][:m], cb["U_cell"][:m]),
            "t": rel(ca["t"][:m], cb["t"][:m]),
            **{f"state_{k}": rel(a["state"][k], b["state"][k]) for k in a["state"]},
            "ledger": rel(a["ledger"], b["ledger"]),
        },
        "newton_its": {"fp64": ca["newton_its"].tolist(), "mixed": cb["newton_its"].tolist()},
        "gmres_its": {"fp64": ca["gmres_its"].tolist(), "mixed": cb["gmres_its"].tolist()},
        "wall_s": {"fp64": a["wall_s"], "mixed": b["wall_s"]},
        "speedup": a["wall_s"] / b["wall_s"] if b["wall_s"] > 0 else None,
        "workspace_gb": {"fp64": a["workspace_bytes"] / 1e9, "mixed": b["workspace_bytes"] / 1e9},
        "U_cell_fp64": ca["U_cell"].tolist(),
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=192)
    ap.add_argument("--porosity", type=float, default=0.7)
    ap.add_argument("--corr-len", type=float, default=8.0)
    ap.add_argument("--f-C", type=float, default=1.0)
    ap.add_argument("--steps", type=int, default=6)
    ap.add_argument("--order", type=int, default=1)
    ap.add_argument("--seed", type=int, default=5)
    ap.add_argument("--h", type=float, default=1e-6)
    ap.add_argument("--dt0", type=float, default=1e-3)
    a = ap.parse_args()
    print(json.dumps(run(a.n, a.porosity, a.corr_len, a.f_C, a.steps, a.order, a.seed, a.h, a.dt0)), flush=True)


if __name__ == "__main__":
    main()
