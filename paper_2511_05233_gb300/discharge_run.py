"""A complete galvanostatic discharge on one synthetic structure: Tab. 6 equilibrium state, the
parabolic relaxation of Sec. 2.8 (40 steps of 0.1 s), then the naive controller (Fig. 4) at the
given C-rate down to the 1.9 V cut-off; DG1 with the vertex-based slope limiter after each accepted
step (App. B), unless --no-limiter; a Newton solve whose line search stalls within 1e-7 of its initial
scaled residual counts as converged (--stall-rtol).  Prints one JSON line with the discharge curve (time, cell
voltage U_cell (Eq. A1), specific capacity c_m (App. B)), the step statistics and the wall time;
with --compare, the same discharge in the other precision and the largest relative difference of
the two curves at the common accepted times.

    python -m paper_2511_05233_gb300.discharge_run --n 32 --order 1 --f-C 0.5 --precision fp64
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np


def discharge_in_chunks(ctx, z, controller, t_end, max_steps, limiter, wall_limit=0.0, chunk=25, progress=False,
                        clock=time.perf_counter, log=None):
    """The discharge in chunks of accepted steps, each resumed from the previous chunk's controller state
    (bitwise the same curve as one call), so that a wall-clock limit can end it between chunks.  Stops
    at the cut-off (U_cell <= 1.9 V), at t_end, at max_steps, on a failed status, or once wall_limit
    seconds have passed since the call.  Returns the concatenated curve and step statistics."""
    log = log if log is not None else sys.stderr
    t1 = clock()
    parts, ck = [], None
    while True:
        n_left = max_steps - sum(len(q["t"]) for q in parts)
        if n_left <= 0:
            break
        r = ctx.discharge(z, controller=controller, dt0=1e-3, dt_min=1e-6, dt_max=10.0, cutoff_V=1.9,
                          t_end=t_end, max_steps=min(chunk, n_left), limiter=limiter, resume=ck)
        parts.append(r)
        ck = r["checkpoint"]
        if progress:
            log.write(json.dumps({"chunk": len(parts), "t": ck["t"], "dt": ck["dt"],
                                  "U_cell": float(r["U_cell"][-1]) if len(r["U_cell"]) else None,
                                  "steps": sum(len(q["t"]) for q in parts), "status": r["status"],
                                  "wall_s": clock() - t1}) + "\n")
            log.flush()
        done = r["status"] != "DG_OK" or len(r["t"]) < min(chunk, n_left) or \
            (len(r["U_cell"]) and r["U_cell"][-1] <= 1.9) or (t_end > 0 and ck["t"] >= t_end)
        if done or (wall_limit > 0 and clock() - t1 > wall_limit):
            break
    res = {k: np.concatenate([q[k] for q in parts]) for k in ("t", "dt", "U_cell", "c_m", "newton_its", "gmres_its")}
    res.update(status=parts[-1]["status"], attempts=sum(q["attempts"] for q in parts),
               failures=sum(q["failures"] for q in parts))
    return res


def run(n, order, porosity, corr_len, f_C, precision, seed, max_steps, limiter, species_mg=2, t_end=0.0, h=1e-6,
        stall_rtol=None, single_cluster=True, wall_limit=0.0, chunk=25, progress=False):
    import torch

    from . import dgls, inputs

    phase = None
    for s in range(seed, seed + 50):
        ph = inputs.make_structure(n, porosity, corr_len, s, single_cluster=single_cluster)
        if np.any(ph[:, :, 0] == inputs.STRUCT):
            phase = ph
            break
    prm = dgls.default_params(dgls.TRADEOFF, order, f_C=f_C, eps_struct=1.0 - porosity,
                              precision=dgls.MIXED if precision == "mixed" else dgls.FP64, species_mg=species_mg,
                              **({"newton_stall_rtol": stall_rtol} if stall_rtol is not None else {}))
    ctx = dgls.Context(phase, h, prm)
    z = ctx.new_state()
    ctx.equilibrium_state(z)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx.relax(z, 0.1, 40)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    res = discharge_in_chunks(ctx, z, dgls.NAIVE, t_end, max_steps, limiter, wall_limit=wall_limit, chunk=chunk,
                              progress=progress)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    out = {"n": n, "order": order, "porosity": porosity, "corr_len": corr_len, "f_C": f_C, "precision": precision,
           "limiter": bool(limiter), "species_mg": species_mg, "newton_stall_rtol": prm.newton_stall_rtol,
           "single_cluster": bool(single_cluster),
           "n_dof": ctx.n_dof, "status": res["status"], "steps": int(len(res["t"])), "attempts": res["attempts"],
           "failures": res["failures"], "reached_cutoff": bool(len(res["U_cell"]) and res["U_cell"][-1] <= 1.9),
           "t_end_s": float(res["t"][-1]) if len(res["t"]) else 0.0,
           "capacity_ah_per_kg": float(res["c_m"][-1]) if len(res["c_m"]) else 0.0,
           "newton_total": int(np.sum(res["newton_its"])), "gmres_total": int(np.sum(res["gmres_its"])),
           "U_end": float(res["U_cell"][-1]) if len(res["U_cell"]) else None,
           "dt_max_reached": float(res["dt"].max()) if len(res["dt"]) else 0.0,
           "wall_relax_s": t1 - t0, "wall_discharge_s": t2 - t1, "wall_limit_s": wall_limit,
           "stopped_by_wall_limit": bool(wall_limit > 0 and t2 - t1 > wall_limit and not (len(res["U_cell"]) and res["U_cell"][-1] <= 1.9)),
           "curve": {"t": res["t"].tolist(), "U_cell": res["U_cell"].tolist(), "c_m": res["c_m"].tolist()}}
    ctx.close()
    return out


def curve_diff(a, b):
    """Largest relative difference of U_cell at the accepted times the two runs share."""
    ta, tb = np.asarray(a["curve"]["t"]), np.asarray(b["curve"]["t"])
    m = min(len(ta), len(tb))
    same = bool(m and np.array_equal(ta[:m], tb[:m]))
    ua, ub = np.asarray(a["curve"]["U_cell"][:m]), np.asarray(b["curve"]["U_cell"][:m])
    return {"same_times_for_first_steps": same, "common_steps": int(m),
            "max_rel_diff_U_cell": float(np.abs(ua - ub).max() / np.abs(ua).max()) if m else None}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=32)
    ap.add_argument("--order", type=int, default=1)
    ap.add_argument("--porosity", type=float, default=0.5)
    ap.add_argument("--corr-len", type=float, default=4.0)
    ap.add_argument("--f-C", type=float, default=0.5)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--seed", type=int, default=3)
    ap.add_argument("--max-steps", type=int, default=5000)
    ap.add_argument("--no-limiter", action="store_true",
                    help="DG1 without the vertex-based slope limiter (on by default for DG1, as in App. B)")
    ap.add_argument("--species-mg", type=int, default=2, choices=[0, 1, 2],
                    help="species coarse level of the preconditioner: off, on, on at large dt (default)")
    ap.add_argument("--t-end", type=float, default=0.0, help="stop at this time in s (0: at the cut-off)")
    ap.add_argument("--stall-rtol", type=float, default=1e-7,
                    help="Newton: a stalled line search counts as converged below this fraction of the initial "
                         "scaled residual (1e-7 here, one decade above the rounding level measured on DG1 "
                         "mid-discharge states; the library default is 1e-8)")
    ap.add_argument("--no-curve", action="store_true", help="print the summary without the curve arrays")
    ap.add_argument("--multi-cluster", action="store_true",
                    help="keep every structure cluster touching the current collector (default: only the largest, "
                         "so that no collector voxel is isolated)")
    ap.add_argument("--wall-limit", type=float, default=0.0, help="stop the discharge after this many seconds (0: none)")
    ap.add_argument("--progress", action="store_true", help="one JSON line per chunk of accepted steps on stderr")
    ap.add_argument("--compare", action="store_true", help="also run the other precision and compare")
    a = ap.parse_args()
    lim = a.order == 1 and not a.no_limiter
    r = run(a.n, a.order, a.porosity, a.corr_len, a.f_C, a.precision, a.seed, a.max_steps, lim, a.species_mg, a.t_end,
            stall_rtol=a.stall_rtol, single_cluster=not a.multi_cluster, wall_limit=a.wall_limit,
            progress=a.progress)
    out = {"run": r}
    if a.compare:
        other = "mixed" if a.precision == "fp64" else "fp64"
        r2 = run(a.n, a.order, a.porosity, a.corr_len, a.f_C, other, a.seed, a.max_steps, lim, a.species_mg, a.t_end,
                 stall_rtol=a.stall_rtol, single_cluster=not a.multi_cluster, wall_limit=a.wall_limit,
                 progress=a.progress)
        out["other"] = r2
        out["comparison"] = curve_diff(r, r2)
    if a.no_curve:
        for v in out.values():
            if isinstance(v, dict):
                v.pop("curve", None)
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
