"""Write the oracle's full discharge to the 1.9 V cut-off (Sec. 3, cut-off; Fig. 4 naive
controller; Eq. A1 cell voltage) on a small synthetic cell, as the expected values of the GPU
replay test.  Calls only the oracle and the seeded structure generator.

    python tests/golden/make_discharge_golden.py [--side 6] [--f_C 1.0] [--out ...]

The cell: a cube of the given side, Gaussian random-field structure (porosity 0.6, correlation
length 2 voxels, seed 1 -- the first seed whose structure keeps a collector voxel), the single
structure cluster touching the collector kept, DG0, Tradeoff Chemistry of Tab. 3, Tab. 6 initial
state and the 40-step parabolic relaxation of Sec. 2.8, then the naive controller from dt = 1e-3 s
up to 10 s until the first accepted step with U_cell <= 1.9 V.  Every discharge step is solved to a
Newton tolerance of 1e-12 (default) so that the curve is pinned well below the 1e-8 comparison.
"""
import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import chemistry as ch, control, init, lis, newton  # noqa: E402
from paper_2511_05233_gb300 import inputs  # noqa: E402


def structure(side, porosity, corr, seed):
    for s in range(seed, seed + 100):
        ph = inputs.make_structure(side, porosity, corr, s, single_cluster=True)
        if np.any(ph[:, :, 0] == inputs.STRUCT):
            return ph, s
    raise RuntimeError("no structure touching x = 0")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--side", type=int, default=6)
    ap.add_argument("--f_C", type=float, default=1.0)
    ap.add_argument("--porosity", type=float, default=0.6)
    ap.add_argument("--rtol", type=float, default=1e-12, help="Newton tolerance of every implicit step")
    ap.add_argument("--out", default=os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                                  "discharge_dg0_tradeoff_6.json"))
    a = ap.parse_args()
    phase, seed = structure(a.side, a.porosity, 2.0, 1)
    grid = lis.Grid(phase, 1e-6)
    model = lis.Model(ch.tradeoff(), order=0, f_C=a.f_C, eps_struct=1.0 - a.porosity)
    t0 = time.time()
    z0 = init.uniform_state(model, grid, init.equilibrium_fields(model))
    zr = init.relax(model, grid, z0, dt=0.1, t_init=4.0)

    def step(z, t, dt):
        z1, info = newton.implicit_euler_step(model, grid, z, t, dt, rtol=a.rtol)
        return info.converged, z1

    def cutoff(z):
        U = lis.cell_voltage(model, grid, z)
        return U <= 1.9, U

    zf, rec = control.naive(step, cutoff, zr, t0=0.0, dt0=1e-3, dt_min=1e-6, dt_max=10.0)
    out = {"what": "oracle discharge to the 1.9 V cut-off (naive controller), DG0 Tradeoff Chemistry",
           "side": a.side, "porosity": a.porosity, "corr_len": 2.0, "structure_seed": seed, "single_cluster": True,
           "f_C": a.f_C, "h": 1e-6, "relax": {"dt": 0.1, "steps": 40}, "newton_rtol": a.rtol,
           "phase": phase.astype(int).tolist(),
           "status": rec.status, "attempts": rec.attempts, "failures": rec.failures,
           "t": rec.t, "dt": rec.dt, "U_cell": rec.U,
           "z_relaxed": zr.tolist(), "z_final": zf.tolist(), "oracle_seconds": time.time() - t0}
    with open(a.out, "w") as f:
        json.dump(out, f)
    print(a.out, rec.status, len(rec.t), "steps", rec.failures, "failures", f"{time.time() - t0:.0f} s",
          "U_end", rec.U[-1] if rec.U else None)


if __name__ == "__main__":
    main()
