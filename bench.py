"""Throughput of the Li-S DG hot path on GB300: one bench step is one implicit Euler step
(Eq. 50) solved by Newton-GMRES through the C ABI (residuals, JVPs, block-Jacobi
preconditioner, Krylov updates), on the 128^3 DG1 workload with the paper's full species set.

Prints one JSON line.  value = (residual + JVP evaluations) x unknowns / time, in GDoF/s,
whole job, inputs resident in HBM.  --impl reference times the CPU oracle instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(n=128, order=1, chem="tradeoff", porosity=0.5, corr_len=4.0, structure_seed=3, noise_seed=4,
                f_C=0.5, dt=1e-3, t=0.0, h=1e-6)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=WORKLOAD["n"])
    ap.add_argument("--order", type=int, default=WORKLOAD["order"])
    ap.add_argument("--chem", default=WORKLOAD["chem"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--precond", default="add", choices=["cpr", "bj", "add"])
    ap.add_argument("--precond-every", type=int, default=0)
    ap.add_argument("--reorth", type=int, default=2, choices=[0, 1, 2],
                    help="GMRES Gram-Schmidt: 2 one pass (default), 0 second pass when needed, 1 always")
    ap.add_argument("--mg-cycles", type=int, default=1)
    ap.add_argument("--eta-min", type=float, default=None, help="floor of the Eisenstat-Walker forcing term")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    return ap.parse_args()


def make_inputs(a, seed_offset=0):
    from paper_2511_05233_gb300 import inputs

    phase = inputs.make_structure(a.n, WORKLOAD["porosity"], WORKLOAD["corr_len"], WORKLOAD["structure_seed"] + seed_offset)
    return phase


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


# FP64 peak of GB300 derived from its unit counts and clock: 152 SMs x 2 DFMA per clock per SM
# (the nominal 1.25 TFLOP/s / (152 x 2.07 GHz x 2 FLOP)) x 2 FLOP x 2.07 GHz.  A DFMA probe
# (independent FMA chains over 8 x 152 x 256 threads) measured 1200 GFLOP/s on the same part.
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.07
# FP64 operations per unknown of one linearised DG1 Jacobian-vector product of the Tradeoff
# Chemistry (transport-factor tangents, node Jacobians, face fluxes once per face, line gather):
# 2 x DFMA + DADD + DMUL thread instructions of the nine launches of one product counted by ncu
# at 64^3 (17,428,880 unknowns), / unknowns.  DRAM bytes of the same launches per unknown, or
# None when the kernels have changed since the counters were taken.
LIN_JVP_DG1_FLOP_PER_DOF = 90.44
LIN_JVP_DG1_DRAM_BYTES_PER_DOF = 263.8


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[3 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def oracle_sample(a, budget_s=15.0):
    """The CPU oracle (numpy, one core) evaluating residuals and complex-step JVPs of the same
    model on a 24^3 crop of the workload structure, repeated for about budget_s seconds."""
    from oracle import chemistry as ch, init, lis, newton
    from paper_2511_05233_gb300 import inputs

    phase = make_inputs(a)
    m = min(24, a.n)
    crop = inputs.clean_connectivity(phase[:m, :m, :m].copy())
    if not np.any(crop[:, :, 0] == inputs.STRUCT):
        crop[:, :, 0] = inputs.STRUCT
    crop[:, :, -max(2, m // 8):] = inputs.SEP
    chem = ch.tradeoff() if a.chem == "tradeoff" else ch.reduced3()
    model = lis.Model(chem, order=a.order, f_C=WORKLOAD["f_C"], eps_struct=1 - WORKLOAD["porosity"])
    grid = lis.Grid(crop, WORKLOAD["h"])
    z0 = init.uniform_state(model, grid, init.equilibrium_fields(model))
    z = init.perturb(model, grid, z0, inputs.uniform_noise(z0.size, WORKLOAD["noise_seed"]))
    v = inputs.normal_noise(z.size, 5)
    n_eval, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < budget_s:
        lis.residual(model, grid, z, z0, WORKLOAD["dt"], WORKLOAD["dt"])
        newton.jvp(model, grid, z, z0, WORKLOAD["dt"], WORKLOAD["dt"], v)
        n_eval += 2
    el = time.perf_counter() - t0
    return dict(value=n_eval * z.size / el / 1e9, unit="GDoF/s", cores=1, kind="oracle",
                sample=f"{n_eval} residual/JVP evaluations of the oracle on a {m}^3 crop ({z.size} unknowns) "
                       f"in {el:.1f} s, one core"), el, n_eval


def reduce_over_ranks(dist, elapsed_ms, units, device):
    """Whole-job figures of a run over several ranks, each stepping its own replica of the cell
    (weak scaling): the slowest rank's time and the units processed by all ranks.  dist is
    torch.distributed (initialised) or None for a single process."""
    if dist is None:
        return elapsed_ms, units
    import torch

    tt = torch.tensor([float(elapsed_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    uu = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(uu, op=dist.ReduceOp.SUM)
    return float(tt.item()), float(uu.item())


def run_reference(a, rank, world):
    if rank != 0:
        return
    total_el, total_n, dof = 0.0, 0, None
    for _ in range(a.warmup):
        oracle_sample(a, budget_s=2.0)
    vals = []
    t_all = time.perf_counter()
    for _ in range(a.steps):
        cb, el, n = oracle_sample(a, budget_s=10.0)
        vals.append(cb["value"])
        total_el += el
        total_n += n
    ms = 1e3 * (time.perf_counter() - t_all) / max(a.steps, 1)
    value = float(np.mean(vals))
    line = {"impl": "reference", "metric": "residual/JVP GDoF/s", "value": value, "unit": "GDoF/s",
            "n_gpus": world, "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(a),
            "cpu_baseline": {"value": value, "unit": "GDoF/s", "cores": 1, "kind": "oracle", "sample": cb["sample"]},
            "e2e": {"value": value, "unit": "GDoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_dict(a):
    return {"workload": f"{a.n}^3 voxel grid, DG{a.order}, {'Tradeoff Chemistry (6 liquid species, 2 solids, 2 potentials)' if a.chem == 'tradeoff' else 'three-species chemistry'}, "
                        f"Gaussian random-field structure porosity {WORKLOAD['porosity']}, correlation length {WORKLOAD['corr_len']} voxels, "
                        f"one implicit Euler step dt={WORKLOAD['dt']} s at {WORKLOAD['f_C']}C, Newton-GMRES(30) rtol 1e-10",
            "grid": a.n, "order": a.order, "chemistry": a.chem, "precision": a.precision, "preconditioner": a.precond,
            "gram_schmidt": ["cgs+dgks", "cgs2", "cgs"][a.reorth], "mg_cycles": a.mg_cycles,
            **({"eta_min": a.eta_min} if a.eta_min is not None else {}),
            "l2": "inputs larger than L2 (every state vector > 129 MB)"}


def main():
    a = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        run_reference(a, rank, world)
        return
    import torch

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2511_05233_gb300 import dgls

    dgls.lib()
    phase = make_inputs(a, seed_offset=0)
    chem = dgls.TRADEOFF if a.chem == "tradeoff" else dgls.REDUCED3
    prm = dgls.default_params(chem, a.order, f_C=WORKLOAD["f_C"], eps_struct=1 - WORKLOAD["porosity"],
                              precision=dgls.MIXED if a.precision == "mixed" else dgls.FP64,
                              preconditioner={"bj": 0, "cpr": 1, "add": 2}[a.precond],
                              precond_every=a.precond_every, reorth=a.reorth, mg_cycles=a.mg_cycles,
                              **({"eta_min": a.eta_min} if a.eta_min is not None else {}))
    stream = torch.cuda.current_stream()
    ctx = dgls.Context(phase, WORKLOAD["h"], prm, stream)
    N = ctx.n_dof
    from paper_2511_05233_gb300 import inputs

    zn = ctx.new_state()
    ctx.equilibrium_state(zn)
    noise = torch.from_numpy(inputs.uniform_noise(N, WORKLOAD["noise_seed"])).cuda()
    nl = 6 if a.chem == "tradeoff" else 3
    conc = slice(0, ctx.offsets[nl])                    # liquid concentration fields come first
    zn[conc] *= 1.0 + 0.01 * noise[conc]
    del noise
    z = ctx.new_state()
    t, dt = WORKLOAD["t"], WORKLOAD["dt"]

    def step():
        st, info = ctx.step(zn, z, t, dt, check=False)
        if st not in (dgls.OK, dgls.ERR_NOCONV):
            raise dgls.DGError(st, "dg_step")
        return info

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ctx.profile(True)
    l0 = ctx.launch_count()
    r0 = ctx.reorth_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    infos = []
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        e0.record(stream)
        for _ in range(a.steps):
            infos.append(step())
        e1.record(stream)
        torch.cuda.synchronize()
    elapsed_ms = e0.elapsed_time(e1)
    launches = ctx.launch_count() - l0
    reorth = ctx.reorth_count() - r0
    prof = ctx.profile_read()
    ctx.profile(False)
    evals = sum(i.residual_evals + i.jvp_evals for i in infos)
    units = evals * N
    elapsed_ms, units = reduce_over_ranks(dist, elapsed_ms, units, "cuda")
    value = units / (elapsed_ms / 1e3) / 1e9

    # ---- dominant kernel roofline (live CUDA-event timing inside the timed steps).  The FP64
    # linearised DG1 product is FP64-ALU-bound on GB300 (FP64 pipe 83-89 % busy, DRAM below half),
    # so it is set against the FP64 peak; other categories against HBM bandwidth.
    peaks = measured_peaks()
    cat = max(("residual", "jvp", "precond_build", "precond_apply", "krylov"), key=lambda k: prof[k][0])
    ms_tot, calls = prof[cat]
    roof = None
    if calls:
        avg_ms = ms_tot / calls
        if cat == "jvp" and a.order == 1 and a.chem == "tradeoff" and a.precision == "fp64":
            achieved = LIN_JVP_DG1_FLOP_PER_DOF * N / (avg_ms / 1e3) / 1e9
            roof = {"kernel": "jvp (linearised DG1 apply: k_lin_g, k_lin_nodes_apply, k_lin_face_flux, "
                              "k_lin_line_gather)",
                    "bound": "alu", "achieved": achieved, "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
                    "frac": achieved / FP64_PEAK_GFLOPS,
                    "traffic": LIN_JVP_DG1_DRAM_BYTES_PER_DOF * N if LIN_JVP_DG1_DRAM_BYTES_PER_DOF else None,
                    "flop_per_dof": LIN_JVP_DG1_FLOP_PER_DOF, "avg_launch_ms": avg_ms,
                    "peak_source": "derived FP64 peak (152 SMs x 4 FLOP/clk x 2.07 GHz)",
                    "hbm_frac_of_measured": (LIN_JVP_DG1_DRAM_BYTES_PER_DOF * N / (avg_ms / 1e3) / 1e9
                                             / peaks.get("hbm_gbs", 6800.0)) if LIN_JVP_DG1_DRAM_BYTES_PER_DOF else None}
        else:
            bpd = {"residual": 24.0, "jvp": 24.0 if a.precision == "fp64" else 12.0}.get(cat)
            if bpd:
                achieved = bpd * N / (avg_ms / 1e3) / 1e9
                pk = peaks.get("hbm_gbs", 6800.0)
                roof = {"kernel": cat, "bound": "hbm", "achieved": achieved, "peak": pk, "unit": "GB/s",
                        "frac": achieved / pk, "traffic": None, "bytes_per_dof": bpd, "avg_launch_ms": avg_ms,
                        "peak_source": "measured" if "hbm_gbs" in peaks else "fallback"}
    breakdown = {k: {"ms": v[0], "calls": v[1]} for k, v in prof.items()}

    # ---- end to end through the host-buffer C-ABI call
    e2e = None
    if not a.no_e2e:   # every rank, like the device-timed steps; whole-job figures as for value
        zn_h = torch.empty(N, dtype=torch.float64, pin_memory=True)
        zn_h.copy_(zn)
        z_h = torch.empty(N, dtype=torch.float64, pin_memory=True)
        zn_np, z_np = zn_h.numpy(), z_h.numpy()
        ev = 0
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(a.steps):
            st, info = ctx.step_host(zn_np, z_np, t, dt, check=False)
            ev += info.residual_evals + info.jvp_evals
        el_ms, e2e_units = reduce_over_ranks(dist, 1e3 * (time.perf_counter() - t0), ev * N, "cuda")
        e2e = {"value": e2e_units / (el_ms / 1e3) / 1e9, "unit": "GDoF/s",
               "h2d_bytes_per_step": 8 * N * world, "d2h_bytes_per_step": 8 * N * world}

    # ---- the same step with the mixed-precision Krylov loop (FP32 JVP, basis and block Jacobi
    # inside the FP64 Newton iteration), and its distance from the FP64 result
    mixed = None
    if rank == 0 and a.precision == "fp64" and not a.no_mixed:
        z64 = z.clone()
        prm32 = dgls.default_params(chem, a.order, f_C=WORKLOAD["f_C"], eps_struct=1 - WORKLOAD["porosity"],
                                    precision=dgls.MIXED, preconditioner={"bj": 0, "cpr": 1, "add": 2}[a.precond],
                                    precond_every=a.precond_every, reorth=a.reorth, mg_cycles=a.mg_cycles,
                              **({"eta_min": a.eta_min} if a.eta_min is not None else {}))
        ctx32 = dgls.Context(phase, WORKLOAD["h"], prm32, stream)
        z32 = ctx32.new_state()
        for _ in range(max(1, min(a.warmup, 2))):
            ctx32.step(zn, z32, t, dt, check=False)
        torch.cuda.synchronize()
        m0, m1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev32 = 0
        ctx32.profile(True)
        m0.record(stream)
        for _ in range(a.steps):
            st32, inf32 = ctx32.step(zn, z32, t, dt, check=False)
            ev32 += inf32.residual_evals + inf32.jvp_evals
        m1.record(stream)
        torch.cuda.synchronize()
        ms32 = m0.elapsed_time(m1)
        prof32 = ctx32.profile_read()
        ctx32.profile(False)
        errs = {}
        lay = list(zip(ctx.offsets, ctx.lengths))
        kinds = {"conc": range(0, nl), "eps": range(nl, ctx.n_fields - 2), "pot": range(ctx.n_fields - 2, ctx.n_fields)}
        for kname, fields in kinds.items():
            if len(fields) == 0:
                continue
            ref = torch.cat([z64[lay[f][0]:lay[f][0] + lay[f][1]] for f in fields])
            got = torch.cat([z32[lay[f][0]:lay[f][0] + lay[f][1]] for f in fields])
            errs[kname] = float((got - ref).abs().max() / ref.abs().max())
        mixed = {"value": ev32 * N / (ms32 / 1e3) / 1e9, "unit": "GDoF/s", "ms_per_step": ms32 / a.steps,
                 "converged": bool(inf32.converged), "newton_iterations": inf32.newton_iterations,
                 "gmres_iterations": inf32.gmres_iterations,
                 "max_rel_diff_vs_fp64": errs, "speedup_vs_fp64_step": (elapsed_ms / a.steps) / (ms32 / a.steps),
                 "kernel_breakdown_ms": {k: {"ms": v[0], "calls": v[1]} for k, v in prof32.items()}}
        ctx32.close()
        del z32

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        cpu, _, _ = oracle_sample(a, budget_s=15.0)

    if rank == 0:
        line = {"metric": "residual/JVP GDoF/s", "value": value, "unit": "GDoF/s", "n_gpus": world,
                "steps": a.steps, "warmup": a.warmup, "ms_per_step": elapsed_ms / a.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64" if a.precision == "fp64" else "f64+f32",
                "data": "synthetic", "config": config_dict(a), "n_dof": N,
                "newton_iterations": [i.newton_iterations for i in infos],
                "gmres_iterations": [i.gmres_iterations for i in infos],
                "converged": [bool(i.converged) for i in infos],
                "evals_per_step": evals / a.steps, "gpu_launches": launches,
                "gram_schmidt_second_passes": reorth, "roofline": roof,
                "kernel_breakdown_ms": breakdown, "clocks": clk.summary(), "e2e": e2e, "cpu_baseline": cpu,
                "mixed_precision": mixed}
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
