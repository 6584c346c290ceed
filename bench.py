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
    # the default batch and stream are smaller than the full-size runs (64 instances; 24 requests of
    # 3 steps, sides 32-128) so that the whole bench ends within minutes
    ap.add_argument("--batch", type=int, default=32, help="instances of the batched workload (0: skip)")
    ap.add_argument("--serve", type=int, default=12, help="requests of the serving workload (0: skip)")
    ap.add_argument("--serve-steps", type=int, default=2)
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--serve-rate", type=float, default=2.0, help="Poisson arrivals per second")
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


# kernels behind the profiled "jvp" category of each precision (the Krylov-loop products)
JVP_KERNELS = {"fp64": "jvp (linearised DG1 apply: k_lin_g, k_lin_nodes_apply, k_lin_nodes_diag, "
                       "k_lin_face_flux, k_lin_line_gather)",
               "mixed": "jvp (fused matrix-free FP32 DG1 product: k_jvp1_batched, one-job table)"}
# DRAM bytes per unknown of one fused FP32 product: ncu dram__bytes_read.sum + dram__bytes_write.sum of
# one launch at this workload's size (128^3, 139,463,920 unknowns; 1.13 GB + 537.0 MB, a 1-pass
# capture) / unknowns; None when the kernel has changed since the counters were taken
FUSED_F32_DRAM_BYTES_PER_DOF = 11.95


def kernel_rates(prof, N, n_pot, hbm, precision):
    """Residual and Jacobian-vector product rates from the per-category CUDA-event times of the
    timed steps, each against HBM with the algorithmic bytes of one evaluation: the residual reads
    z and z^n and writes R (24 B per time-dependent unknown, 16 B per potential unknown, which has
    no z^n term); the product reads z and v and writes J v (24 B per unknown in FP64, 12 B in FP32)."""
    out = {}
    for cat in ("residual", "jvp"):
        ms, calls = prof[cat]
        if not calls:
            continue
        avg = ms / calls
        if cat == "residual":
            bytes_ = 24.0 * N - 8.0 * n_pot
        else:
            bytes_ = (24.0 if precision == "fp64" else 12.0) * N
        out[cat] = {"avg_ms": avg, "calls": calls, "gdof_s": N / (avg / 1e3) / 1e9, "bytes_per_dof": bytes_ / N,
                    "hbm_gbs": bytes_ / (avg / 1e3) / 1e9, "hbm_frac": bytes_ / (avg / 1e3) / 1e9 / hbm}
    return out


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


_ORACLE_CASES = {}


def _oracle_worker(args):
    """One host process of the CPU baseline: residual + complex-step JVP evaluations of the oracle on
    its own crop of the workload structure, repeated until budget_s has passed.  A top-level
    function so that a spawn pool can run it."""
    a_n, a_order, a_chem, m, k0, budget_s = args
    from oracle import newton

    key = (a_n, a_order, a_chem, m, k0)
    if key not in _ORACLE_CASES:    # set up once per process (the pool's processes serve every step)
        from oracle import chemistry as ch, init, lis
        from paper_2511_05233_gb300 import inputs

        phase = inputs.make_structure(a_n, WORKLOAD["porosity"], WORKLOAD["corr_len"], WORKLOAD["structure_seed"])
        crop = inputs.clean_connectivity(phase[k0:k0 + m, :m, :m].copy())
        if not np.any(crop[:, :, 0] == inputs.STRUCT):
            crop[:, :, 0] = inputs.STRUCT
        crop[:, :, -max(2, m // 8):] = inputs.SEP
        chem = ch.tradeoff() if a_chem == "tradeoff" else ch.reduced3()
        model = lis.Model(chem, order=a_order, f_C=WORKLOAD["f_C"], eps_struct=1 - WORKLOAD["porosity"])
        grid = lis.Grid(crop, WORKLOAD["h"])
        z0 = init.uniform_state(model, grid, init.equilibrium_fields(model))
        z = init.perturb(model, grid, z0, inputs.uniform_noise(z0.size, WORKLOAD["noise_seed"]))
        _ORACLE_CASES[key] = (model, grid, z0, z, inputs.normal_noise(z.size, 5))
    model, grid, z0, z, v = _ORACLE_CASES[key]
    from oracle import lis
    n_res = n_jvp = 0
    t_res = t_jvp = 0.0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < budget_s or n_res == 0:
        t1 = time.perf_counter()
        lis.residual(model, grid, z, z0, WORKLOAD["dt"], WORKLOAD["dt"])
        t2 = time.perf_counter()
        newton.jvp(model, grid, z, z0, WORKLOAD["dt"], WORKLOAD["dt"], v)
        t3 = time.perf_counter()
        n_res += 1
        n_jvp += 1
        t_res += t2 - t1
        t_jvp += t3 - t2
    return dict(dof=int(z.size), n_res=n_res, n_jvp=n_jvp, t_res=t_res, t_jvp=t_jvp, wall=time.perf_counter() - t0)


def oracle_pool(procs=None):
    """A spawn process pool with one process per host core for the CPU oracle (spawn: safe to start
    after CUDA is initialised in this process)."""
    import multiprocessing as mp

    return mp.get_context("spawn").Pool(procs or os.cpu_count() or 1)


def oracle_sample(a, budget_s=15.0, pool=None, m=32):
    """The CPU oracle (numpy, as it stands) timed on the host cores: one process per core, each
    evaluating residuals and complex-step JVPs of the same model on its own m^3 crop of the workload
    structure (crops at different z offsets) for about budget_s seconds.  value = unknowns evaluated
    by all processes / wall time."""
    own = pool is None
    if own:
        pool = oracle_pool()
    procs = pool._processes
    m = min(m, a.n)
    offs = [(i * m) % max(1, a.n - m + 1) for i in range(procs)]
    try:
        t0 = time.perf_counter()
        res = pool.map(_oracle_worker, [(a.n, a.order, a.chem, m, k0, budget_s) for k0 in offs], chunksize=1)
        wall = time.perf_counter() - t0
    finally:
        if own:
            pool.close()
            pool.join()
    evals = sum(r["n_res"] + r["n_jvp"] for r in res)
    units = sum((r["n_res"] + r["n_jvp"]) * r["dof"] for r in res)
    dof = res[0]["dof"]
    one_core = {"residual_gdof_s": float(np.mean([r["dof"] * r["n_res"] / r["t_res"] for r in res]) / 1e9),
                "jvp_gdof_s": float(np.mean([r["dof"] * r["n_jvp"] / r["t_jvp"] for r in res]) / 1e9)}
    return dict(value=units / wall / 1e9, unit="GDoF/s", cores=procs, kind="oracle",
                sample=f"{evals} residual/JVP evaluations of the oracle by {procs} processes, each on its own "
                       f"{m}^3 crop of the {a.n}^3 workload structure ({dof} unknowns), in {wall:.1f} s wall",
                per_core=one_core, host_cpu_count=os.cpu_count()), wall, evals


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
    pool = oracle_pool()
    try:
        for _ in range(a.warmup):        # the first one also sets every process up
            oracle_sample(a, budget_s=1.0, pool=pool)
        vals = []
        t_all = time.perf_counter()
        for _ in range(a.steps):
            cb, el, n = oracle_sample(a, budget_s=5.0, pool=pool)
            vals.append(cb["value"])
        ms = 1e3 * (time.perf_counter() - t_all) / max(a.steps, 1)
    finally:
        pool.close()
        pool.join()
    value = float(np.mean(vals))
    line = {"impl": "reference", "metric": "residual/JVP GDoF/s", "value": value, "unit": "GDoF/s",
            "n_gpus": world, "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(a),
            "cpu_baseline": {"value": value, "unit": "GDoF/s", "cores": cb["cores"], "kind": "oracle",
                             "sample": cb["sample"], "per_core": cb["per_core"]},
            "e2e": {"value": value, "unit": "GDoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def batch_specs(n, seed=11, side=(24, 96)):
    """Instances of the batched workload: cubic sides uniform in side, porosity uniform in 0.4-0.8,
    correlation length uniform in 2-8 voxels, C-rate log-uniform in 0.1-2 per hour, DG0 or DG1 at
    50/50 (seeded)."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        out.append(dict(side=int(rng.integers(side[0], side[1] + 1)), porosity=float(rng.uniform(0.4, 0.8)),
                        corr=float(rng.uniform(2.0, 8.0)), f_C=float(np.exp(rng.uniform(np.log(0.1), np.log(2.0)))),
                        order=int(k % 2), seed=100 + k))
    return out


def run_batch(a, dgls, torch, reps=5):
    """Batched instances: FP32 Jacobian-vector products of all instances as one launch per kind
    against the same products one instance at a time, and one implicit step of every instance run
    concurrently against the same steps one after another (all mixed precision).  Wall clock with the
    device synchronised around each measurement."""
    from paper_2511_05233_gb300 import inputs

    specs = batch_specs(a.batch)
    ctxs, zs, vs, outs = [], [], [], []
    for sp in specs:
        phase = None
        for s_ in range(sp["seed"], sp["seed"] + 50):
            ph = inputs.make_structure(sp["side"], sp["porosity"], sp["corr"], s_)
            if np.any(ph[:, :, 0] == inputs.STRUCT):
                phase = ph
                break
        prm = dgls.default_params(dgls.TRADEOFF, sp["order"], f_C=sp["f_C"], eps_struct=1 - sp["porosity"],
                                  precision=dgls.MIXED)
        ctx = dgls.Context(phase, WORKLOAD["h"], prm, stream=torch.cuda.Stream())
        z = ctx.new_state()
        ctx.equilibrium_state(z)
        noise = torch.from_numpy(inputs.uniform_noise(ctx.n_dof, sp["seed"])).cuda()
        z[: ctx.offsets[6]] *= 1.0 + 0.01 * noise[: ctx.offsets[6]]
        ctxs.append(ctx)
        zs.append(z)
        vs.append((torch.from_numpy(inputs.normal_noise(ctx.n_dof, sp["seed"] + 1)).cuda() * (z.abs() + 1e-3)).float())
        outs.append(torch.empty_like(vs[-1]))
    torch.cuda.synchronize()
    units = sum(c.n_dof for c in ctxs)
    ts, dts = [0.0] * len(ctxs), [WORKLOAD["dt"]] * len(ctxs)
    st = torch.cuda.current_stream()
    batch = dgls.Batch(ctxs, stream=st)
    choice = batch.autotune(zs, ts, dts, vs, outs)

    def wall(fn):
        """Wall-clock ms per call with the device synchronised before and after (launch overheads
        included: batching removes them)."""
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            fn()
        torch.cuda.synchronize()
        return 1e3 * (time.perf_counter() - t0) / reps

    l0 = batch.launch_count()
    ms_b = wall(lambda: batch.jvp(zs, ts, dts, vs, outs))
    launches_b = (batch.launch_count() - l0) / (reps + 1)

    def one_at_a_time():               # each instance's product, waiting for it before the next
        for c, z, v, o in zip(ctxs, zs, vs, outs):
            c.jvp_fused(z, 0.0, WORKLOAD["dt"], v, o)
            c.stream.synchronize()

    def streams():                     # every instance's product on its own stream, then one wait
        for c, z, v, o in zip(ctxs, zs, vs, outs):
            c.jvp_fused(z, 0.0, WORKLOAD["dt"], v, o)
    ms_1 = wall(one_at_a_time)
    ms_s = wall(streams)
    # implicit steps: concurrently (one host thread per instance, each on its context's stream) and
    # one after another, wall-clock (each step synchronises)
    zo = [torch.empty_like(z) for z in zs]
    batch.step(zs, zo, ts, dts)                      # warm-up
    t0 = time.perf_counter()
    sts, infos = batch.step(zs, zo, ts, dts)
    ms_step_b = 1e3 * (time.perf_counter() - t0)
    t0 = time.perf_counter()
    for c, z, o in zip(ctxs, zs, zo):
        c.step(z, o, 0.0, WORKLOAD["dt"], check=False)
    ms_step_1 = 1e3 * (time.perf_counter() - t0)
    res = {"instances": len(ctxs), "n_dof_total": units,
           "sides": [sp["side"] for sp in specs], "orders": [sp["order"] for sp in specs],
           "workload": f"{len(ctxs)} instances, sides uniform 24-96, porosity 0.4-0.8, correlation length 2-8, "
                       f"C-rate log-uniform 0.1-2, DG0/DG1 alternating, mixed precision (FP32 products)",
           "schedule": {"dg1_block_order": ["instance after instance", "round robin"][choice[0]],
                        "dg0_block_size": choice[1]},
           "jvp_batched_ms": ms_b, "jvp_one_at_a_time_ms": ms_1, "jvp_gain": ms_1 / ms_b,
           "jvp_separate_streams_ms": ms_s, "jvp_gain_vs_streams": ms_s / ms_b, "timing": "wall clock, device synchronised",
           "jvp_batched_gdof_s": units / (ms_b / 1e3) / 1e9, "jvp_batched_launches": launches_b,
           "step_concurrent_ms": ms_step_b, "step_sequential_ms": ms_step_1, "step_gain": ms_step_1 / ms_step_b,
           "steps_converged": int(sum(1 for s_, i in zip(sts, infos) if s_ == dgls.OK and i.converged))}
    batch.close()
    for c in ctxs:
        c.close()
    del zs, vs, outs, zo
    torch.cuda.empty_cache()
    return res


def run_serving(a, dgls):
    """The serving workload: a seeded Poisson stream of discharge requests (cubic sides 32-128, DG0 and
    DG1, C-rate log-uniform 0.1-2 per hour), each capped at a few accepted steps of the naive
    controller; served with continuous batching (slots with pooled workspaces, an HBM budget of
    150 GB, mixed precision) against the plain sequential FP64 loop on the same requests.  Structures
    are generated before the clocks start."""
    import copy

    from paper_2511_05233_gb300 import serve

    reqs = serve.make_requests(a.serve, rate_hz=a.serve_rate, seed=7, side_range=(32, 128), n_steps=a.serve_steps)
    for r in reqs:
        serve.request_structure(r)
    served, wall = serve.serve(copy.deepcopy(reqs), slots=a.serve_slots, hbm_budget=150 << 30,
                               precision=dgls.MIXED, keep_state=True)
    seqd, wall_seq = serve.sequential(copy.deepcopy(reqs), precision=dgls.FP64, keep_state=True)
    st_s, st_q = serve.latency_stats(served, wall), serve.latency_stats(seqd, wall_seq)
    return {"requests": len(reqs), "steps_per_request": a.serve_steps, "slots": a.serve_slots,
            "arrival_rate_hz": a.serve_rate, "hbm_budget_gb": 150,
            "sides": [r.side for r in reqs], "orders": [r.order for r in reqs],
            "served_mixed": st_s, "sequential_fp64": st_q,
            "throughput_gain": st_s["sims_per_hr"] / st_q["sims_per_hr"], "p99_gain": st_q["p99_s"] / st_s["p99_s"],
            "max_rel_diff_vs_fp64": serve.max_rel_diff(served, seqd),
            "statuses": sorted({str(r.result.get("status")) for r in served})}


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
    hbm = peaks.get("hbm_gbs", 6800.0)
    hbm_src = "of measured (MEASURED_PEAKS.json hbm_gbs)" if "hbm_gbs" in peaks else "of fallback (6.8 TB/s)"
    n_pot = ctx.lengths[ctx.n_fields - 2] + ctx.lengths[ctx.n_fields - 1]
    kern = kernel_rates(prof, N, n_pot, hbm, a.precision)
    cat = max(("residual", "jvp", "precond_build", "precond_apply", "krylov"), key=lambda k: prof[k][0])
    roof = None
    if cat in kern:
        k = kern[cat]
        roof = {"kernel": {"residual": "residual", "jvp": JVP_KERNELS[a.precision]}[cat], "bound": "hbm",
                "achieved": k["hbm_gbs"], "peak": hbm, "unit": "GB/s", "frac": k["hbm_frac"],
                "traffic": None, "bytes_per_dof": k["bytes_per_dof"], "avg_launch_ms": k["avg_ms"],
                "peak_source": hbm_src}
        if cat == "jvp" and a.order == 1 and a.chem == "tradeoff" and a.precision == "fp64":
            # the FP64 product is bound by the FP64 pipe on this part, far below its HBM bytes
            gfl = LIN_JVP_DG1_FLOP_PER_DOF * N / (k["avg_ms"] / 1e3) / 1e9
            roof["traffic"] = LIN_JVP_DG1_DRAM_BYTES_PER_DOF * N if LIN_JVP_DG1_DRAM_BYTES_PER_DOF else None
            roof["fp64_pipe"] = {"achieved_gflops": gfl, "peak_gflops": FP64_PEAK_GFLOPS,
                                 "frac": gfl / FP64_PEAK_GFLOPS, "flop_per_dof": LIN_JVP_DG1_FLOP_PER_DOF,
                                 "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 FLOP x 2.07 GHz "
                                                "(a DFMA probe measured 1200 GFLOP/s on the same part)"}
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
        k32 = kernel_rates(prof32, N, n_pot, hbm, "mixed")
        roof32 = None
        if "jvp" in k32:
            kj = k32["jvp"]
            roof32 = {"kernel": JVP_KERNELS["mixed"], "bound": "hbm", "achieved": kj["hbm_gbs"], "peak": hbm,
                      "unit": "GB/s", "frac": kj["hbm_frac"], "bytes_per_dof": kj["bytes_per_dof"],
                      "avg_launch_ms": kj["avg_ms"], "peak_source": hbm_src,
                      "traffic": FUSED_F32_DRAM_BYTES_PER_DOF * N if FUSED_F32_DRAM_BYTES_PER_DOF else None}
        mixed = {"value": ev32 * N / (ms32 / 1e3) / 1e9, "unit": "GDoF/s", "ms_per_step": ms32 / a.steps,
                 "converged": bool(inf32.converged), "newton_iterations": inf32.newton_iterations,
                 "gmres_iterations": inf32.gmres_iterations,
                 "max_rel_diff_vs_fp64": errs, "speedup_vs_fp64_step": (elapsed_ms / a.steps) / (ms32 / a.steps),
                 "kernels": k32, "roofline_jvp": roof32,
                 "kernel_breakdown_ms": {k: {"ms": v[0], "calls": v[1]} for k, v in prof32.items()}}
        ctx32.close()
        del z32

    batched = None
    if rank == 0 and (a.batch > 0 or a.serve > 0):   # the workload's own context is done: free its HBM
        ctx.close()
        del zn, z
        torch.cuda.empty_cache()
    if rank == 0 and a.batch > 0:
        try:
            batched = run_batch(a, dgls, torch)
        except Exception as e:  # reported in the line, the main figures stand
            batched = {"error": f"{type(e).__name__}: {e}"}
        torch.cuda.empty_cache()
    serving = None
    if rank == 0 and a.serve > 0:
        try:
            serving = run_serving(a, dgls)
        except Exception as e:
            serving = {"error": f"{type(e).__name__}: {e}"}
        torch.cuda.empty_cache()

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
                "gram_schmidt_second_passes": reorth, "roofline": roof, "kernels": kern,
                "kernel_breakdown_ms": breakdown, "clocks": clk.summary(), "e2e": e2e, "cpu_baseline": cpu,
                "mixed_precision": mixed, "batched": batched, "serving": serving}
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
