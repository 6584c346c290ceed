"""Continuous-batching server for discharge simulations on one GPU.

Requests (structure size, porosity, correlation length, C-rate, DG order) arrive on a seeded
Poisson clock.  Each admitted request gets a slot: a host thread with its own CUDA stream and its
own library context (state, Krylov and preconditioner workspaces stay on the device for the whole
simulation).  A request is admitted when a slot is free and its workspace fits in what is left of
the HBM budget; requests that arrive while others run are admitted as slots and memory free up, so
their kernels overlap on the device.  The library releases the GIL in every call (ctypes), and every
reduction in it has a fixed order, so a simulation's result does not depend on what else runs.

    python -m paper_2511_05233_gb300.serve --requests 16 --slots 4
"""
from __future__ import annotations

import argparse
import hashlib
import heapq
import json
import threading
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Request:
    rid: int
    arrival: float              # seconds after the start of the run
    side: int
    porosity: float
    corr_len: float
    f_C: float
    order: int
    n_steps: int = 6            # accepted implicit steps of the discharge
    seed: int = 0
    start: float = 0.0
    end: float = 0.0
    result: dict = field(default_factory=dict)


def make_requests(n, rate_hz, seed, side_range=(16, 40), n_steps=6, orders=(0, 1)):
    """Seeded Poisson arrivals with mixed sizes, C-rates and orders (the request recipe)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += rng.exponential(1.0 / rate_hz)
        out.append(Request(rid=i, arrival=t, side=int(rng.integers(side_range[0], side_range[1] + 1)),
                           porosity=float(rng.uniform(0.45, 0.65)), corr_len=float(rng.uniform(2.0, 6.0)),
                           f_C=float(np.exp(rng.uniform(np.log(0.1), np.log(2.0)))),
                           order=int(rng.choice(orders)), n_steps=n_steps, seed=1000 + i))
    return out


_STRUCTURES = {}


def request_structure(req):
    """The request's structure: the seeded random field (the first seed that keeps a collector
    voxel), its single structure cluster on the collector kept; generated once per request and kept,
    so that a served request carries its structure as a client would send it."""
    from . import inputs

    key = (req.side, req.porosity, req.corr_len, req.seed)
    if key not in _STRUCTURES:
        for s in range(req.seed, req.seed + 50):
            # one structure cluster on the collector: no isolated collector voxel can passivate
            ph = inputs.make_structure(req.side, req.porosity, req.corr_len, s, single_cluster=True)
            if np.any(ph[:, :, 0] == inputs.STRUCT):
                _STRUCTURES[key] = ph
                break
    return _STRUCTURES[key]


def request_cell(req, precision=None):
    """The request's structure and its library parameters."""
    from . import dgls

    phase = request_structure(req)
    prm = dgls.default_params(dgls.TRADEOFF, req.order, f_C=req.f_C, eps_struct=1 - req.porosity,
                              precision=dgls.FP64 if precision is None else precision)
    return phase, prm


def workspace_estimate(req, precision=None):
    """Device bytes of the request's context, from the library (dg_workspace_estimate), plus its
    state vector."""
    from . import dgls

    phase, prm = request_cell(req, precision)
    return dgls.workspace_estimate(phase, 1e-6, prm) + (1 << 20)


def run_one(req, stream=None, precision=None, keep_state=False, workspace=None):
    """Set up the cell (inside `workspace`, a device uint8 buffer the caller reuses, when given),
    take the Tab. 6 equilibrium state and run the naive controller for req.n_steps accepted steps;
    returns the curve and a checksum of the final state (and the state itself with keep_state).
    precision: dgls.FP64 (default) or dgls.MIXED."""
    import torch

    from . import dgls

    phase, prm = request_cell(req, precision)
    with torch.cuda.stream(stream) if stream is not None else _null():
        ctx = dgls.Context(phase, 1e-6, prm, stream=stream or torch.cuda.current_stream(), workspace=workspace)
        z = ctx.new_state()
        ctx.equilibrium_state(z)
        res = ctx.discharge(z, controller=dgls.NAIVE, dt0=1e-3, max_steps=req.n_steps)
        zh = z.cpu().numpy()
        ctx.close()
    out = {"t": res["t"].tolist(), "dt": res["dt"].tolist(), "U_cell": res["U_cell"].tolist(),
           "status": res["status"], "sha256": hashlib.sha256(zh.tobytes()).hexdigest(),
           "n_dof": int(zh.size)}
    if keep_state:
        out["state"] = zh
    return out


class Admission:
    """Host-side admission of the serving loop.  Every slot keeps a device workspace buffer across
    requests (a context is set up inside it, no allocation per request); the HBM budget covers the
    buffers the slots hold together.  Requests are taken first come, first served: the head of the
    queue goes to a free slot whose buffer already fits it (the smallest such), else to the free slot
    with the largest buffer, grown to the request's workspace if the budget allows the growth.  A
    request whose workspace alone exceeds the budget is rejected when it arrives, so it cannot block
    the queue behind it."""

    def __init__(self, slots, budget, size_of):
        self.buf = [0] * slots          # bytes of each slot's workspace buffer
        self.busy = [False] * slots
        self.budget = budget
        self.size_of = size_of
        self.queue = []
        self.rejected = []

    @property
    def free_slots(self):
        return self.busy.count(False)

    def held(self):
        return sum(self.buf)

    def arrive(self, req):
        need = self.size_of(req)
        if need > self.budget:
            req.result = {"status": f"rejected: workspace {need} B exceeds the HBM budget {self.budget} B"}
            self.rejected.append(req)
            return False
        heapq.heappush(self.queue, (req.arrival, req.rid, req, need))
        return True

    def admit(self):
        """Pop every request that fits now: [(req, need, slot, new buffer bytes)]."""
        out = []
        while self.queue:
            _, _, req, need = self.queue[0]
            free = [k for k in range(len(self.buf)) if not self.busy[k]]
            if not free:
                break
            fit = [k for k in free if self.buf[k] >= need]
            if fit:
                k = min(fit, key=lambda q: self.buf[q])
            else:
                k = max(free, key=lambda q: self.buf[q])
                if self.held() - self.buf[k] + need > self.budget:
                    break
                self.buf[k] = need
            heapq.heappop(self.queue)
            self.busy[k] = True
            out.append((req, need, k, self.buf[k]))
        return out

    def release(self, slot):
        self.busy[slot] = False

    def idle(self):
        return not self.queue


class _null:
    def __enter__(self):
        return None

    def __exit__(self, *a):
        return False


def serve(requests, slots=4, hbm_budget=150 << 30, time_scale=1.0, precision=None, keep_state=False):
    """Run the requests with continuous batching; returns them with start/end times filled."""
    import torch

    t0 = time.perf_counter()
    pending = sorted(requests, key=lambda r: r.arrival)
    lock = threading.Condition()
    adm = Admission(slots, hbm_budget, lambda r: workspace_estimate(r, precision))
    streams = [torch.cuda.Stream() for _ in range(slots)]
    buffers = [None] * slots           # each slot's workspace buffer, kept across requests
    threads = []

    def worker(req, slot, need):
        req.start = time.perf_counter() - t0
        try:
            req.result = run_one(req, streams[slot], precision, keep_state, workspace=buffers[slot])
        except Exception as e:  # a failed request is reported, not fatal to the server
            req.result = {"status": f"error: {e}"}
        req.end = time.perf_counter() - t0
        with lock:
            adm.release(slot)
            lock.notify_all()

    i = 0
    while i < len(pending) or not adm.idle():
        now = time.perf_counter() - t0
        with lock:
            while i < len(pending) and pending[i].arrival * time_scale <= now:
                if not adm.arrive(pending[i]):
                    pending[i].start = pending[i].end = now
                i += 1
            started = adm.admit()
            for req, need, slot, nbytes in started:
                if buffers[slot] is None or buffers[slot].numel() < nbytes:
                    buffers[slot] = None          # the old buffer goes back to torch's cache first
                    buffers[slot] = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
                th = threading.Thread(target=worker, args=(req, slot, need), daemon=True)
                threads.append(th)
                th.start()
            if not started:
                wait = 0.01
                if i < len(pending):
                    wait = max(0.0, min(0.05, pending[i].arrival * time_scale - now))
                lock.wait(timeout=wait if wait > 0 else 0.001)
    for th in threads:
        th.join()
    wall = time.perf_counter() - t0
    # hand the slot buffers back to the device, not only to torch's cache: contexts set up after the
    # server allocate with cudaMalloc
    buffers.clear()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return requests, wall


def sequential(requests, time_scale=1.0, precision=None, keep_state=False):
    """The plain loop: one request at a time on the default stream, each starting at its arrival
    or when the previous one is done."""
    t0 = time.perf_counter()
    for r in sorted(requests, key=lambda q: q.arrival):
        now = time.perf_counter() - t0
        if r.arrival * time_scale > now:
            time.sleep(r.arrival * time_scale - now)
        r.start = time.perf_counter() - t0
        r.result = run_one(r, None, precision, keep_state)
        r.end = time.perf_counter() - t0
    return requests, time.perf_counter() - t0


def max_rel_diff(reqs, refs):
    """Largest relative difference over the requests of the U_cell curve and of the final state
    (scaled by the largest value of that request's quantity) against reference runs."""
    by_id = {r.rid: r for r in refs}
    du = ds = 0.0
    for r in reqs:
        a, b = r.result, by_id[r.rid].result
        if "state" not in a or "state" not in b or len(a["U_cell"]) != len(b["U_cell"]):
            return None
        ua, ub = np.asarray(a["U_cell"]), np.asarray(b["U_cell"])
        du = max(du, float(np.abs(ua - ub).max() / np.abs(ub).max()))
        ds = max(ds, float(np.abs(a["state"] - b["state"]).max() / np.abs(b["state"]).max()))
    return {"U_cell": du, "state": ds}


def latency_stats(reqs, wall):
    lat = np.array([r.end - r.arrival for r in reqs])
    return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "sims_per_hr": len(reqs) / wall * 3600.0, "wall_s": wall}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=16)
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--rate", type=float, default=4.0, help="Poisson arrival rate, requests per second")
    ap.add_argument("--seed", type=int, default=7)
    ap.add_argument("--steps", type=int, default=6)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"],
                    help="precision of the served runs; the sequential baseline is always FP64")
    a = ap.parse_args()
    import copy

    from . import dgls

    prec = dgls.MIXED if a.precision == "mixed" else dgls.FP64
    reqs = make_requests(a.requests, a.rate, a.seed, n_steps=a.steps)
    served, wall = serve(copy.deepcopy(reqs), slots=a.slots, precision=prec, keep_state=True)
    seqd, wall_seq = sequential(copy.deepcopy(reqs), keep_state=True)
    out = {"served": latency_stats(served, wall), "sequential_fp64": latency_stats(seqd, wall_seq),
           "precision_served": a.precision, "requests": len(reqs), "slots": a.slots,
           "statuses": sorted({r.result.get("status") for r in served})}
    if prec == dgls.FP64:
        out["identical_results_alone_and_in_mix"] = all(
            x.result.get("U_cell") == y.result.get("U_cell") and x.result.get("sha256") == y.result.get("sha256")
            for x, y in zip(sorted(served, key=lambda r: r.rid), sorted(seqd, key=lambda r: r.rid)))
    else:
        out["max_rel_diff_vs_fp64"] = max_rel_diff(served, seqd)
    out["throughput_gain"] = out["served"]["sims_per_hr"] / out["sequential_fp64"]["sims_per_hr"]
    out["p99_gain"] = out["sequential_fp64"]["p99_s"] / out["served"]["p99_s"]
    print(json.dumps(out))


if __name__ == "__main__":
    main()
