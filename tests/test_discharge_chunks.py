"""The chunked discharge loop of discharge_run.py on the host (no GPU): a fake context stands in for
dg_discharge, so that the chunking, the resume hand-off and every stopping rule are checked."""
import io
import json

import numpy as np

from paper_2511_05233_gb300.discharge_run import discharge_in_chunks


class FakeContext:
    """Accepted steps of 1 s each; U_cell falls by 0.01 V per step from 2.4 V, so the step that
    reaches 1.9 V is the 50th.  `fail_at` makes the call that would take that step return a failure."""

    def __init__(self, fail_at=None):
        self.calls = []
        self.fail_at = fail_at

    def discharge(self, z, controller, dt0, dt_min, dt_max, cutoff_V, t_end, max_steps, limiter, resume):
        k0 = 0 if resume is None else int(round(resume["t"]))
        self.calls.append({"resume": resume, "max_steps": max_steps, "controller": controller})
        t, U = [], []
        status = "DG_OK"
        for k in range(k0 + 1, k0 + max_steps + 1):
            if self.fail_at is not None and k == self.fail_at:
                status = "DG_ERR_ABORTED"
                break
            t.append(float(k))
            U.append(2.4 - 0.01 * k)
            if U[-1] <= cutoff_V + 1e-12 or (t_end > 0 and k >= t_end):
                break
        n = len(t)
        tk = t[-1] if n else float(k0)
        return {"t": np.array(t), "dt": np.ones(n), "U_cell": np.array(U), "c_m": np.array(t) * 0.2,
                "newton_its": np.full(n, 4, np.int32), "gmres_its": np.full(n, 30, np.int32), "status": status,
                "attempts": n + (status != "DG_OK"), "failures": int(status != "DG_OK"),
                "checkpoint": {"t": tk, "dt": 1.0, "err_prev": 0.0, "dt_prev": 0.0, "sct": 0, "halvings": 0}}


def test_chunks_resume_from_each_other_and_stop_at_the_cutoff():
    ctx = FakeContext()
    log = io.StringIO()
    res = discharge_in_chunks(ctx, None, 0, 0.0, 5000, True, chunk=20, progress=True, log=log)
    assert [c["max_steps"] for c in ctx.calls] == [20, 20, 20]
    assert ctx.calls[0]["resume"] is None
    assert [c["resume"]["t"] for c in ctx.calls[1:]] == [20.0, 40.0]
    assert len(res["t"]) == 50 and np.array_equal(res["t"], np.arange(1.0, 51.0))
    assert res["U_cell"][-1] <= 1.9 and res["status"] == "DG_OK"
    assert res["attempts"] == 50 and res["failures"] == 0
    lines = [json.loads(x) for x in log.getvalue().splitlines()]
    assert [x["steps"] for x in lines] == [20, 40, 50] and lines[-1]["t"] == 50.0


def test_max_steps_and_t_end_end_the_run():
    ctx = FakeContext()
    res = discharge_in_chunks(ctx, None, 0, 0.0, 33, True, chunk=10)
    assert [c["max_steps"] for c in ctx.calls] == [10, 10, 10, 3] and len(res["t"]) == 33
    ctx = FakeContext()
    res = discharge_in_chunks(ctx, None, 0, 25.0, 5000, True, chunk=10)
    assert res["t"][-1] == 25.0 and len(ctx.calls) == 3


def test_a_failed_chunk_ends_the_run_with_its_status():
    ctx = FakeContext(fail_at=17)
    res = discharge_in_chunks(ctx, None, 0, 0.0, 5000, True, chunk=10)
    assert res["status"] == "DG_ERR_ABORTED" and len(res["t"]) == 16 and res["failures"] == 1
    assert len(ctx.calls) == 2


def test_the_wall_clock_limit_ends_the_run_between_chunks():
    ticks = iter(range(0, 10000, 10))            # every clock read advances 10 s
    ctx = FakeContext()
    res = discharge_in_chunks(ctx, None, 0, 0.0, 5000, True, wall_limit=25.0, chunk=5, clock=lambda: next(ticks))
    # reads: start 0; after chunk 1: 10 (<= 25, go on); after chunk 2: 20; after chunk 3: 30 (> 25, stop)
    assert len(ctx.calls) == 3 and len(res["t"]) == 15 and res["status"] == "DG_OK"
