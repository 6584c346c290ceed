"""Adaptive time-step controllers (Sec. 2.7): naive feedback (Fig. 4) and H211b (Eqs. 51-54).

Test infrastructure (see package docstring).  Both controllers drive a callback
``step(z, t, dt) -> (ok, z_new)`` that performs one implicit Euler step and report the
accepted steps; ``cutoff(z) -> (stop, U_cell)`` ends the discharge (1.9 V, Sec. 3).

Readings (the flow charts of Figs. 4 and 5 are not reproduced in the text):
* naive: on a converged step sct += 1 and, when sct reaches 3, dt *= 1.2 and sct = 0;
  dt is capped at dt_max.  On a failed step dt /= 2 and sct = 0; the 31st consecutive
  halving (or dt below dt_min) aborts the run.
* H211b: each attempt solves the coarse step z_C (dt) and the fine pair z_F (2 x dt/2);
  err = ||z_F - z_C||_2 / ||z_F||_2 over the whole state (Eq. 53);
  ratio = (tol/err)^{1/4} (tol/err_prev)^{1/4} (dt/dt_prev)^{-1/4} (Eq. 51) and
  lim = 1 + atan(ratio - 1) (Eq. 52).  The attempt is rejected when err > 1.02 tol or
  lim < 0.9 and retried with dt *= lim; otherwise z = 2 z_F - z_C (Eq. 54), t += dt and
  the next dt = lim * dt.  lim starts at 0 each step, forcing one filter call.  For the
  first step err_prev = tol and dt_prev = dt.  Each filter call takes the most recent
  attempt as its previous data point: after a rejected attempt (err_prev, dt_prev) are that
  attempt's values (with the accepted step's history instead, the retry loop can settle on
  a dt whose filter ratio is 1 while err stays above tol).  More than 50 retries in one
  step abort the run.  Solver failures halve dt as in the naive controller.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Record:
    t: list = field(default_factory=list)
    dt: list = field(default_factory=list)
    U: list = field(default_factory=list)
    status: str = "running"
    failures: int = 0
    attempts: int = 0


def naive(step, cutoff, z0, t0=0.0, dt0=1e-3, dt_min=1e-6, dt_max=10.0, max_halvings=30,
          max_steps=10 ** 9, t_end=math.inf, replay=None):
    """Fig. 4.  ``replay``: a list of step sizes to take instead of the controller's (each must converge)."""
    rec = Record()
    z, t, dt, sct, halv = z0, t0, dt0, 0, 0
    n = 0
    while n < max_steps and t < t_end:
        if replay is not None:
            if n >= len(replay):
                break
            dt = replay[n]
        rec.attempts += 1
        ok, zn = step(z, t, dt)
        if ok:
            z, t = zn, t + dt
            n += 1
            halv = 0
            stop, U = cutoff(z)
            rec.t.append(t)
            rec.dt.append(dt)
            rec.U.append(U)
            if stop:
                rec.status = "cutoff"
                return z, rec
            sct += 1
            if sct == 3:
                dt *= 1.2
                sct = 0
            dt = min(dt, dt_max)
        else:
            if replay is not None:
                rec.status = "replay_failed"
                return z, rec
            rec.failures += 1
            dt *= 0.5
            sct = 0
            halv += 1
            if halv > max_halvings or dt < dt_min:
                rec.status = "aborted"
                return z, rec
    rec.status = "max_steps" if n >= max_steps else "t_end"
    return z, rec


def h211b_ratio(err, err_prev, dt, dt_prev, tol):
    """Eq. 51: dt^{n+1}/dt^n."""
    return (tol / err) ** 0.25 * (tol / err_prev) ** 0.25 * (dt / dt_prev) ** -0.25


def h211b_limit(ratio):
    """Eq. 52: 1 + arctan(ratio - 1)."""
    return 1.0 + math.atan(ratio - 1.0)


def rel_error(zF, zC):
    """Eq. 53: sqrt(sum (z_F - z_C)^2 / sum z_F^2)."""
    return float(np.sqrt(np.sum((zF - zC) ** 2) / np.sum(zF ** 2)))


def h211b(step, cutoff, z0, tol, t0=0.0, dt0=1e-3, dt_min=1e-6, dt_max=10.0, max_halvings=30,
          max_steps=10 ** 9, t_end=math.inf, max_retries=50):
    """Fig. 5 with Eqs. 51-54 (see module docstring for the reading)."""
    rec = Record()
    z, t, dt = z0, t0, dt0
    err_prev, dt_prev = tol, dt0
    halv = 0
    n = 0
    while n < max_steps and t < t_end:
        lim = 0.0
        err = math.inf
        tries = 0
        while err > 1.02 * tol or lim < 0.9:
            rec.attempts += 1
            okC, zC = step(z, t, dt)
            okF1, zF1 = step(z, t, 0.5 * dt) if okC else (False, None)
            okF, zF = step(zF1, t + 0.5 * dt, 0.5 * dt) if okF1 else (False, None)
            if not (okC and okF1 and okF):
                rec.failures += 1
                dt *= 0.5
                halv += 1
                lim = 0.0
                err = math.inf
                if halv > max_halvings or dt < dt_min:
                    rec.status = "aborted"
                    return z, rec
                continue
            halv = 0
            err = max(rel_error(zF, zC), 1e-300)
            lim = h211b_limit(h211b_ratio(err, err_prev, dt, dt_prev, tol))
            if err > 1.02 * tol or lim < 0.9:
                tries += 1
                if tries > max_retries:
                    rec.status = "aborted"
                    return z, rec
                err_prev, dt_prev = err, dt
                dt = min(dt * lim, dt_max)
        z = 2.0 * zF - zC
        t += dt
        n += 1
        stop, U = cutoff(z)
        rec.t.append(t)
        rec.dt.append(dt)
        rec.U.append(U)
        err_prev, dt_prev = err, dt
        dt = min(lim * dt, dt_max)
        if stop:
            rec.status = "cutoff"
            return z, rec
    rec.status = "max_steps" if n >= max_steps else "t_end"
    return z, rec
