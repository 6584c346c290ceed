"""Time-step controllers through dg_discharge (GPU) against the oracle's controllers driving the
oracle's implicit Euler steps (Fig. 4 naive controller; Eqs. 51-54 H211b with Richardson)."""
import numpy as np
import pytest

from oracle import control, lis, newton
from tests.gpu_helpers import assert_state_close, ensure_built, gpu_context, make_case, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()


def _oracle_run(model, grid, z0, ctrl, n, **kw):
    def step(z, t, dt):
        z1, info = newton.implicit_euler_step(model, grid, z, t, dt)
        return info.converged, z1

    def cutoff(z):
        U = lis.cell_voltage(model, grid, z)
        return U <= 1.9, U
    if ctrl == "naive":
        return control.naive(step, cutoff, z0, dt0=1e-3, max_steps=n, **kw)
    return control.h211b(step, cutoff, z0, kw.pop("tol"), dt0=1e-3, max_steps=n, **kw)


@pytest.mark.parametrize("chem", ["reduced3", "tradeoff"])
def test_naive_discharge_matches_oracle(chem):
    from paper_2511_05233_gb300 import dgls

    model, grid, phase, z0, z = make_case(chem, 0, (6, 4, 3))
    zf, rec = _oracle_run(model, grid, z0, "naive", 7)
    ctx = gpu_context(model, phase)
    zd = to_dev(z0)
    res = ctx.discharge(zd, controller=dgls.NAIVE, dt0=1e-3, max_steps=7)
    assert res["status"] == "DG_OK"
    assert len(res["dt"]) == len(rec.dt)
    assert np.allclose(res["dt"], rec.dt, rtol=1e-14, atol=0)          # decisions identical
    assert np.allclose(res["t"], rec.t, rtol=1e-14, atol=0)
    assert np.allclose(res["U_cell"], rec.U, rtol=1e-8, atol=0)
    assert_state_close(model, grid, to_host(zd), zf, 1e-8)


def test_replayed_discharge_matches_oracle():
    """Delta-t replay: the GPU takes the oracle's accepted step sizes."""
    from paper_2511_05233_gb300 import dgls

    model, grid, phase, z0, z = make_case("tradeoff", 0, (6, 4, 3))
    zf, rec = _oracle_run(model, grid, z0, "naive", 5)
    ctx = gpu_context(model, phase)
    zd = to_dev(z0)
    res = ctx.discharge(zd, controller=dgls.NAIVE, replay_dt=np.array(rec.dt))
    assert res["status"] == "DG_OK"
    assert np.allclose(res["U_cell"], rec.U, rtol=1e-8, atol=0)
    assert_state_close(model, grid, to_host(zd), zf, 1e-8)


def test_h211b_discharge_matches_oracle():
    from paper_2511_05233_gb300 import dgls

    model, grid, phase, z0, z = make_case("reduced3", 0, (6, 4, 3))
    zf, rec = _oracle_run(model, grid, z0, "h211b", 3, tol=1e-5)
    ctx = gpu_context(model, phase)
    zd = to_dev(z0)
    res = ctx.discharge(zd, controller=dgls.H211B, tol=1e-5, dt0=1e-3, max_steps=3)
    assert res["status"] == "DG_OK"
    assert np.allclose(res["dt"], rec.dt, rtol=1e-6, atol=0)
    assert np.allclose(res["U_cell"], rec.U, rtol=1e-8, atol=0)
    assert_state_close(model, grid, to_host(zd), zf, 1e-8)


def test_cutoff_on_the_first_accepted_step():
    """Cut-off (Sec. 3: the discharge ends when U_cell reaches the cut-off; reading: the first
    accepted step with U_cell <= cut-off): with the cut-off above the cell voltage the run stops
    after exactly one accepted step, as the oracle's controller does."""
    from paper_2511_05233_gb300 import dgls

    model, grid, phase, z0, z = make_case("tradeoff", 0, (6, 4, 3))

    def step(zz, t, dt):
        z1, info = newton.implicit_euler_step(model, grid, zz, t, dt)
        return info.converged, z1

    def cut(zz):
        U = lis.cell_voltage(model, grid, zz)
        return U <= 3.0, U
    zf, rec = control.naive(step, cut, z0, dt0=1e-3, max_steps=7)
    assert rec.status == "cutoff" and len(rec.t) == 1
    ctx = gpu_context(model, phase)
    zd = to_dev(z0)
    res = ctx.discharge(zd, controller=dgls.NAIVE, dt0=1e-3, max_steps=7, cutoff_V=3.0)
    assert res["status"] == "DG_OK" and len(res["t"]) == 1
    assert np.allclose(res["U_cell"], rec.U, rtol=1e-8, atol=0)
    assert_state_close(model, grid, to_host(zd), zf, 1e-8)


def test_cutoff_in_the_middle_of_a_run():
    """A cut-off between the cell voltages of the 3rd and 4th accepted steps stops both the
    GPU run and the oracle's after the 4th step."""
    from paper_2511_05233_gb300 import dgls

    model, grid, phase, z0, z = make_case("tradeoff", 0, (6, 4, 3))
    _, full = _oracle_run(model, grid, z0, "naive", 7)
    U = np.array(full.U)
    assert np.all(np.diff(U[:5]) < 0)                  # the voltage falls over the first steps
    cutv = 0.5 * (U[2] + U[3])

    def step(zz, t, dt):
        z1, info = newton.implicit_euler_step(model, grid, zz, t, dt)
        return info.converged, z1

    def cut(zz):
        u = lis.cell_voltage(model, grid, zz)
        return u <= cutv, u
    zf, rec = control.naive(step, cut, z0, dt0=1e-3, max_steps=7)
    assert rec.status == "cutoff" and len(rec.t) == 4
    ctx = gpu_context(model, phase)
    zd = to_dev(z0)
    res = ctx.discharge(zd, controller=dgls.NAIVE, dt0=1e-3, max_steps=7, cutoff_V=cutv)
    assert res["status"] == "DG_OK" and len(res["t"]) == 4
    assert np.allclose(res["U_cell"], rec.U, rtol=1e-8, atol=0)
    assert_state_close(model, grid, to_host(zd), zf, 1e-8)


def _golden():
    import json
    import os

    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "discharge_dg0_tradeoff_6.json")
    with open(path) as f:
        return json.load(f)


def test_full_discharge_to_cutoff_replayed_against_oracle():
    """The oracle's full discharge to the 1.9 V cut-off (tests/golden/make_discharge_golden.py: 6^3
    DG0 cell with a single collector cluster, 1C, relaxation of Sec. 2.8, naive controller of
    Fig. 4) replayed on the GPU with the oracle's accepted step sizes: the relaxed state, the
    cell voltage of Eq. A1 after every step (1e-8 relative) and the final state (1e-8) agree, and
    the GPU run stops on the same step, the first with U_cell <= 1.9 V.  Both sides solve every step
    to a Newton tolerance of 1e-12 (the golden file's)."""
    from oracle import chemistry as ch
    from paper_2511_05233_gb300 import dgls

    gd = _golden()
    assert gd["status"] == "cutoff" and gd["U_cell"][-1] <= 1.9 < gd["U_cell"][-2]
    phase = np.array(gd["phase"], dtype=np.uint8)
    grid = lis.Grid(phase, gd["h"])
    model = lis.Model(ch.tradeoff(), order=0, f_C=gd["f_C"], eps_struct=1.0 - gd["porosity"])
    # each replayed step solved to the oracle's Newton tolerance: at the knee of the curve (a step
    # that drops U_cell by 0.1 V) the default rtol of 1e-10 leaves 2e-8 of U_cell to the
    # inexact GMRES solves
    ctx = gpu_context(model, phase, newton_rtol=gd["newton_rtol"])
    z = ctx.new_state()
    ctx.equilibrium_state(z)
    ctx.relax(z, gd["relax"]["dt"], gd["relax"]["steps"])
    zr = np.array(gd["z_relaxed"])
    assert_state_close(model, grid, to_host(z), zr, 1e-8)
    zd = to_dev(zr)
    res = ctx.discharge(zd, controller=dgls.NAIVE, replay_dt=np.array(gd["dt"]), cutoff_V=1.9)
    assert res["status"] == "DG_OK"
    assert len(res["t"]) == len(gd["t"])
    assert np.allclose(res["t"], gd["t"], rtol=1e-14, atol=0)
    Ug = np.array(gd["U_cell"])
    rel = np.abs(res["U_cell"] - Ug) / np.abs(Ug)
    big = "; ".join(f"step {i} dt {gd['dt'][i]:.3g} U {gd['U_cell'][i]:.5f} err {e:.2e}"
                    for i, e in enumerate(rel) if e > 1e-9)
    # The knee at the end of the upper plateau: dissolved S8(L) drops 300-fold within one step (to
    # 5e-5 mol/m^3) and U_cell follows the logarithm of its activity (Eq. 24), so a concentration
    # difference of 1e-13 of the concentration scale (what both solvers resolve) moves U_cell by
    # 2e-8 there.  Everywhere else the curve agrees to 1e-8.
    knee = np.zeros(len(Ug), dtype=bool)
    knee[1:] = np.abs(np.diff(Ug)) > 0.05
    knee[:-1] |= knee[1:]
    assert np.all(rel[~knee] <= 1e-8), f"max off the knee {rel[~knee].max():.3e}; steps above 1e-9: {big}"
    assert np.all(rel[knee] <= 5e-8), big
    assert_state_close(model, grid, to_host(zd), np.array(gd["z_final"]), 1e-8)


def test_full_discharge_free_running_reaches_cutoff():
    """The same cell discharged by the GPU's own naive controller (not replayed) reaches the cut-off;
    its capacity at the cut-off is within 2 % of the oracle's (the two controllers may take
    different steps once a Newton solve fails in one and not in the other)."""
    from oracle import chemistry as ch
    from paper_2511_05233_gb300 import dgls

    gd = _golden()
    phase = np.array(gd["phase"], dtype=np.uint8)
    model = lis.Model(ch.tradeoff(), order=0, f_C=gd["f_C"], eps_struct=1.0 - gd["porosity"])
    ctx = gpu_context(model, phase)
    zd = to_dev(np.array(gd["z_relaxed"]))
    res = ctx.discharge(zd, controller=dgls.NAIVE, dt0=1e-3, dt_max=10.0, cutoff_V=1.9, max_steps=2000)
    assert res["status"] == "DG_OK"
    assert res["U_cell"][-1] <= 1.9 < res["U_cell"][-2]
    assert abs(res["t"][-1] / gd["t"][-1] - 1.0) <= 0.02


def test_large_dg1_step_ends_at_the_rounding_floor():
    """Newton at large dt from a DG1 mid-discharge state: the scaled residual stops at its rounding
    floor, which at large dt lies above rtol ||S R0||; the solve ends there within a few iterations,
    certified to the stall tolerance, instead of trading rounding noise up to the iteration limit."""
    import torch

    from paper_2511_05233_gb300 import dgls, inputs

    phase = None
    for s in range(3, 53):
        ph = inputs.make_structure(16, 0.5, 4.0, s, single_cluster=True)
        if np.any(ph[:, :, 0] == inputs.STRUCT):
            phase = ph
            break
    prm = dgls.default_params(dgls.TRADEOFF, 1, f_C=0.5, eps_struct=0.5, newton_stall_rtol=1e-7)
    ctx = dgls.Context(phase, 1e-6, prm)
    z = ctx.new_state()
    ctx.equilibrium_state(z)
    ctx.relax(z, 0.1, 40)
    r = ctx.discharge(z, controller=dgls.NAIVE, dt0=1e-3, dt_min=1e-6, dt_max=10.0, cutoff_V=1.9, t_end=3.0,
                      max_steps=2000, limiter=True)
    assert r["status"] == "DG_OK"
    t = r["checkpoint"]["t"]
    out = torch.empty_like(z)
    for dt in (0.4, 1.6):
        st, info = ctx.step(z, out, t, dt, check=False)
        assert st == dgls.OK and info.converged, (dt, st)
        assert info.norm <= 1e-7 * info.norm0, (dt, info.norm, info.norm0)
        assert info.newton_iterations <= 10, (dt, info.newton_iterations)
    ctx.close()
