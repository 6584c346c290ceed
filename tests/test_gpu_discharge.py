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
