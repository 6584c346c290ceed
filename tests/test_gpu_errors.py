"""Error paths and checkpoint/resume of the C ABI.  Every failure is made on the host -- a workspace
budget, a NaN planted in a host copy of the state, a structure without a collector voxel, a Newton
limit no step can meet -- so no test faults, traps or hangs the GPU."""
import numpy as np
import pytest

from tests.gpu_helpers import ensure_built, gpu_context, make_case, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()


def test_workspace_budget_below_need_is_oom():
    from paper_2511_05233_gb300 import dgls

    model, grid, phase, z0, z = make_case("tradeoff", 0, (8, 5, 4))
    with pytest.raises(dgls.DGError) as e:
        gpu_context(model, phase, hbm_budget_bytes=4096)
    assert e.value.status == dgls.ERR_OOM
    ctx = gpu_context(model, phase, hbm_budget_bytes=1 << 34)     # 16 GiB: fits
    assert 0 < ctx.workspace_bytes() <= 1 << 34


def test_structure_without_collector_voxel_is_rejected():
    from paper_2511_05233_gb300 import dgls

    model, grid, phase, z0, z = make_case("tradeoff", 0, (8, 5, 4))
    ph = phase.copy()
    ph[:, :, 0][ph[:, :, 0] == 1] = 0                 # no structure voxel on the x = 0 face
    with pytest.raises(dgls.DGError) as e:
        gpu_context(model, ph)
    assert e.value.status == dgls.ERR_ARG


@pytest.mark.parametrize("order", [0, 1])
def test_nan_in_uploaded_state_is_nonfinite(order):
    """A NaN in the host copy of z^n that dg_step_host uploads: the first residual is not finite,
    the step returns DG_ERR_NONFINITE and says so."""
    from paper_2511_05233_gb300 import dgls

    model, grid, phase, z0, z = make_case("tradeoff", order, (6, 4, 3))
    ctx = gpu_context(model, phase)
    zh = z.copy()
    zh[zh.size // 3] = np.nan
    out = np.zeros_like(zh)
    st, info = ctx.step_host(zh, out, 0.0, 1e-3, check=False)
    assert st == dgls.ERR_NONFINITE
    assert "non-finite" in ctx._lib.dg_last_error(ctx._h).decode()
    st, info = ctx.step_host(z, out, 0.0, 1e-3, check=False)     # the context stays usable
    assert st == dgls.OK and info.converged


def test_naive_controller_aborts_on_the_31st_consecutive_halving():
    """Fig. 4: a failed step halves dt; the 31st consecutive failure ends the run with
    DG_ERR_ABORTED.  From a perturbed state (concentrations 1 % off equilibrium) the first residual
    is far above the Newton tolerance, and with newton_max_it = 0 no attempt may iterate, so every
    attempt fails and the controller halves until it gives up."""
    from paper_2511_05233_gb300 import dgls

    model, grid, phase, z0, z = make_case("tradeoff", 0, (6, 4, 3))
    ctx = gpu_context(model, phase, newton_max_it=0)
    zd = to_dev(z)
    res = ctx.discharge(zd, controller=dgls.NAIVE, dt0=1e-3, dt_min=1e-300, max_steps=10)
    assert res["status"] == "DG_ERR_ABORTED"
    assert res["attempts"] == 31 and res["failures"] == 31 and len(res["t"]) == 0
    assert res["checkpoint"]["halvings"] == 31


def _discharge_split(order, controller, n_total, n_first, **kw):
    """(uninterrupted run, run split at n_first with the state copied to the host and continued in
    a new context from the checkpoint)."""
    import torch

    from paper_2511_05233_gb300 import dgls

    model, grid, phase, z0, z = make_case("tradeoff", order, (8, 5, 4) if order == 0 else (6, 4, 3))
    ctx = gpu_context(model, phase)
    za = ctx.new_state()
    ctx.equilibrium_state(za)
    zb = za.clone()
    full = ctx.discharge(za, controller=controller, max_steps=n_total, **kw)
    first = ctx.discharge(zb, controller=controller, max_steps=n_first, **kw)
    host = zb.cpu().numpy().copy()                     # the checkpoint: state on the host + record
    ck = first["checkpoint"]
    ctx.close()
    ctx2 = gpu_context(model, phase)
    zc = torch.from_numpy(host).cuda()
    second = ctx2.discharge(zc, controller=controller, max_steps=n_total - n_first, resume=ck, **kw)
    return full, first, second, za.cpu().numpy(), zc.cpu().numpy()


@pytest.mark.parametrize("order,controller", [(0, 0), (0, 1), (1, 0)])
def test_checkpoint_resume_is_bitwise(order, controller):
    """A discharge stopped after some accepted steps, its state saved on the host, and resumed in
    a fresh context from the controller record continues bitwise as the uninterrupted run: same
    step sizes, same U_cell values, same final state (deterministic reductions)."""
    n_total, n_first = (10, 4) if order == 0 else (4, 2)
    full, first, second, zfull, zsplit = _discharge_split(order, controller, n_total, n_first,
                                                          dt0=1e-3, tol=1e-4)
    assert full["status"] == first["status"] == second["status"] == "DG_OK"
    for k in ("t", "dt", "U_cell"):
        joined = np.concatenate([first[k], second[k]])
        assert np.array_equal(joined, full[k]), k
    assert np.array_equal(zsplit, zfull)
    assert second["checkpoint"] == full["checkpoint"]


def test_isolated_passivated_collector_voxel_keeps_the_preconditioner_finite():
    """A collector voxel with no structure neighbour whose surface has passivated (a_V = 0, Eq. 18
    with the Eq. 57 localisation) has an empty Phi^S row.  On a grid of at most 64 voxels the
    multigrid's dense coarsest inverse is built on the fine level itself, where that row used to
    give a zero pivot and NaN.  The step has no solution (the collector current of that face has
    nowhere to go), so it must end as DG_ERR_NOCONV with a finite state, not DG_ERR_NONFINITE."""
    import torch

    from paper_2511_05233_gb300 import dgls

    ph = np.zeros((4, 4, 4), dtype=np.uint8)           # (z, y, x)
    ph[:, :, 2:] = 2                                   # separator layers x = 2, 3
    ph[0:2, 0:2, 0:2] = 1                              # a structure cluster on the collector
    ph[3, 3, 0] = 1                                    # isolated collector voxel
    assert ph[3, 3, 1] == 0 and ph[2, 3, 0] == 0 and ph[3, 2, 0] == 0
    p = dgls.default_params(dgls.TRADEOFF, 0, f_C=0.5, eps_struct=0.4, gmres_max_it=200)
    ctx = dgls.Context(ph, 1e-6, p)
    z = ctx.new_state()
    ctx.equilibrium_state(z)
    off7, len7 = ctx.offsets[7], ctx.lengths[7]         # eps_Li2S, one value per structure voxel
    z[off7 + len7 - 1] = 0.1                           # > a e^{-b f_C} / eps_struct = 0.0665: a_V = 0
    out = torch.empty_like(z)
    st, info = ctx.step(z, out, 0.0, 1e-3, check=False)
    assert st == dgls.ERR_NOCONV, dgls.STATUS.get(st, st)
    assert torch.isfinite(out).all()
