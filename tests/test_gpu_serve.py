"""Continuous-batching server: every simulation gives the same result alone and in the mix."""
import copy

import pytest

from tests.gpu_helpers import ensure_built

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()


def test_served_results_equal_sequential_results():
    from paper_2511_05233_gb300 import serve

    reqs = serve.make_requests(5, rate_hz=50.0, seed=3, side_range=(10, 16), n_steps=3)
    served, wall = serve.serve(copy.deepcopy(reqs), slots=3)
    alone, _ = serve.sequential(copy.deepcopy(reqs), time_scale=0.0)
    by_id = {r.rid: r for r in alone}
    for r in served:
        assert r.result["status"] == "DG_OK", r.result
        ref = by_id[r.rid].result
        assert r.result["U_cell"] == ref["U_cell"]          # bitwise: fixed-order reductions
        assert r.result["sha256"] == ref["sha256"]
    overlap = any(a.start < b.end and b.start < a.end for a in served for b in served if a.rid < b.rid)
    assert overlap, "no two requests ran concurrently"


def test_mixed_precision_serving_matches_fp64():
    """Requests served concurrently in mixed precision: bitwise the same as the same mixed runs
    alone, and within 1e-8 (U_cell curve and final state, relative) of the FP64 runs."""
    from paper_2511_05233_gb300 import dgls, serve

    reqs = serve.make_requests(4, rate_hz=50.0, seed=5, side_range=(10, 14), n_steps=3)
    served, _ = serve.serve(copy.deepcopy(reqs), slots=3, precision=dgls.MIXED, keep_state=True)
    alone, _ = serve.sequential(copy.deepcopy(reqs), time_scale=0.0, precision=dgls.MIXED, keep_state=True)
    ref, _ = serve.sequential(copy.deepcopy(reqs), time_scale=0.0, keep_state=True)
    by_id = {r.rid: r for r in alone}
    for r in served:
        assert r.result["status"] == "DG_OK", r.result
        assert r.result["sha256"] == by_id[r.rid].result["sha256"]
    err = serve.max_rel_diff(served, ref)
    assert err is not None and err["U_cell"] <= 1e-8 and err["state"] <= 1e-8, err


def test_context_in_caller_workspace_equals_own_allocations():
    """dg_setup_in: a context carved from a caller buffer of exactly dg_workspace_estimate bytes steps
    bitwise as one with its own allocations (and the buffer can be reused by the next context); a
    buffer 256 bytes short is refused with DG_ERR_OOM."""
    import numpy as np
    import torch

    from paper_2511_05233_gb300 import dgls
    from tests.gpu_helpers import make_case, to_dev

    for order in (0, 1):
        model, grid, phase, z0, z = make_case("tradeoff", order, (8, 5, 4))
        p = dgls.default_params(dgls.TRADEOFF, order, f_C=model.f_C, eps_struct=model.eps_struct)
        need = dgls.workspace_estimate(phase, 1e-6, p)
        ws = torch.empty(need, dtype=torch.uint8, device="cuda")
        outs = []
        for trial in range(2):                     # the second context reuses the first one's buffer
            c = dgls.Context(phase, 1e-6, p, workspace=ws)
            o = to_dev(np.zeros_like(z))
            st, info = c.step(to_dev(z), o, 0.0, 1e-3)
            assert info.converged
            outs.append(o.cpu().numpy())
            c.close()
        ref = dgls.Context(phase, 1e-6, p)
        o = to_dev(np.zeros_like(z))
        ref.step(to_dev(z), o, 0.0, 1e-3)
        assert np.array_equal(outs[0], o.cpu().numpy()) and np.array_equal(outs[1], outs[0])
        with pytest.raises(dgls.DGError) as e:
            dgls.Context(phase, 1e-6, p, workspace=ws[: need - 256])
        assert e.value.status == dgls.ERR_OOM
