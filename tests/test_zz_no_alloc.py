"""dg_residual_noalloc: the DG0 residual for callers that cannot allocate device memory when they
call (for example inside CUDA stream capture) and must not use the context's workspaces.  It keeps
its scratch in a static device array; its result must equal dg_residual's, call after call.

Collected last (file name), so that a run stopping at the first failure has run everything else."""

import numpy as np
import pytest

from tests.gpu_helpers import ensure_built, gpu_context, make_case, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()


def test_noalloc_residual_matches_dg_residual_twice():
    from oracle import lis

    model, grid, phase, z0, z = make_case("tradeoff", 0, (13, 7, 5), potential_noise=0.01)
    ctx = gpu_context(model, phase)
    t, dt = 1.5, 1e-3
    M = lis.residual_magnitude(model, grid, z, z0, t, dt)
    zd, z0d = to_dev(z), to_dev(z0)
    ref = to_dev(np.zeros_like(z))
    ctx.residual(zd, z0d, t, dt, ref)
    R = to_host(ref)
    for _ in range(2):
        out = to_dev(np.full_like(z, np.nan))
        ctx.residual_noalloc(zd, z0d, t, dt, out)
        got = to_host(out)
        assert np.all(np.abs(got - R) <= 1e-12 * M)
    # a second, different input through the same static scratch
    z2 = z * (1.0 + 1e-3)
    ctx.residual(to_dev(z2), z0d, t, dt, ref)
    out = to_dev(np.zeros_like(z))
    ctx.residual_noalloc(to_dev(z2), z0d, t, dt, out)
    M2 = lis.residual_magnitude(model, grid, z2, z0, t, dt)
    assert np.all(np.abs(to_host(out) - to_host(ref)) <= 1e-12 * M2)


def test_noalloc_rejects_dg1_with_a_message():
    from paper_2511_05233_gb300 import dgls

    model, grid, phase, z0, z = make_case("reduced3", 1, (6, 4, 3))
    ctx = gpu_context(model, phase)
    out = to_dev(np.zeros_like(z))
    with pytest.raises(dgls.DGError, match="DG0 contexts only"):
        ctx.residual_noalloc(to_dev(z), to_dev(z0), 0.0, 1e-3, out)
