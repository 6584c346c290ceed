"""Batches of uneven instances (dg_batch_*): every instance's product, residual and implicit step in
the batch equal the same instance run alone, bitwise (the batched launches run the same device
functions on the same inputs; the steps run each context's own solver)."""
import numpy as np
import pytest

from oracle import chemistry as ch, init, lis
from paper_2511_05233_gb300 import inputs
from tests.gpu_helpers import ensure_built, structure_with_collector, to_dev

pytestmark = pytest.mark.gpu

# (side, order, porosity, correlation length, C-rate): uneven cubes of both orders, like the
# batched workload (sides 24-96 there; small here so that the test stays short)
SPECS = [(12, 1, 0.5, 2.0, 0.5), (9, 0, 0.6, 2.0, 1.0), (16, 1, 0.45, 3.0, 0.2), (20, 0, 0.7, 4.0, 2.0),
         (7, 1, 0.55, 2.0, 0.1), (33, 0, 0.5, 2.0, 0.7)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()


def _instances(precision):
    import torch

    from paper_2511_05233_gb300 import dgls

    out = []
    for k, (n, order, por, corr, fC) in enumerate(SPECS):
        phase = structure_with_collector(n, por, corr, 10 + k)
        model = lis.Model(ch.tradeoff(), order=order, f_C=fC, eps_struct=1.0 - por)
        grid = lis.Grid(phase, 1e-6)
        z0 = init.uniform_state(model, grid, init.equilibrium_fields(model))
        z = init.perturb(model, grid, z0, inputs.uniform_noise(z0.size, 20 + k))
        v = inputs.normal_noise(z.size, 30 + k) * (np.abs(z) + 1e-3)
        p = dgls.default_params(dgls.TRADEOFF, order, f_C=fC, eps_struct=1.0 - por, precision=precision)
        ctx = dgls.Context(phase, 1e-6, p, stream=torch.cuda.Stream())
        out.append((ctx, to_dev(z0), to_dev(z), to_dev(v)))
    return out


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batched_products_equal_products_alone(prec):
    import torch

    from paper_2511_05233_gb300 import dgls

    inst = _instances(dgls.MIXED)
    ts, dts = [1.5 + 0.1 * k for k in range(len(inst))], [1e-3 * (k + 1) for k in range(len(inst))]
    vs = [v if prec == "fp64" else v.float() for _, _, _, v in inst]
    alone = []
    for (ctx, z0, z, v), t, dt, vv in zip(inst, ts, dts, vs):
        o = torch.zeros_like(vv)
        ctx.jvp_fused(z, t, dt, vv, o)
        alone.append(o)
    torch.cuda.synchronize()
    batch = dgls.Batch([c for c, _, _, _ in inst])
    outs = [torch.full_like(vv, float("nan")) for vv in vs]
    batch.jvp([z for _, _, z, _ in inst], ts, dts, vs, outs)
    torch.cuda.synchronize()
    for k, (a, b) in enumerate(zip(alone, outs)):
        d = (a.double() - b.double()).abs()
        msg = (f"instance {k}: {int((a != b).sum())} of {a.numel()} differ, max |diff| {float(d.max()):.3e}, "
               f"max |diff|/|a| {float((d / a.double().abs().clamp_min(1e-30)).max()):.3e}, max |a| {float(a.abs().max()):.3e}")
        assert torch.equal(a, b), msg
    # after the autotuner has chosen the schedules, still the same results
    order, bs = batch.autotune([z for _, _, z, _ in inst], ts, dts, vs, outs)
    assert order in (0, 1) and bs in (64, 128, 256, 512)
    outs2 = [torch.full_like(vv, float("nan")) for vv in vs]
    batch.jvp([z for _, _, z, _ in inst], ts, dts, vs, outs2)
    torch.cuda.synchronize()
    for k, (a, b) in enumerate(zip(alone, outs2)):
        assert torch.equal(a, b), k
    n1 = sum(1 for s in SPECS if s[1] == 1)
    assert n1 > 1 and len(SPECS) - n1 > 1
    batch.close()


def test_batched_residuals_equal_residuals_alone():
    import torch

    from paper_2511_05233_gb300 import dgls

    inst = _instances(dgls.FP64)
    ts, dts = [0.7 * k for k in range(len(inst))], [1e-3] * len(inst)
    alone = []
    for (ctx, z0, z, v), t, dt in zip(inst, ts, dts):
        r = torch.zeros_like(z)
        ctx.residual(z, z0, t, dt, r)
        alone.append(r)
    torch.cuda.synchronize()
    batch = dgls.Batch([c for c, _, _, _ in inst])
    outs = [torch.full_like(z, float("nan")) for _, _, z, _ in inst]
    l0 = batch.launch_count()
    batch.residual([z for _, _, z, _ in inst], [z0 for _, z0, _, _ in inst], ts, dts, outs)
    torch.cuda.synchronize()
    for k, (a, b) in enumerate(zip(alone, outs)):
        assert torch.equal(a, b), k
    assert batch.launch_count() > l0
    batch.close()


def test_batched_steps_equal_steps_alone():
    import torch

    from paper_2511_05233_gb300 import dgls

    inst = _instances(dgls.FP64)
    ts, dts = [0.0] * len(inst), [1e-3] * len(inst)
    alone = []
    for (ctx, z0, z, v), t, dt in zip(inst, ts, dts):
        o = torch.zeros_like(z)
        st, info = ctx.step(z, o, t, dt)
        assert info.converged
        alone.append(o)
    batch = dgls.Batch([c for c, _, _, _ in inst])
    outs = [torch.zeros_like(z) for _, _, z, _ in inst]
    sts, infos = batch.step([z for _, _, z, _ in inst], outs, ts, dts)
    assert all(s == dgls.OK for s in sts) and all(i.converged for i in infos)
    for k, (a, b) in enumerate(zip(alone, outs)):
        assert torch.equal(a, b), k
    batch.close()


def test_batch_rejects_mixed_chemistries():
    from paper_2511_05233_gb300 import dgls

    ph = structure_with_collector(8, 0.5, 2.0, 1)
    a = dgls.Context(ph, 1e-6, dgls.default_params(dgls.TRADEOFF, 0))
    b = dgls.Context(ph, 1e-6, dgls.default_params(dgls.REDUCED3, 0))
    with pytest.raises(dgls.DGError):
        dgls.Batch([a, b])
