"""Parity of the fused matrix-free DG1 Jacobian-vector product (dg_jvp_fused) with the oracle's
complex-step product, element by element.

FP64 instantiation: |err| <= 1e-12 |J| |v| (rounding of a sum of products of the size |J| |v|).
FP32 instantiation (the product of the mixed-precision Krylov loop): z and v are rounded to FP32
(relative 2^-24 = 6e-8) and the arithmetic is FP32, with the hardware exponential and logarithm.
The largest sensitivity is the Butler-Volmer exponent F (Phi^S - Phi^L - U0) / (2RT): a rounding
of Phi^S ~ 2.5 V moves it by 19.5 V^-1 x 2.5 V x 6e-8 = 3e-6, and through the exponentials each
reaction term by that fraction; the hardware exponential adds |x| 2^-24 <= 2.4e-6 for the
arguments |x| <= 40 of the rates, and sums of a few dozen rounded products add about as much
again.  The stated bound is |err| <= 2e-5 |J| |v| (measured maximum 8.2e-6 on the 10 x 6 x 5
and 16^3 cases).
"""
import numpy as np
import pytest

from oracle import newton
from paper_2511_05233_gb300 import inputs
from tests.gpu_helpers import ensure_built, gpu_context, make_case, to_dev, to_host

pytestmark = pytest.mark.gpu

CASES = [("reduced3", (7, 5, 4)), ("tradeoff", (7, 5, 4)), ("tradeoff", (10, 6, 5)), ("tradeoff", (33, 3, 2))]
FP32_BOUND = 2e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()


def _case(chem, n, seed=1):
    model, grid, phase, z0, z = make_case(chem, 1, n, potential_noise=0.01, seed=seed)
    v = inputs.normal_noise(z.size, 7) * (np.abs(z) + 1e-3)
    return model, grid, phase, z0, z, v


@pytest.mark.parametrize("chem,n", CASES)
def test_fused_fp64_product_matches_oracle(chem, n):
    """(33, 3, 2): two blocks of 32 voxels along x, so the neighbour across a block edge comes from
    global memory and the ragged last block has idle lanes."""
    model, grid, phase, z0, z, v = _case(chem, n)
    t, dt = 1.5, 1e-3
    ref = newton.jvp(model, grid, z, z0, t, dt, v)
    mag = newton.abs_jacobian_times(model, grid, z, z0, t, dt, v, workers=7)
    ctx = gpu_context(model, phase)
    out = to_dev(np.zeros_like(z))
    ctx.jvp_fused(to_dev(z), t, dt, to_dev(v), out)
    err = np.abs(to_host(out) - ref)
    assert np.all(err <= 1e-12 * mag + 1e-300), (err / np.maximum(mag, 1e-300)).max()


@pytest.mark.parametrize("chem,n", CASES)
def test_fused_fp32_product_matches_oracle(chem, n):
    import torch

    from paper_2511_05233_gb300 import dgls

    model, grid, phase, z0, z, v = _case(chem, n)
    t, dt = 1.5, 1e-3
    ref = newton.jvp(model, grid, z, z0, t, dt, v)
    mag = newton.abs_jacobian_times(model, grid, z, z0, t, dt, v, workers=7)
    ctx = gpu_context(model, phase, precision=dgls.MIXED)
    v32 = torch.from_numpy(v.astype(np.float32)).cuda()
    out = torch.zeros(z.size, dtype=torch.float32, device="cuda")
    ctx.jvp_fused(to_dev(z), t, dt, v32, out)
    err = np.abs(out.cpu().numpy().astype(np.float64) - ref)
    assert np.all(err <= FP32_BOUND * mag + 1e-30), (err / np.maximum(mag, 1e-300)).max()


def test_fused_products_on_16_cubed_structure():
    """A 16^3 random-field structure (4096 voxels, 128 blocks, every kind of boundary voxel): the
    FP64 product at 1e-12 |J||v| and the FP32 product at the FP32 bound, element by element."""
    import torch

    from paper_2511_05233_gb300 import dgls

    model, grid, phase, z0, z, v = _case("tradeoff", (16, 16, 16))
    t, dt = 1.5, 1e-3
    ref = newton.jvp(model, grid, z, z0, t, dt, v)
    mag = newton.abs_jacobian_times(model, grid, z, z0, t, dt, v, workers=8)
    ctx = gpu_context(model, phase, precision=dgls.MIXED)
    out = to_dev(np.zeros_like(z))
    ctx.jvp_fused(to_dev(z), t, dt, to_dev(v), out)
    err = np.abs(to_host(out) - ref)
    assert np.all(err <= 1e-12 * mag + 1e-300), (err / np.maximum(mag, 1e-300)).max()
    v32 = torch.from_numpy(v.astype(np.float32)).cuda()
    o32 = torch.zeros(z.size, dtype=torch.float32, device="cuda")
    ctx.jvp_fused(to_dev(z), t, dt, v32, o32)
    err = np.abs(o32.cpu().numpy().astype(np.float64) - ref)
    assert np.all(err <= FP32_BOUND * mag + 1e-30), (err / np.maximum(mag, 1e-300)).max()
    # the linearised FP64 product of dg_jvp on the same grid, at the same element-wise bound
    out2 = to_dev(np.zeros_like(z))
    c64 = gpu_context(model, phase)
    c64.jvp(to_dev(z), t, dt, to_dev(v), out2)
    err = np.abs(to_host(out2) - ref)
    assert np.all(err <= 1e-12 * mag + 1e-300), (err / np.maximum(mag, 1e-300)).max()


def test_fp32_product_needs_mixed_context_and_dg0_routes_to_its_product():
    """An FP32 product from an FP64 context (no FP32 copy of z) is an argument error; on a DG0 context
    dg_jvp_fused is the DG0 dual-number product (the batch's DG0 kernels), equal to dg_jvp and to the
    oracle at the FP64 bound."""
    import torch

    from paper_2511_05233_gb300 import dgls

    model, grid, phase, z0, z, v = _case("tradeoff", (6, 4, 3))
    ctx = gpu_context(model, phase)
    v32 = torch.zeros(z.size, dtype=torch.float32, device="cuda")
    with pytest.raises(dgls.DGError) as e:
        ctx.jvp_fused(to_dev(z), 1.5, 1e-3, v32, torch.zeros_like(v32))
    assert e.value.status == dgls.ERR_ARG
    m0, g0, p0, z00, zz0 = make_case("tradeoff", 0, (6, 4, 3))
    v0 = inputs.normal_noise(zz0.size, 7) * (np.abs(zz0) + 1e-3)
    c0 = gpu_context(m0, p0)
    a, b = to_dev(np.zeros_like(zz0)), to_dev(np.zeros_like(zz0))
    c0.jvp_fused(to_dev(zz0), 1.5, 1e-3, to_dev(v0), a)
    c0.jvp(to_dev(zz0), 1.5, 1e-3, to_dev(v0), b)
    ref = newton.jvp(m0, g0, zz0, z00, 1.5, 1e-3, v0)
    mag = newton.abs_jacobian_times(m0, g0, zz0, z00, 1.5, 1e-3, v0)
    for got in (to_host(a), to_host(b)):
        assert np.all(np.abs(got - ref) <= 1e-12 * mag + 1e-300)
