"""GPU parity of the DG0 path (libdgls via its C ABI) against the CPU oracle."""
import numpy as np
import pytest

from oracle import init, lis, newton
from paper_2511_05233_gb300 import inputs
from tests.gpu_helpers import assert_state_close, ensure_built, gpu_context, jvp_magnitude, make_case, to_dev, to_host

pytestmark = pytest.mark.gpu

CASES = [("reduced3", (13, 7, 5)), ("tradeoff", (13, 7, 5)), ("tradeoff", (21, 9, 11))]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()


@pytest.mark.parametrize("chem,n", CASES)
def test_dg0_residual_parity(chem, n):
    model, grid, phase, z0, z = make_case(chem, 0, n, potential_noise=0.01)
    ctx = gpu_context(model, phase)
    assert ctx.n_dof == z.size
    t, dt = 1.5, 1e-3
    R_or = lis.residual(model, grid, z, z0, t, dt)
    M = lis.residual_magnitude(model, grid, z, z0, t, dt)
    r = to_dev(np.zeros_like(z))
    ctx.residual(to_dev(z), to_dev(z0), t, dt, r)
    R = to_host(r)
    err = np.abs(R - R_or)
    assert np.all(err <= 1e-12 * M), (err / M).max()


@pytest.mark.parametrize("chem", ["reduced3", "tradeoff"])
def test_dg0_relaxation_parity(chem):
    """Parabolic relaxation (Sec. 2.8): two steps of dt = 0.1 s from the equilibrium state."""
    model, grid, phase, z0, z = make_case(chem, 0, (9, 6, 5))
    ctx = gpu_context(model, phase)
    ref = init.relax(model, grid, z0, dt=0.1, t_init=0.2)
    zd = to_dev(z0)
    ctx.relax(zd, 0.1, 2)
    assert_state_close(model, grid, to_host(zd), ref, 1e-8)


@pytest.mark.parametrize("chem,n", CASES)
def test_dg0_jvp_parity(chem, n):
    model, grid, phase, z0, z = make_case(chem, 0, n, potential_noise=0.01)
    ctx = gpu_context(model, phase)
    t, dt = 1.5, 1e-3
    v = inputs.normal_noise(z.size, 7) * (np.abs(z) + 1e-3)
    ref = newton.jvp(model, grid, z, z0, t, dt, v)
    mag, _ = jvp_magnitude(model, grid, z, z0, t, dt, v)
    out = to_dev(np.zeros_like(z))
    ctx.jvp(to_dev(z), t, dt, to_dev(v), out)
    jv = to_host(out)
    err = np.abs(jv - ref)
    assert np.all(err <= 1e-12 * mag + 1e-300), (err / np.maximum(mag, 1e-300)).max()


def test_dg0_block_jacobi_parity():
    model, grid, phase, z0, z = make_case("tradeoff", 0, (9, 6, 5), potential_noise=0.01)
    ctx = gpu_context(model, phase)
    t, dt = 1.5, 1e-3
    J = newton.assemble_jacobian(model, grid, z, z0, t, dt).tocsr()
    S = newton.row_scales(model, grid, dt)
    v = inputs.normal_noise(z.size, 3)
    # oracle: diagonal blocks of S J per voxel, solved directly
    maps, _ = newton._dof_maps(model, grid)
    ref = np.zeros_like(v)
    for cell in range(grid.n_cell):
        idx = [off + loc[cell] for (f, off, ln, st, loc) in maps if loc[cell] >= 0]
        B = (S[idx, None] * J[idx][:, idx].toarray())
        ref[idx] = np.linalg.solve(B, v[idx])
    out = to_dev(np.zeros_like(z))
    ctx.block_jacobi(to_dev(z), t, dt, to_dev(v), out)
    got = to_host(out)
    assert np.abs(got - ref).max() <= 1e-9 * np.abs(ref).max()


@pytest.mark.parametrize("chem,n", [("reduced3", (10, 6, 5)), ("tradeoff", (9, 5, 4))])
def test_dg0_step_parity(chem, n):
    """One implicit Euler step (Eq. 50), Newton-GMRES on the GPU vs exact Newton in the oracle."""
    model, grid, phase, z0, z = make_case(chem, 0, n)
    ctx = gpu_context(model, phase)
    t, dt = 0.0, 1e-3
    ref, info = newton.implicit_euler_step(model, grid, z, t, dt)
    assert info.converged
    zd = to_dev(z)
    out = to_dev(np.zeros_like(z))
    st, ginfo = ctx.step(zd, out, t, dt)
    assert ginfo.converged
    assert_state_close(model, grid, to_host(out), ref, 1e-8)


def test_dg0_equilibrium_and_voltage():
    model, grid, phase, z0, z = make_case("tradeoff", 0, (9, 6, 5))
    ctx = gpu_context(model, phase)
    zd = ctx.new_state()
    ctx.equilibrium_state(zd)
    got = to_host(zd)
    assert np.allclose(got, z0, rtol=1e-13, atol=0)
    U = ctx.cell_voltage(to_dev(z))
    assert abs(U - lis.cell_voltage(model, grid, z)) <= 1e-13 * abs(U)
    led = ctx.ledger(to_dev(z))
    mo = lis.cell_means(model, grid, z)
    assert abs(led[0] - mo["sulfur"]) <= 1e-12 * abs(mo["sulfur"])
    assert abs(led[1] - mo["lithium"]) <= 1e-12 * abs(mo["lithium"])


def test_dg0_config1_full_size_residual_and_jvp():
    """32^3 DG0 three-species workload (porosity 0.6, correlation length 4, seeds 1/2): residual
    and JVP element by element at the full size."""
    model, grid, phase, z0, z = make_case("reduced3", 0, 32, porosity=0.6, corr=4.0, seed=1, noise_seed=2)
    ctx = gpu_context(model, phase)
    t, dt = 1e-3, 1e-3
    R_or = lis.residual(model, grid, z, z0, t, dt)
    M = lis.residual_magnitude(model, grid, z, z0, t, dt)
    r = to_dev(np.zeros_like(z))
    ctx.residual(to_dev(z), to_dev(z0), t, dt, r)
    assert np.all(np.abs(to_host(r) - R_or) <= 1e-12 * M)
    v = inputs.normal_noise(z.size, 5) * (np.abs(z) + 1e-3)
    ref = newton.jvp(model, grid, z, z0, t, dt, v)
    mag, _ = jvp_magnitude(model, grid, z, z0, t, dt, v)
    out = to_dev(np.zeros_like(z))
    ctx.jvp(to_dev(z), t, dt, to_dev(v), out)
    err = np.abs(to_host(out) - ref)
    assert np.all(err <= 1e-12 * mag + 1e-300), (err / np.maximum(mag, 1e-300)).max()


def test_dg0_mixed_precision_step_matches_fp64():
    from paper_2511_05233_gb300 import dgls

    model, grid, phase, z0, z = make_case("reduced3", 0, (12, 8, 6))
    c64 = gpu_context(model, phase)
    c32 = gpu_context(model, phase, precision=dgls.MIXED)
    a, b = to_dev(np.zeros_like(z)), to_dev(np.zeros_like(z))
    _, i64 = c64.step(to_dev(z), a, 0.0, 1e-3)
    _, i32 = c32.step(to_dev(z), b, 0.0, 1e-3)
    assert i64.converged and i32.converged
    assert_state_close(model, grid, to_host(b), to_host(a), 1e-8)


def test_dg0_large_step_after_relaxation():
    """A step of dt = 0.5 s from a relaxed state (species diffusion D dt / h^2 ~ 500: transport, not
    storage, dominates the species blocks), Newton-GMRES on the GPU against exact Newton in the
    oracle."""
    from oracle import init

    model, grid, phase, z0, _ = make_case("tradeoff", 0, (9, 6, 5))
    zr = init.relax(model, grid, z0, dt=0.1, t_init=0.4)
    ref, info = newton.implicit_euler_step(model, grid, zr, 0.4, 0.5)
    assert info.converged
    ctx = gpu_context(model, phase)
    zd = to_dev(z0)
    ctx.relax(zd, 0.1, 4)
    assert_state_close(model, grid, to_host(zd), zr, 1e-8)
    out = to_dev(np.zeros_like(z0))
    st, ginfo = ctx.step(zd, out, 0.4, 0.5)
    assert ginfo.converged
    assert_state_close(model, grid, to_host(out), ref, 1e-8)
