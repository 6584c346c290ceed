"""GPU parity of the DG1 (Q1 interior-penalty) path against the CPU oracle."""
import numpy as np
import pytest

from oracle import lis, newton
from paper_2511_05233_gb300 import inputs
from tests.gpu_helpers import assert_state_close, ensure_built, gpu_context, jvp_magnitude, make_case, to_dev, to_host

pytestmark = pytest.mark.gpu

CASES = [("reduced3", (7, 5, 4)), ("tradeoff", (7, 5, 4)), ("tradeoff", (10, 6, 5))]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()


@pytest.mark.parametrize("chem,n", CASES)
def test_dg1_residual_parity(chem, n):
    model, grid, phase, z0, z = make_case(chem, 1, n, potential_noise=0.01)
    ctx = gpu_context(model, phase)
    assert ctx.n_dof == z.size
    t, dt = 1.5, 1e-3
    R_or = lis.residual(model, grid, z, z0, t, dt)
    M = lis.residual_magnitude(model, grid, z, z0, t, dt)
    r = to_dev(np.zeros_like(z))
    ctx.residual(to_dev(z), to_dev(z0), t, dt, r)
    err = np.abs(to_host(r) - R_or)
    assert np.all(err <= 1e-12 * M), (err / M).max()


@pytest.mark.parametrize("chem,n", CASES[:2])
def test_dg1_jvp_parity(chem, n):
    model, grid, phase, z0, z = make_case(chem, 1, n, potential_noise=0.01)
    ctx = gpu_context(model, phase)
    t, dt = 1.5, 1e-3
    v = inputs.normal_noise(z.size, 7) * (np.abs(z) + 1e-3)
    ref = newton.jvp(model, grid, z, z0, t, dt, v)
    mag, _ = jvp_magnitude(model, grid, z, z0, t, dt, v)
    out = to_dev(np.zeros_like(z))
    ctx.jvp(to_dev(z), t, dt, to_dev(v), out)
    err = np.abs(to_host(out) - ref)
    assert np.all(err <= 1e-12 * mag + 1e-300), (err / np.maximum(mag, 1e-300)).max()


def test_dg1_point_block_parity():
    """Per-node diagonal blocks of S J (DG1 point-block Jacobi) against the oracle's Jacobian."""
    model, grid, phase, z0, z = make_case("tradeoff", 1, (5, 4, 3), potential_noise=0.01)
    ctx = gpu_context(model, phase)
    t, dt = 1.5, 1e-3
    J = newton.assemble_jacobian(model, grid, z, z0, t, dt).tocsr()
    S = newton.row_scales(model, grid, dt)
    v = inputs.normal_noise(z.size, 3)
    maps, nn = newton._dof_maps(model, grid)
    ref = np.zeros_like(v)
    for node in range(8):
        for cell in range(grid.n_cell):
            idx = [off + node * ln + loc[cell] for (f, off, ln, st, loc) in maps if loc[cell] >= 0]
            B = S[idx, None] * J[idx][:, idx].toarray()
            ref[idx] = np.linalg.solve(B, v[idx])
    out = to_dev(np.zeros_like(z))
    ctx.block_jacobi(to_dev(z), t, dt, to_dev(v), out)
    assert np.abs(to_host(out) - ref).max() <= 1e-9 * np.abs(ref).max()


@pytest.mark.parametrize("reorth", [0, 1, 2])
def test_dg1_step_parity(reorth):
    """One implicit Euler step with each Gram-Schmidt rule in GMRES (second pass when the first
    cancelled, always, never): all reach the oracle's exact-Newton state."""
    model, grid, phase, z0, z = make_case("reduced3", 1, (6, 4, 3))
    ctx = gpu_context(model, phase, reorth=reorth)
    ref, info = newton.implicit_euler_step(model, grid, z, 0.0, 1e-3)
    assert info.converged
    out = to_dev(np.zeros_like(z))
    st, ginfo = ctx.step(to_dev(z), out, 0.0, 1e-3)
    assert ginfo.converged
    assert_state_close(model, grid, to_host(out), ref, 1e-8)
    passes = ctx.reorth_count()
    if reorth == 1:
        assert passes == ginfo.gmres_iterations
    elif reorth == 2:
        assert passes == 0
    else:
        assert 0 <= passes <= ginfo.gmres_iterations


def test_dg1_cell_voltage_and_ledger():
    model, grid, phase, z0, z = make_case("tradeoff", 1, (7, 5, 4))
    ctx = gpu_context(model, phase)
    U = ctx.cell_voltage(to_dev(z))
    assert abs(U - lis.cell_voltage(model, grid, z)) <= 1e-13 * abs(U)
    led = ctx.ledger(to_dev(z))
    mo = lis.cell_means(model, grid, z)
    assert abs(led[0] - mo["sulfur"]) <= 1e-12 * abs(mo["sulfur"])
    assert abs(led[1] - mo["lithium"]) <= 1e-12 * abs(mo["lithium"])


def test_dg1_mixed_precision_step_matches_fp64():
    """The mixed-precision path (FP32 product from the FP32 copy of the linearisation, FP32 Krylov
    basis and blocks, FP64 Newton) reaches the FP64 step's state to 1e-8."""
    from paper_2511_05233_gb300 import dgls

    model, grid, phase, z0, z = make_case("tradeoff", 1, (8, 5, 4), potential_noise=0.01)
    c64 = gpu_context(model, phase)
    c32 = gpu_context(model, phase, precision=dgls.MIXED)
    a, b = to_dev(np.zeros_like(z)), to_dev(np.zeros_like(z))
    _, i64 = c64.step(to_dev(z), a, 0.0, 1e-3)
    _, i32 = c32.step(to_dev(z), b, 0.0, 1e-3)
    assert i64.converged and i32.converged
    assert_state_close(model, grid, to_host(b), to_host(a), 1e-8)


def test_dg1_limiter_parity():
    """dg_limit (vertex-based slope limiter on eps_L c) against the oracle's limiter."""
    from oracle import limiter

    model, grid, phase, z0, _ = make_case("tradeoff", 1, (7, 5, 4))
    z = z0 * (1.0 + 0.4 * inputs.uniform_noise(z0.size, 11))
    ref = limiter.kuzmin_limit(model, grid, z)
    assert not np.array_equal(ref, z)
    ctx = gpu_context(model, phase)
    zd = to_dev(z)
    ctx.limit(zd)
    assert_state_close(model, grid, to_host(zd), ref, 1e-12)


def test_dg1_discharge_with_limiter_matches_oracle():
    """Naive controller with the limiter after every accepted step, against the oracle's controller
    driving oracle steps followed by the oracle's limiter."""
    from oracle import control, limiter
    from paper_2511_05233_gb300 import dgls

    model, grid, phase, z0, _ = make_case("reduced3", 1, (6, 4, 3))

    def step(zz, t, dt):
        z1, info = newton.implicit_euler_step(model, grid, zz, t, dt)
        return info.converged, (limiter.kuzmin_limit(model, grid, z1) if info.converged else z1)

    def cutoff(zz):
        U = lis.cell_voltage(model, grid, zz)
        return U <= 1.9, U

    zf, rec = control.naive(step, cutoff, z0, dt0=1e-3, max_steps=3)
    ctx = gpu_context(model, phase)
    zd = to_dev(z0)
    res = ctx.discharge(zd, controller=dgls.NAIVE, dt0=1e-3, max_steps=3, limiter=True)
    assert res["status"] == "DG_OK"
    assert np.allclose(res["dt"], rec.dt, rtol=1e-14, atol=0)
    assert np.allclose(res["U_cell"], rec.U, rtol=1e-8, atol=0)
    assert_state_close(model, grid, to_host(zd), zf, 1e-8)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_dg1_relaxation_parity(precision):
    """Parabolic relaxation (Sec. 2.8) of a DG1 state, one step of dt = 0.1 s: the relaxation
    form of the linearised products and blocks (FP64, and FP32 inside the mixed Newton iteration).
    (A second step starts almost relaxed and its Newton target sits at the rounding level of the
    scaled residual for this small grid.)"""
    from oracle import init
    from paper_2511_05233_gb300 import dgls

    model, grid, phase, z0, _ = make_case("tradeoff", 1, (6, 4, 3))
    kw = {"precision": dgls.MIXED} if precision == "mixed" else {}
    ctx = gpu_context(model, phase, **kw)
    ref = init.relax(model, grid, z0, dt=0.1, t_init=0.1)
    zd = to_dev(z0)
    ctx.relax(zd, 0.1, 1)
    assert_state_close(model, grid, to_host(zd), ref, 1e-8)


@pytest.mark.parametrize("order,n,n_big", [(1, (6, 4, 3), (12, 10, 8)), (0, (12, 8, 6), (24, 16, 12))])
def test_full_relaxation_converges_and_matches_oracle(order, n, n_big):
    """The initialisation of Sec. 2.8 as the discharge uses it: the first relaxation steps match the
    oracle's, and the full 40 steps of 0.1 s (to 4 s) all converge on a larger grid."""
    from oracle import init

    model, grid, phase, z0, _ = make_case("tradeoff", order, n)
    ctx = gpu_context(model, phase)
    ref = init.relax(model, grid, z0, dt=0.1, t_init=0.3)
    zd = to_dev(z0)
    ctx.relax(zd, 0.1, 3)
    assert_state_close(model, grid, to_host(zd), ref, 1e-8)
    mb, gb, pb, zb0, _ = make_case("tradeoff", order, n_big)
    cb = gpu_context(mb, pb)
    z40 = to_dev(zb0)
    cb.relax(z40, 0.1, 40)                       # raises unless all 40 steps converge
    assert np.all(np.isfinite(to_host(z40)))


def test_dg1_species_coarse_level_step_matches_oracle():
    """A step of dt = 0.1 s from a relaxed state (D dt / h^2 ~ 100: species diffusion reaches far
    past the neighbouring voxels) with the species coarse level on and off: both reach the oracle's
    exact-Newton state; the preconditioner changes the iterations, not the solution."""
    from oracle import init

    model, grid, phase, z0, _ = make_case("tradeoff", 1, (6, 4, 3))
    zr = init.relax(model, grid, z0, dt=0.1, t_init=0.4)
    ref, info = newton.implicit_euler_step(model, grid, zr, 0.4, 0.1)
    assert info.converged
    for sp in (0, 1):
        ctx = gpu_context(model, phase, species_mg=sp)
        zd = to_dev(z0)
        ctx.relax(zd, 0.1, 4)
        out = to_dev(np.zeros_like(z0))
        st, ginfo = ctx.step(zd, out, 0.4, 0.1)
        assert ginfo.converged, sp
        assert_state_close(model, grid, to_host(out), ref, 1e-8)


def test_dg1_species_coarse_level_cuts_gmres_iterations():
    """On a 16^3 synthetic structure, a relaxed state and a step of dt = 0.1 s: the species coarse
    level (applied with the potential one in the multiplicative form) needs at most a third of the
    GMRES iterations of the potential level alone, and both steps reach the same state."""
    from paper_2511_05233_gb300 import dgls

    phase = None
    for s in range(3, 60):
        ph = inputs.make_structure(16, 0.5, 4.0, s)
        if np.any(ph[:, :, 0] == inputs.STRUCT):
            phase = ph
            break
    outs, its = [], []
    for sp in (0, 1):
        prm = dgls.default_params(dgls.TRADEOFF, 1, f_C=0.5, eps_struct=0.5, species_mg=sp)
        ctx = dgls.Context(phase, 1e-6, prm)
        z = ctx.new_state()
        ctx.equilibrium_state(z)
        ctx.relax(z, 0.1, 40)
        out = z.clone()
        st, info = ctx.step(z, out, 4.0, 0.1)
        assert info.converged, sp
        outs.append(out.cpu().numpy())
        its.append(info.gmres_iterations)
        ctx.close()
    assert 3 * its[1] <= its[0], its
    scale = np.abs(outs[0]).max()
    assert np.abs(outs[1] - outs[0]).max() <= 1e-8 * scale
