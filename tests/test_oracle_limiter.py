"""Pins of the oracle's vertex-based DG1 slope limiter (App. B, Kuzmin's rule): conservation,
linear and constant fields kept, no new extrema at the corners, positivity, and a loop version."""
import numpy as np

from oracle import chemistry as ch, dg, init, limiter, lis
from paper_2511_05233_gb300 import inputs


def _q1_of(fun, nz, ny, nx):
    """Nodal values of fun(x, y, z) at the Gauss nodes of a unit-width voxel grid."""
    s = np.array([-1.0, 1.0]) / (2.0 * np.sqrt(3.0))
    q = np.zeros((2, 2, 2, nz, ny, nx))
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    for az in (0, 1):
        for ay in (0, 1):
            for ax in (0, 1):
                q[az, ay, ax] = fun(i + 0.5 + s[ax], j + 0.5 + s[ay], k + 0.5 + s[az])
    return q


def _case(n=(6, 4, 3), seed=1):
    chem = ch.tradeoff()
    for s in range(seed, seed + 50):
        phase = inputs.make_structure(n, 0.5, 2.0, s)
        if np.any(phase[:, :, 0] == inputs.STRUCT):
            break
    grid = lis.Grid(phase, 1e-6)
    model = lis.Model(chem, order=1, eps_struct=0.5)
    z0 = init.uniform_state(model, grid, init.equilibrium_fields(model))
    return model, grid, z0


def test_loop_version_agrees():
    rng = np.random.default_rng(0)
    q = rng.normal(size=(2, 2, 2, 3, 4, 5)) + 2.0
    got, _ = limiter.limit_field(q)
    assert np.allclose(got, limiter.limit_field_loops(q), rtol=0, atol=1e-13)


def test_constant_and_linear_fields_are_kept():
    nz, ny, nx = 5, 6, 7
    c = np.full((2, 2, 2, nz, ny, nx), 3.25)
    assert np.array_equal(limiter.limit_field(c)[0], c)
    q = _q1_of(lambda x, y, z: 1.0 + 0.3 * x - 0.2 * y + 0.1 * z, nz, ny, nx)
    got, alpha = limiter.limit_field(q)
    inner = (slice(1, -1),) * 3           # voxels whose corners all have a full ring of neighbours
    assert np.allclose(alpha[inner], 1.0)
    assert np.allclose(got[(slice(None),) * 3 + inner], q[(slice(None),) * 3 + inner], rtol=0, atol=1e-13)


def test_corner_values_bounded_and_positive():
    rng = np.random.default_rng(1)
    nz, ny, nx = 4, 5, 6
    mean = rng.uniform(0.1, 1.0, size=(nz, ny, nx))
    q = mean[None, None, None] + rng.normal(scale=2.0, size=(2, 2, 2, nz, ny, nx))
    q -= q.mean(axis=(0, 1, 2)) - mean                 # keep the chosen means, strong oscillations
    got, _ = limiter.limit_field(q)
    assert np.allclose(got.mean(axis=(0, 1, 2)), mean, rtol=1e-14)
    vmax, vmin = limiter.vertex_bounds(mean)
    uc = limiter.corner_values(got)
    for cz in (0, 1):
        for cy in (0, 1):
            for cx in (0, 1):
                hi = vmax[cz:cz + nz, cy:cy + ny, cx:cx + nx]
                lo = vmin[cz:cz + nz, cy:cy + ny, cx:cx + nx]
                assert np.all(uc[cz, cy, cx] <= hi + 1e-12) and np.all(uc[cz, cy, cx] >= lo - 1e-12)
    assert got.min() >= -1e-12                          # positive means -> non-negative nodes
    assert q.min() < 0                                  # the input did undershoot


def test_state_limiter_conserves_every_species():
    model, grid, z0 = _case()
    rng = np.random.default_rng(2)
    z = z0 * (1.0 + 0.4 * rng.uniform(-1, 1, size=z0.size))
    zl = limiter.kuzmin_limit(model, grid, z)
    U, Ul = lis.unpack(model, grid, z), lis.unpack(model, grid, zl)
    eL = limiter.node_liquid_fraction(model, grid, U)
    for f in model.chem.liquid:
        before = (eL * U[f]).sum(axis=(0, 1, 2))
        after = (eL * Ul[f]).sum(axis=(0, 1, 2))
        assert np.allclose(after, before, rtol=1e-13, atol=0)
    for f in ("eps_S8s", "eps_Li2Ss", "PhiL", "PhiS"):
        assert np.array_equal(Ul[f], U[f])
    assert not np.array_equal(zl, z)                     # something was limited


def test_trace_weights_match_corner_extrapolation():
    q = _q1_of(lambda x, y, z: 2.0 * x * y * z + x, 2, 2, 2)
    uc = limiter.corner_values(q)
    # the corner (1,1,1) of voxel (0,0,0) is the point (1,1,1)
    assert abs(uc[1, 1, 1, 0, 0, 0] - 3.0) < 1e-12
    # a corner is the x = +1 face trace, extrapolated again along y and z with the same weights
    tx = dg.trace(q, "x", +1)                               # (2 z-nodes, 2 y-nodes, cells)
    corner = dg.ALPHA * (dg.ALPHA * tx[1, 1] + dg.BETA * tx[1, 0]) + dg.BETA * (dg.ALPHA * tx[0, 1] + dg.BETA * tx[0, 0])
    assert np.allclose(corner, uc[1, 1, 1], rtol=1e-14)
