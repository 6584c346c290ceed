"""Full-size parity of the DG1 residual and Jacobian-vector product on the 128^3 workload the bench
times (same structure, state recipe and kernels), on sampled voxels.

The DG operator is local: the residual and the product at a voxel depend only on that voxel and its
six face neighbours, plus boundary terms at x = 0 (collector) and x = nx (anode).  So, for voxels
away from those two faces, the oracle evaluates them on a small crop of the same state around the
voxel and the crop's centre must equal the full-grid result.  The bench uses a perturbed Tab. 6
state (structure seed 3, noise seed 4); the state is built here by the oracle's initialiser on the
CPU, never by the library.
"""
import numpy as np
import pytest

from oracle import chemistry as ch, init, lis, newton
from paper_2511_05233_gb300 import inputs
from tests.gpu_helpers import ensure_built, gpu_context, jvp_magnitude, to_dev, to_host

pytestmark = pytest.mark.gpu

N_SIDE, POROSITY, CORR, STRUCT_SEED, NOISE_SEED, F_C = 128, 0.5, 4.0, 3, 4, 0.5
SAMPLES = 8


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()


def _crop(model, grid, U, k, j, i):
    """Oracle grid and flat state of the crop around voxel (k, j, i): 3 x 3 voxels across, and in x
    one more layer on the -x side, marked as structure so that the crop has a collector face (the
    oracle requires one).  That layer is two voxels from the centre and does not reach it."""
    sl = (slice(k - 1, k + 2), slice(j - 1, j + 2), slice(i - 2, i + 2))
    ph = grid.phase[sl].copy()
    ph[:, :, 0] = lis.STRUCT
    g = lis.Grid(ph, grid.h)
    d = {f: a[(slice(None),) * 3 + sl] for f, a in U.items()}
    return g, lis.pack(model, g, d)


CENTRE = (1, 1, 2)


def _centre(model, g, r):
    """Values of the centre voxel (all nodes, all fields present there) of a crop's flat vector."""
    R = lis.unpack(model, g, r)
    st = g.phase[CENTRE] == lis.STRUCT
    return np.concatenate([R[f][(slice(None),) * 3 + CENTRE].ravel() for f in model.chem.fields
                           if st or not model.chem.is_struct_field(f)])


def test_dg1_128_sampled_residual_and_jvp():
    phase = inputs.make_structure(N_SIDE, POROSITY, CORR, STRUCT_SEED)
    grid = lis.Grid(phase, 1e-6)
    model = lis.Model(ch.tradeoff(), order=1, f_C=F_C, eps_struct=1.0 - POROSITY)
    z0 = init.uniform_state(model, grid, init.equilibrium_fields(model))
    z = init.perturb(model, grid, z0, inputs.uniform_noise(z0.size, NOISE_SEED))
    v = inputs.normal_noise(z0.size, 5) * (np.abs(z) + 1e-3)
    t, dt = 1.5, 1e-3
    ctx = gpu_context(model, phase)
    zd, z0d, vd = to_dev(z), to_dev(z0), to_dev(v)
    r = to_dev(np.zeros_like(z))
    ctx.residual(zd, z0d, t, dt, r)
    jv = to_dev(np.zeros_like(z))
    ctx.jvp(zd, t, dt, vd, jv)
    R, JV = lis.unpack(model, grid, to_host(r)), lis.unpack(model, grid, to_host(jv))
    del r, jv, zd, z0d, vd
    U, U0, Uv = lis.unpack(model, grid, z), lis.unpack(model, grid, z0), lis.unpack(model, grid, v)
    rng = np.random.default_rng(0)
    picks = []
    while len(picks) < SAMPLES:    # interior voxels away from the collector and anode layers
        k, j, i = rng.integers(1, N_SIDE - 1), rng.integers(1, N_SIDE - 1), rng.integers(2, N_SIDE - 3)
        want_struct = len(picks) % 2 == 0
        if (phase[k, j, i] == lis.STRUCT) == want_struct:
            picks.append((k, j, i))
    for k, j, i in picks:
        g, zc = _crop(model, grid, U, k, j, i)
        _, z0c = _crop(model, grid, U0, k, j, i)
        _, vc = _crop(model, grid, Uv, k, j, i)
        st = phase[k, j, i] == lis.STRUCT
        fields = [f for f in model.chem.fields if st or not model.chem.is_struct_field(f)]
        got_r = np.concatenate([R[f][:, :, :, k, j, i].ravel() for f in fields])
        got_jv = np.concatenate([JV[f][:, :, :, k, j, i].ravel() for f in fields])
        ref_r = _centre(model, g, lis.residual(model, g, zc, z0c, t, dt))
        mag_r = _centre(model, g, lis.residual_magnitude(model, g, zc, z0c, t, dt))
        assert np.all(np.abs(got_r - ref_r) <= 1e-12 * mag_r), (k, j, i)
        ref_jv = _centre(model, g, newton.jvp(model, g, zc, z0c, t, dt, vc))
        mag_jv, _ = jvp_magnitude(model, g, zc, z0c, t, dt, vc)
        mag_jv = _centre(model, g, mag_jv)
        assert np.all(np.abs(got_jv - ref_jv) <= 1e-12 * mag_jv + 1e-300), (k, j, i)
