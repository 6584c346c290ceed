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
    """Oracle model, grid and flat-state packer for the crop around voxel (k, j, i), and the centre's
    index in the crop.  The crop is 3 x 3 voxels across; along x it keeps two layers on each side
    where the grid has them.  The oracle requires a collector face, so an interior crop's first
    layer is marked as structure (two voxels from the centre, out of its reach).  A crop at the real
    collector (i = 0) keeps the real collector face: its model takes the collector current density
    per structure face of the full grid (Eq. 25 with reading 5's rescaling), j_el adjusted for the
    crop's face count.  A crop at the anode (i = nx - 1) keeps the real anode face (Eqs. 26-27)."""
    from dataclasses import replace

    nx = grid.nx
    if i == 0:
        xs = slice(0, 3)
        centre = (1, 1, 0)
    elif i == nx - 1:
        xs = slice(nx - 4, nx)
        centre = (1, 1, 3)
    else:
        xs = slice(i - 2, i + 2)
        centre = (1, 1, 2)
    sl = (slice(k - 1, k + 2), slice(j - 1, j + 2), xs)
    ph = grid.phase[sl].copy()
    if i != 0:
        ph[:, :, 0] = lis.STRUCT
    g = lis.Grid(ph, grid.h)
    m = model
    if i == 0:
        j_face = lis.j_el(model, grid) * grid.ny * grid.nz / grid.n_cc
        m = replace(model, j_el=j_face * g.n_cc / (g.ny * g.nz))

    def pack(Uf):
        d = {f: a[(slice(None),) * 3 + sl] for f, a in Uf.items()}
        return lis.pack(m, g, d)
    return m, g, pack, centre


def _centre(model, g, r, centre):
    """Values of the centre voxel (all nodes, all fields present there) of a crop's flat vector."""
    R = lis.unpack(model, g, r)
    st = g.phase[centre] == lis.STRUCT
    return np.concatenate([R[f][(slice(None),) * 3 + centre].ravel() for f in model.chem.fields
                           if st or not model.chem.is_struct_field(f)])


def test_dg1_128_sampled_residual_and_jvp():
    """Interior voxels (structure and pore), collector-face structure voxels (x = 0) and anode-face
    voxels (x = nx - 1): residual (1e-12 of the terms' size), the FP64 product of dg_jvp and of the
    fused kernel (1e-12 |J||v|), and the fused FP32 product of the mixed-precision Krylov loop
    (2e-5 |J||v|, the bound derived in test_gpu_fused_jvp)."""
    import torch

    from paper_2511_05233_gb300 import dgls

    phase = inputs.make_structure(N_SIDE, POROSITY, CORR, STRUCT_SEED)
    grid = lis.Grid(phase, 1e-6)
    model = lis.Model(ch.tradeoff(), order=1, f_C=F_C, eps_struct=1.0 - POROSITY)
    z0 = init.uniform_state(model, grid, init.equilibrium_fields(model))
    z = init.perturb(model, grid, z0, inputs.uniform_noise(z0.size, NOISE_SEED))
    v = inputs.normal_noise(z0.size, 5) * (np.abs(z) + 1e-3)
    t, dt = 1.5, 1e-3
    ctx = gpu_context(model, phase)                  # FP64: linearised dg_jvp and the fused FP64 kernel
    zd, z0d, vd = to_dev(z), to_dev(z0), to_dev(v)
    r = to_dev(np.zeros_like(z))
    ctx.residual(zd, z0d, t, dt, r)
    R = lis.unpack(model, grid, to_host(r))
    ctx.jvp(zd, t, dt, vd, r)
    JV = lis.unpack(model, grid, to_host(r))
    ctx.jvp_fused(zd, t, dt, vd, r)
    JF = lis.unpack(model, grid, to_host(r))
    del r
    ctx.close()
    ctx = gpu_context(model, phase, precision=dgls.MIXED)   # the FP32 product of the mixed Krylov loop
    v32 = vd.float()
    o32 = torch.empty_like(v32)
    ctx.jvp_fused(zd, t, dt, v32, o32)
    J32 = lis.unpack(model, grid, o32.double().cpu().numpy())
    ctx.close()
    del v32, o32, zd, z0d, vd
    U, U0, Uv = lis.unpack(model, grid, z), lis.unpack(model, grid, z0), lis.unpack(model, grid, v)
    rng = np.random.default_rng(0)
    picks = []
    while len(picks) < SAMPLES:    # interior voxels away from the collector and anode layers
        k, j, i = rng.integers(1, N_SIDE - 1), rng.integers(1, N_SIDE - 1), rng.integers(2, N_SIDE - 3)
        want_struct = len(picks) % 2 == 0
        if (phase[k, j, i] == lis.STRUCT) == want_struct:
            picks.append((k, j, i))
    cc = 0
    while cc < 3:                  # structure voxels on the collector face
        k, j = rng.integers(1, N_SIDE - 1), rng.integers(1, N_SIDE - 1)
        if phase[k, j, 0] == lis.STRUCT:
            picks.append((k, j, 0))
            cc += 1
    for _ in range(3):             # anode-face voxels (separator)
        picks.append((rng.integers(1, N_SIDE - 1), rng.integers(1, N_SIDE - 1), N_SIDE - 1))
    for k, j, i in picks:
        m, g, pack, centre = _crop(model, grid, U, k, j, i)
        zc, z0c, vc = pack(U), pack(U0), pack(Uv)
        st = phase[k, j, i] == lis.STRUCT
        fields = [f for f in model.chem.fields if st or not model.chem.is_struct_field(f)]
        pick = lambda A: np.concatenate([A[f][:, :, :, k, j, i].ravel() for f in fields])  # noqa: E731
        ref_r = _centre(m, g, lis.residual(m, g, zc, z0c, t, dt), centre)
        mag_r = _centre(m, g, lis.residual_magnitude(m, g, zc, z0c, t, dt), centre)
        assert np.all(np.abs(pick(R) - ref_r) <= 1e-12 * mag_r), (k, j, i)
        ref_jv = _centre(m, g, newton.jvp(m, g, zc, z0c, t, dt, vc), centre)
        mag_jv, _ = jvp_magnitude(m, g, zc, z0c, t, dt, vc)
        mag_jv = _centre(m, g, mag_jv, centre)
        assert np.all(np.abs(pick(JV) - ref_jv) <= 1e-12 * mag_jv + 1e-300), (k, j, i)
        assert np.all(np.abs(pick(JF) - ref_jv) <= 1e-12 * mag_jv + 1e-300), (k, j, i)
        assert np.all(np.abs(pick(J32) - ref_jv) <= 2e-5 * mag_jv + 1e-30), (k, j, i)
