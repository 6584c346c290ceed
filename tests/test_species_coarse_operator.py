"""The species coarse level of the preconditioner assumes that, with the voxel-constant
prolongation P, P^T J P of a liquid species couples neighbouring voxels only through the
interior-penalty term of Eq. 46 (DG1) or the two-point flux of Eq. 48 (DG0):

    (P^T J P)_{QP} = -(h^2/4)(penalty/h) D_m^0 sum_{4 face points} H(g_P, g_Q)   (DG1)
    (P^T J P)_{QP} = -h D_m^0 H(g_P, g_Q)                                         (DG0)

for face neighbours P, Q, where the volume term and the consistency term vanish on voxel
constants.  On a uniform state the migration and transport-factor derivatives multiply zero
differences, so these are exact there; this test checks them against the oracle's complex-step
Jacobian for a neutral species (S8(L)) and a charged one (Li+), across pore-pore,
pore-structure and structure-structure faces in x and y, and that voxels two apart are not
coupled."""
import numpy as np
import pytest

from oracle import chemistry as ch, constants as K, init, lis, newton

PHASE = np.array([[[1, 0, 0, 1], [1, 1, 0, 0], [1, 0, 1, 1]],
                  [[1, 1, 0, 0], [1, 0, 0, 1], [1, 1, 1, 0]]], dtype=np.uint8)   # (z, y, x)
H = 1e-6


def _g(model, vals, ph):
    eps = {"S8s": vals["eps_S8s"], "Li2Ss": vals["eps_Li2Ss"]}
    epsL = lis.liquid_fraction(model, np.array([ph]), eps)
    return float(ch.transport_factor(epsL, {m: vals[m] for m in model.chem.liquid})[0])


def _harm(a, b):
    return 2.0 * a * b / (a + b)


@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("species", ["S8L", "Li"])
def test_voxel_coupling_of_a_species_is_the_penalty_conductance(order, species):
    model = lis.Model(ch.tradeoff(), order=order, f_C=0.5, eps_struct=0.5)
    grid = lis.Grid(PHASE, H)
    vals = init.equilibrium_fields(model)
    z = init.uniform_state(model, grid, vals)
    t, dt = 1.5, 1e-2
    pairs = [((0, 0, 1), (0, 0, 2)),    # pore - pore, x
             ((0, 0, 2), (0, 0, 3)),    # pore - structure, x
             ((0, 2, 2), (0, 2, 3)),    # structure - structure, x
             ((0, 0, 1), (0, 1, 1)),    # pore - structure, y
             ((1, 2, 0), (1, 2, 1))]    # structure - structure, y
    for P, Q in pairs:
        U = lis.unpack(model, grid, z)
        Uv = {f: np.zeros_like(a) for f, a in U.items()}
        Uv[species][..., P[0], P[1], P[2]] = 1.0
        jv = lis.unpack(model, grid, newton.jvp(model, grid, z, z, t, dt, lis.pack(model, grid, Uv)))[species]
        gP, gQ = _g(model, vals, PHASE[P]), _g(model, vals, PHASE[Q])
        if order == 1:
            want = -(H * H / 4.0) * (model.penalty / H) * K.D0[species] * 4.0 * _harm(gP, gQ)
        else:
            want = -H * K.D0[species] * _harm(gP, gQ)
        got = jv[..., Q[0], Q[1], Q[2]].sum()
        assert abs(got - want) <= 1e-12 * abs(want), (P, Q, got, want)
        # and no coupling to a voxel two faces away (same row, two voxels along x or y)
        far = (Q[0], Q[1], Q[2] + 1) if Q[2] + 1 < PHASE.shape[2] and Q[2] > P[2] else None
        if far is not None:
            assert jv[..., far[0], far[1], far[2]].sum() == 0.0


@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("species", ["S8L", "Li"])
def test_voxel_diagonal_is_node_terms_plus_conductances(order, species):
    """(P^T J P)_{PP} = V (eps_L/dt - dS_m/dc_m) + sum over the face neighbours of the conductance,
    plus, for Li+ in the x = nx layer, the anode exchange derivative (Eq. 27) on that face; the
    source derivative by a complex step of the oracle's point sources."""
    model = lis.Model(ch.tradeoff(), order=order, f_C=0.5, eps_struct=0.5)
    grid = lis.Grid(PHASE, H)
    vals = init.equilibrium_fields(model)
    z = init.uniform_state(model, grid, vals)
    t, dt = 1.5, 1e-2
    V = H ** 3
    nz, ny, nx = PHASE.shape
    for P in [(0, 1, 1), (0, 0, 1), (0, 1, 3), (0, 2, 3), (1, 1, 2)]:
        U = lis.unpack(model, grid, z)
        Uv = {f: np.zeros_like(a) for f, a in U.items()}
        Uv[species][..., P[0], P[1], P[2]] = 1.0
        jv = lis.unpack(model, grid, newton.jvp(model, grid, z, z, t, dt, lis.pack(model, grid, Uv)))[species]
        got = jv[..., P[0], P[1], P[2]].sum()
        ph = PHASE[P]
        eps = {"S8s": vals["eps_S8s"], "Li2Ss": vals["eps_Li2Ss"]}
        epsL = float(lis.liquid_fraction(model, np.array([ph]), eps)[0])
        pt = {f: np.array([complex(v)]) for f, v in vals.items()}
        pt[species] = pt[species] + 1e-30j
        S, _, _ = lis.point_sources(model, np.array([ph]), pt, lis._smooth_factor(model, t))
        want = V * (epsL / dt - S[species][0].imag / 1e-30)
        gP = _g(model, vals, ph)
        for dk, dj, di in ((0, 0, 1), (0, 0, -1), (0, 1, 0), (0, -1, 0), (1, 0, 0), (-1, 0, 0)):
            k, j, i = P[0] + dk, P[1] + dj, P[2] + di
            if 0 <= k < nz and 0 <= j < ny and 0 <= i < nx:
                G = K.D0[species] * _harm(gP, _g(model, vals, PHASE[k, j, i]))
                want += (H * H / 4.0) * (model.penalty / H) * 4.0 * G if order == 1 else H * G
        if species == "Li" and P[2] == nx - 1:
            dr = lis.anode_rate(model, complex(vals["Li"]) + 1e-30j, vals["PhiL"]).imag / 1e-30
            want += H * H * K.K_ANO * dr
        assert abs(got - want) <= 1e-12 * abs(want), (P, got, want)
