"""Pins of the CPU oracle against what the paper prints and what the mathematics fixes.

None of these tests uses the CUDA library; they check the oracle before it is trusted.
"""
import math

import numpy as np
import pytest

from oracle import appendix, chemistry as ch, constants as K, control, dg, init, lis, newton
from paper_2511_05233_gb300 import inputs


# ------------------------------------------------------------------ Tab. 6 -> Tab. 5.1 / 5.2

def _printed_match(value, printed, digits_unit):
    """|value - printed| within half a unit (one unit) of the last printed digit."""
    return abs(value - printed) <= digits_unit


def test_equilibrium_reproduces_tab52_and_tab51():
    """Tab. 6 evaluated with the parameters of Tab. 5.1/5.2 gives the 'Equi.' columns."""
    e = ch.equilibrium(T=298.15)
    assert _printed_match(e["c_A"], 1499.976, 0.5e-3)
    assert _printed_match(e["c_S_2"], 3.56e-12, 0.5e-14)
    assert _printed_match(e["c_S4_2"], 1.854e-3, 0.5e-6)
    assert _printed_match(e["c_S6_2"], 3.855e-3, 0.5e-6)
    assert _printed_match(e["c_S8_2"], 6.184e-3, 1.0e-6)     # printed 6.184e-3, formula 6.1833e-3
    assert _printed_match(e["c_S8L"], 6.0, 0.05)
    assert _printed_match(e["U5"], 2.313, 0.5e-3)
    assert _printed_match(e["U6"], 2.54, 0.5e-2)


def test_temperature_reading():
    """With T = 298 K (Sec. 2.2 text) the polysulfide column is off by more than 1 %; with
    298.15 K it matches -- the oracle's reading of the temperature."""
    e = ch.equilibrium(T=298.0)
    assert abs(e["c_S8_2"] / 6.184e-3 - 1) > 0.01
    e = ch.equilibrium(T=298.15)
    assert abs(e["c_S8_2"] / 6.184e-3 - 1) < 2e-4


def test_equilibrium_state_has_zero_rates():
    """Sec. 2.8: at the Tab. 6 state every Delta_R G vanishes, so every rate does (to roundoff)."""
    chem = ch.tradeoff()
    e = ch.equilibrium()
    c = {m: np.array(e["c_" + m]) for m in chem.liquid}
    r = ch.rates_mass_action(chem, c, 0.0, e["dPhi0"])
    a = ch.activities(chem, c)
    for rx in chem.reactions:
        ar, ap = ch.net_activities(rx, a)
        if rx.kind == "C":
            scale = ar * math.sqrt(rx.K_sp)
        else:
            scale = ar * math.exp(-K.F * (e["dPhi0"] - rx.U0) / (2 * K.R_GAS * K.T_DEFAULT))
        assert abs(float(r[rx.name])) <= 1e-13 * scale, rx.name


def test_anode_equilibrium():
    """The anode rate vanishes at Phi^L = -RT/F ln(a_Li) (Nernst, Eq. 24 with U0_Ano = 0)."""
    m = lis.Model(ch.tradeoff())
    phiL = -K.R_GAS * m.T / K.F * math.log(1500.0 / 1000.0)
    assert abs(lis.anode_rate(m, 1500.0, phiL)) < 1e-14


# ------------------------------------------------------------------ printed derived numbers

def test_derived_numbers_app_b_and_eq56():
    assert round(K.c_theo_ah_per_kg()) == 1672 or abs(K.c_theo_ah_per_kg() - 1671) < 1.0
    assert abs(K.j_el_from_rate(0.1, 105e-6) - 3.45) < 0.005            # Eq. 56 text
    ratio = math.exp(-K.VISC_EXP * 5581.8)                                # eta(0)/eta(max c_S)
    assert round(ratio, 3) == 0.013
    F_RT = K.F / (K.R_GAS * K.T_DEFAULT)
    l1, l3 = 20e-6, 2e-6
    A1d = F_RT * K.j_el_from_rate(0.1, 105e-6) * l1 / 0.19
    B1d = K.K_C1 * l1 ** 2 / (K.D0["S_2"] * 0.013 * K.C_REF)
    C1d = K.K_E[1] * l1 / (K.D0["S_2"] * 0.013 * K.C_REF)
    assert round(A1d, 3) == 0.014 and round(B1d, 3) == 61.538 and round(C1d, 3) == 0.065
    A3d = F_RT * K.j_el_from_rate(0.5, 105e-6) * l3 / 0.19
    B3d = K.K_C1 * l3 ** 2 / (K.D0["S_2"] * 0.013 * K.C_REF)
    C3d = K.K_E[1] * l3 / (K.D0["S_2"] * 0.013 * K.C_REF)
    assert round(A3d, 3) == 0.007 and round(B3d, 5) == 0.61538 and round(C3d, 4) == 0.0065
    assert round(K.K_C1 * l1 ** 2 / (K.D0["S8_2"] * K.C_REF), 2) == 0.09
    assert round(K.sulfur_loading(105e-6), 2) == 0.02                       # m_A,S8, Sec. 3.2


def test_anion_from_charge_neutrality():
    """Sec. 2.5 (i): c_A = -sum z_j c_j / z_A."""
    e = ch.equilibrium()
    s = sum(K.Z[m] * e["c_" + m] for m in ("Li", "S8L", "S8_2", "S6_2", "S4_2", "S_2"))
    assert abs(e["c_A"] - s) < 1e-12


# ------------------------------------------------------------------ kinetics identities

def test_mass_action_equals_sinh_ln_form():
    """The mass-action rates equal Eqs. 19_simp/21/22/23/24 for positive activities."""
    chem = ch.tradeoff()
    rng = np.random.default_rng(7)
    n = 200
    e = ch.equilibrium()
    c = {m: e["c_" + m] * np.exp(rng.uniform(-2, 2, n)) for m in chem.liquid}
    phiL = rng.uniform(-0.05, 0.05, n)
    phiS = 2.3 + rng.uniform(-0.2, 0.2, n)
    r1 = ch.rates_mass_action(chem, c, phiL, phiS)
    r2 = ch.rates_literal(chem, c, phiL, phiS)
    a = ch.activities(chem, c)
    for rx in chem.reactions:
        ar, ap = ch.net_activities(rx, a)
        if rx.kind == "C":
            scale = ar * math.sqrt(rx.K_sp) + ap / math.sqrt(rx.K_sp)
        else:
            x = K.F * (phiS - phiL - rx.U0) / (2 * K.R_GAS * K.T_DEFAULT)
            scale = ar * np.exp(-x) + ap * np.exp(x)
        assert np.all(np.abs(r1[rx.name] - r2[rx.name]) <= 1e-12 * scale), rx.name


def test_stoichiometry_balances():
    """Tab. 3: sulfur and lithium balance in every reaction; each E reaction moves charge -1
    from the liquid (one e- consumed); chemical reactions are electroneutral per phase."""
    S_atoms = dict(K.SULFUR, S8s=8, Li2Ss=1)
    Li_atoms = {"Li": 1, "Li2Ss": 2}
    for rx in ch.reaction_table():
        assert sum(float(nu) * S_atoms.get(m, 0) for m, nu in rx.nu.items()) == 0, rx.name
        assert sum(float(nu) * Li_atoms.get(m, 0) for m, nu in rx.nu.items()) == 0, rx.name
        q = sum(float(nu) * K.Z.get(m, 0) for m, nu in rx.nu.items())
        assert q == (-1.0 if rx.kind == "E" else 0.0), rx.name


# ------------------------------------------------------------------ generic DG operators

def test_dg_operators_telescope():
    """With v = 1 the interior-face terms cancel and the volume term vanishes (grad 1 = 0):
    the sum over all cells (and nodes) of each operator is zero for any K, psi."""
    rng = np.random.default_rng(3)
    shp = (3, 4, 5)
    Kc = rng.uniform(0.1, 2, shp)
    psi = rng.normal(size=shp)
    assert abs(dg.dg0_faces(Kc, psi, 0.7).sum()) < 1e-12
    shp1 = (2, 2, 2) + shp
    Kn = rng.uniform(0.1, 2, shp1)
    psi1 = rng.normal(size=shp1)
    Kf = {d: (rng.uniform(0.1, 2, dg.trace(Kn, d, 1).shape), rng.uniform(0.1, 2, dg.trace(Kn, d, 1).shape))
          for d in ("x", "y", "z")}
    assert abs(dg.dg1_volume(Kn, psi1, 0.7).sum()) < 1e-12
    assert abs(dg.dg1_faces(Kf, psi1, 0.7).sum()) < 1e-12


def test_dg1_reproduces_linear_fields():
    """A globally linear psi with constant K has zero interior-face and volume residual except
    at the domain boundary (consistency of the IP form): interior cells get exactly 0."""
    shp = (2, 2, 2, 3, 3, 4)
    h = 0.5
    zc, yc, xc, kk, jj, ii = np.meshgrid(*[np.arange(s) for s in shp], indexing="ij")
    s3 = 1.0 / np.sqrt(3.0)
    x = (ii + 0.5 + 0.5 * (2 * xc - 1) * s3) * h
    y = (jj + 0.5 + 0.5 * (2 * yc - 1) * s3) * h
    psi = 2.0 * x - 3.0 * y + 0.25
    Kn = np.full(shp, 1.7)
    Kf = {d: (dg.trace(Kn, d, 1), dg.trace(Kn, d, -1)) for d in ("x", "y", "z")}
    r = dg.dg1_volume(Kn, psi, h) + dg.dg1_faces(Kf, psi, h)
    assert np.abs(r[..., 1:-1, 1:-1, 1:-1]).max() < 1e-12


def test_dg0_is_two_point_flux():
    """Eq. 48 on two cells: A {K}_H (psi_P - psi_Q)/h with the harmonic mean of Eq. 45."""
    h = 2.0
    Kc = np.array([1.0, 3.0]).reshape(1, 1, 2)
    psi = np.array([5.0, 1.0]).reshape(1, 1, 2)
    r = dg.dg0_faces(Kc, psi, h).ravel()
    H = 2 * 1.0 * 3.0 / 4.0
    assert np.allclose(r, [h * h * H * 4.0 / h, -h * h * H * 4.0 / h], rtol=0, atol=1e-13)
    assert dg.harmonic(np.array(2.0), np.array(0.0)) == 0.0      # footnote to Eq. 45


# ------------------------------------------------------------------ App. A

def test_app_a1_dg0_first_order():
    ns = [50, 100, 200]
    e = [appendix.a1_solve(0, n) for n in ns]
    assert 0.85 < appendix.order_fit(ns, e) < 1.2          # App. A1: order ~ 1
    assert e[-1] < 1e-2


def test_app_a1_dg1_converges():
    ns = [25, 50, 100]
    e = [appendix.a1_solve(1, n) for n in ns]
    assert appendix.order_fit(ns, e) > 0.9                   # at least the paper's order 1
    assert e[-1] < e[0]


def test_app_a3_dg0_first_order():
    ns = [10, 20, 40]
    e = [appendix.a3_solve(0, n, t_eval=1.0) for n in ns]
    assert 0.85 < appendix.order_fit(ns, e) < 1.2           # App. A3: DG0 linear


def test_app_a3_dg1_second_order():
    ns = [8, 16, 32]
    e = [appendix.a3_solve(1, n, t_eval=1.0) for n in ns]
    assert 1.8 < appendix.order_fit(ns, e) < 2.3            # App. A3: DG1 quadratic


# ------------------------------------------------------------------ Li-S residual

def _setup(chemname, order, n=(6, 4, 3), seed=1, porosity=0.6, noise_seed=2):
    chem = ch.reduced3() if chemname == "reduced3" else ch.tradeoff()
    ph = inputs.make_structure(n, porosity, 2.0, seed)
    g = lis.Grid(ph, 1e-6)
    m = lis.Model(chem, order=order, f_C=0.5, eps_struct=1 - porosity)
    z0 = init.uniform_state(m, g, init.equilibrium_fields(m))
    N = lis.n_dof(m, g)
    z = init.perturb(m, g, z0, inputs.uniform_noise(N, noise_seed))
    return m, g, z0, z


@pytest.mark.parametrize("chemname,order", [("reduced3", 0), ("tradeoff", 0), ("reduced3", 1), ("tradeoff", 1)])
def test_charge_and_species_ledgers(chemname, order):
    """Summed over the grid, fluxes telescope and reactions cancel:
    sum R_PhiL + sum R_PhiS = anode + collector boundary terms (any state); sum of the sulfur-weighted
    species and solid rows = change of total sulfur / dt; Li rows likewise plus the anode flux."""
    m, g, z0, z = _setup(chemname, order)
    rng = np.random.default_rng(11)
    z = z.copy()
    for f, off, n, st in lis.layout(m, g):
        if f in ("PhiL", "PhiS"):
            z[off:off + n] += rng.uniform(-0.01, 0.01, n)
    dt, t = 1e-3, 2.0
    R = lis.residual(m, g, z, z0, t, dt)
    U = lis.unpack(m, g, R)
    Z = lis.unpack(m, g, z)
    h = g.h
    A = h * h
    if order == 0:
        rA = lis.anode_rate(m, Z["Li"][:, :, -1], Z["PhiL"][:, :, -1])
        bnd_anode = A * K.K_ANO * rA.sum()
        bnd_cc = A * lis.j_el(m, g) * g.ny * g.nz
    else:
        rA = lis.anode_rate(m, dg.trace(Z["Li"], "x", 1)[..., -1], dg.trace(Z["PhiL"], "x", 1)[..., -1])
        bnd_anode = 0.25 * A * K.K_ANO * rA.sum()
        bnd_cc = A * lis.j_el(m, g) * g.ny * g.nz
    qsum = U["PhiL"].sum() + U["PhiS"].sum()
    assert abs(qsum - (K.F * bnd_anode + bnd_cc)) <= 1e-11 * (abs(K.F * bnd_anode) + abs(bnd_cc))
    # sulfur
    mass_now = lis.cell_means(m, g, z)
    mass_old = lis.cell_means(m, g, z0)
    s_rows = sum(K.SULFUR[c] * U[c].sum() for c in m.chem.liquid)
    if "S8s" in m.chem.solid:
        s_rows += 8 * U["eps_S8s"].sum() + U["eps_Li2Ss"].sum()
    ds = (mass_now["sulfur"] - mass_old["sulfur"]) / dt
    scale = sum(K.SULFUR[c] * abs(U[c]).sum() for c in m.chem.liquid) + abs(ds)
    assert abs(s_rows - ds) <= 1e-11 * scale
    li_rows = U["Li"].sum() + (2 * U["eps_Li2Ss"].sum() if "Li2Ss" in m.chem.solid else 0.0)
    dli = (mass_now["lithium"] - mass_old["lithium"]) / dt + bnd_anode
    assert abs(li_rows - dli) <= 1e-11 * (abs(U["Li"]).sum() + abs(dli))


@pytest.mark.parametrize("order", [0, 1])
def test_homogeneous_slab_equals_1d(order):
    """A cathode made entirely of structure with y/z-independent fields reduces to the 1D
    homogenised model cell by cell (Sec. 3.4, eps_struct = 1 recovers the 1D parameters)."""
    chem = ch.tradeoff()
    nx = 8
    p1 = inputs.homogeneous_slab(nx, 1, 1)
    p3 = inputs.homogeneous_slab(nx, 3, 2)
    m = lis.Model(chem, order=order, f_C=0.5, eps_struct=1.0)
    g1, g3 = lis.Grid(p1, 1e-6), lis.Grid(p3, 1e-6)
    rng = np.random.default_rng(5)
    vals = init.equilibrium_fields(m)
    z1 = init.uniform_state(m, g1, vals)
    z1 = z1 * (1 + 0.01 * rng.uniform(-1, 1, z1.size))
    U1 = lis.unpack(m, g1, z1)
    # extrude along y, z (for DG1 the y/z node pairs take the same values)
    U3 = {}
    for f, v in U1.items():
        if order == 0:
            U3[f] = np.broadcast_to(v, (2, 3, nx)).copy()
        else:
            v0 = v[:, :, :, 0, 0, :]                                   # (2,2,2,nx)
            xv = v0[0, 0]                                             # (2, nx): x-nodes
            U3[f] = np.broadcast_to(xv.reshape(1, 1, 2, 1, 1, nx), (2, 2, 2, 2, 3, nx)).copy()
            U1[f] = np.broadcast_to(xv.reshape(1, 1, 2, 1, 1, nx), (2, 2, 2, 1, 1, nx)).copy()
    z1 = lis.pack(m, g1, U1)
    z3 = lis.pack(m, g3, U3)
    zo1 = init.uniform_state(m, g1, vals)
    zo3 = init.uniform_state(m, g3, vals)
    R1 = lis.unpack(m, g1, lis.residual(m, g1, z1, zo1, 2.0, 1e-3))
    R3 = lis.unpack(m, g3, lis.residual(m, g3, z3, zo3, 2.0, 1e-3))
    for f in chem.fields:
        a = R1[f][..., 0, 0, :]
        b = R3[f]
        sc = np.abs(a).max() + 1e-300
        for k in range(2):
            for j in range(3):
                assert np.abs(b[..., k, j, :] - a).max() <= 1e-12 * sc, f


@pytest.mark.parametrize("chemname,order", [("reduced3", 0), ("tradeoff", 0), ("reduced3", 1), ("tradeoff", 1)])
def test_complex_step_jvp_matches_finite_differences(chemname, order):
    m, g, z0, z = _setup(chemname, order)
    v = inputs.normal_noise(z.size, 9) * (np.abs(z) + 1e-3)
    jv = newton.jvp(m, g, z, z0, 1e-3, 1e-3, v)
    eps = 1e-6
    fd = (lis.residual(m, g, z + eps * v, z0, 1e-3, 1e-3) - lis.residual(m, g, z - eps * v, z0, 1e-3, 1e-3)) / (2 * eps)
    assert np.abs(jv - fd).max() <= 1e-7 * np.abs(jv).max()


def test_coloured_jacobian_reproduces_jvp():
    m, g, z0, z = _setup("tradeoff", 0)
    J = newton.assemble_jacobian(m, g, z, z0, 1e-3, 1e-3)
    v = inputs.normal_noise(z.size, 4)
    jv = newton.jvp(m, g, z, z0, 1e-3, 1e-3, v)
    assert np.abs(J @ v - jv).max() <= 1e-13 * np.abs(jv).max()


def test_newton_step_converges_and_conserves():
    """Implicit Euler step (Eq. 50) of the three-species model: converged residual, and the total
    dissolved sulfur changes only by reaction-free transport (E1 conserves sulfur; no boundary flux)."""
    m, g, z0, z = _setup("reduced3", 0, n=(8, 6, 5))
    z1, info = newton.implicit_euler_step(m, g, z, 0.0, 1e-3)
    assert info.converged and info.iterations <= 8
    s0 = lis.cell_means(m, g, z)["sulfur"]
    s1 = lis.cell_means(m, g, z1)["sulfur"]
    assert abs(s1 - s0) <= 1e-9 * abs(s0)


# ------------------------------------------------------------------ controllers

def _scripted(outcomes):
    it = iter(outcomes)

    def step(z, t, dt):
        return next(it), z + dt
    return step


def test_naive_controller_scripted():
    """Fig. 4: three successes grow dt by 1.2; a failure halves it and resets the counter."""
    step = _scripted([True, True, True, True, False, True, True, True, True])
    z, rec = control.naive(step, lambda z: (False, 0.0), 0.0, dt0=1.0, max_steps=8)
    assert rec.dt == pytest.approx([1.0, 1.0, 1.0, 1.2, 0.6, 0.6, 0.6, 0.72])
    assert rec.failures == 1


def test_naive_controller_aborts_after_30_halvings():
    step = _scripted([True] + [False] * 40)
    z, rec = control.naive(step, lambda z: (False, 0.0), 0.0, dt0=1.0, dt_min=1e-30)
    assert rec.status == "aborted" and rec.failures == 31


def test_naive_controller_cutoff_and_cap():
    step = _scripted([True] * 100)
    z, rec = control.naive(step, lambda z: (z > 20.0, -z), 0.0, dt0=1.0, dt_max=1.5)
    assert rec.status == "cutoff" and max(rec.dt) == 1.5


def test_h211b_formulas():
    assert control.h211b_ratio(1e-6, 1e-6, 2.0, 2.0, 1e-6) == pytest.approx(1.0)
    assert control.h211b_ratio(1e-6 / 16, 1e-6, 1.0, 1.0, 1e-6) == pytest.approx(2.0)
    assert control.h211b_limit(1.0) == 1.0
    assert control.h211b_limit(3.0) == pytest.approx(1 + math.atan(2.0))


def test_h211b_controls_error_on_linear_decay():
    """y' = -y with implicit Euler: every accepted step meets err <= 1.02 tol, and Richardson
    extrapolation (Eq. 54) is second order: its error is far below the coarse step's."""
    lam = -1.0

    def step(z, t, dt):
        return True, z / (1 - lam * dt)
    tol = 1e-6
    z, rec = control.h211b(step, lambda z: (False, 0.0), np.array([1.0]), tol, dt0=1e-3, t_end=1.0)
    assert rec.t[-1] >= 1.0
    errs = []
    zz = np.array([1.0])
    for dt in rec.dt:
        zC = zz / (1 - lam * dt)
        zF = zz / (1 - lam * dt / 2) ** 2
        errs.append(control.rel_error(zF, zC))
        zz = 2 * zF - zC
    assert max(errs) <= 1.02 * tol
    assert abs(z[0] - math.exp(-rec.t[-1])) < 1e-4


# ------------------------------------------------------------------ structures

def test_structure_generator():
    ph = inputs.make_structure(32, 0.6, 4.0, 1, clean=False)
    ncat = 32 - inputs.separator_layers(32)
    frac = (ph[:, :, :ncat] == inputs.PORE).mean()
    assert abs(frac - 0.6) < 0.01
    assert np.all(ph[:, :, ncat:] == inputs.SEP)
    ph2 = inputs.make_structure(32, 0.6, 4.0, 1)
    assert np.array_equal(ph2, inputs.make_structure(32, 0.6, 4.0, 1))
    from scipy import ndimage
    lab, n = ndimage.label(ph2 == inputs.STRUCT, structure=ndimage.generate_binary_structure(3, 1))
    assert set(np.unique(lab[:, :, 0])) - {0} == set(range(1, n + 1))


def test_structure_single_cluster_option():
    """single_cluster keeps the largest structure cluster touching the collector and turns every
    other structure voxel to pore (10^3, seed 3 has several clusters on the collector); off by
    default, so the default structures are unchanged."""
    from scipy import ndimage

    six = ndimage.generate_binary_structure(3, 1)
    a = inputs.make_structure(10, 0.5, 4.0, 3)
    b = inputs.make_structure(10, 0.5, 4.0, 3, single_cluster=True)
    lab_a, n_a = ndimage.label(a == inputs.STRUCT, structure=six)
    lab_b, n_b = ndimage.label(b == inputs.STRUCT, structure=six)
    assert n_a > 1 and n_b == 1
    sizes = np.bincount(lab_a.ravel())[1:]
    largest = lab_a == 1 + int(np.argmax(sizes))
    assert np.array_equal(b == inputs.STRUCT, largest)
    assert np.all((a != b) <= ((a == inputs.STRUCT) & (b == inputs.PORE)))
    assert np.array_equal(inputs.make_structure(32, 0.6, 4.0, 1), inputs.make_structure(32, 0.6, 4.0, 1, single_cluster=False))


@pytest.mark.parametrize("level,expect", [(1e-9, True), (1e-6, False)])
def test_newton_stall_rule(monkeypatch, level, expect):
    """A Newton solve that stagnates at a residual floor is converged if the floor is below 1e-8 of
    the initial scaled residual and a failure if it is above.  The floor is planted in the oracle: a
    noise vector of the given size that changes with the state (seeded by its bytes), like rounding,
    and is real, so the complex-step Jacobian does not see it."""
    model, grid, phase, z0, z = _stall_case()
    dt = 1e-3
    R0 = lis.residual(model, grid, z, z, dt, dt)
    S = newton.row_scales(model, grid, dt)
    n0 = np.linalg.norm(S * R0)
    base = lis.residual

    def noisy(m, g, zz, *a, **k):
        r = base(m, g, zz, *a, **k)
        if np.iscomplexobj(zz):
            return r
        e = np.random.default_rng(abs(hash(np.asarray(zz).tobytes())) % (2 ** 32)).normal(size=r.size)
        return r + e * (level * n0 / np.linalg.norm(S * e))

    monkeypatch.setattr(lis, "residual", noisy)
    _, info = newton.newton(model, grid, z, dt, dt)
    assert info.converged is expect
    if not expect:
        assert info.reason in ("line_search", "max_it")


def _stall_case():
    phase = inputs.make_structure((6, 4, 3), 0.6, 2.0, 1)
    for s in range(1, 60):
        phase = inputs.make_structure((6, 4, 3), 0.6, 2.0, s)
        if np.any(phase[:, :, 0] == inputs.STRUCT):
            break
    grid = lis.Grid(phase, 1e-6)
    model = lis.Model(ch.reduced3(), order=0, eps_struct=0.4)
    z0 = init.uniform_state(model, grid, init.equilibrium_fields(model))
    z = init.perturb(model, grid, z0, inputs.uniform_noise(z0.size, 2))
    return model, grid, phase, z0, z
