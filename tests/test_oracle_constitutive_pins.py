"""Pins of the oracle's constitutive laws, transport coefficients, cell voltage and parabolic
relaxation against values the paper prints, closed forms and physical laws.

Each test calls the oracle function itself and fails on a plausible mistake in it: a wrong
exponent, sign, factor, species weight or localisation.  No CUDA code is used.
"""
import numpy as np
import pytest

from oracle import chemistry as ch, constants as K, init, lis

LIQ = ["Li", "S8L", "S8_2", "S6_2", "S4_2", "S_2"]


# ------------------------------------------------------------------ Eqs. 2-3 and Eq. 18 (final)

@pytest.mark.parametrize("species,weight", [("S8L", 8), ("S8_2", 8), ("S6_2", 6), ("S4_2", 4), ("S_2", 1)])
def test_transport_factor_viscosity_ratio_printed(species, weight):
    """Sec. 3.1 (text after Eq. 56) prints eta(0)/eta(max c_S) = 0.013 at c_S = 5581.8 mol/m^3.
    Pure electrolyte (eps_L = 1, Bruggeman factor 1) with all dissolved sulfur carried by one
    species at the weight of the c_S definition in Sec. 2.2 must give that ratio."""
    c = {m: 0.0 for m in LIQ}
    c[species] = 5581.8 / weight
    g = float(ch.transport_factor(1.0, c))
    assert abs(g - 0.013) <= 0.5e-3            # printed to 3 decimals
    assert abs(g - 0.013148) <= 1e-6           # exp(-7.76e-4 * 5581.8), Eq. 2 ratio


def test_transport_factor_lithium_carries_no_sulfur():
    """Li+ is not in c_S (Sec. 2.2): any Li+ concentration leaves the viscosity at eta(0)."""
    c = {m: 0.0 for m in LIQ}
    c["Li"] = 1500.0
    assert float(ch.transport_factor(1.0, c)) == 1.0


@pytest.mark.parametrize("eps", [0.04, 0.25, 0.6, 0.9])
def test_transport_factor_bruggeman_scaling(eps):
    """Eq. 18 (final): D_eff = (eps_L / tau) D with tau = eps_L^{-1/2} (Sec. 2.3).  At fixed c_S the
    factor relative to pure electrolyte is eps / eps^{-1/2}; 0.25 gives exactly 1/8."""
    rng = np.random.default_rng(3)
    c = {m: float(v) for m, v in zip(LIQ, rng.uniform(0.0, 50.0, 6))}
    ratio = float(ch.transport_factor(eps, c) / ch.transport_factor(1.0, c))
    tau = eps ** -0.5
    assert abs(ratio - eps / tau) <= 1e-15
    if eps == 0.25:
        assert ratio == 0.125


def test_transport_factor_clips_negative_liquid_fraction():
    """Reading 9: a non-positive liquid fraction transports nothing."""
    assert float(ch.transport_factor(-0.1, {"Li": 1000.0})) == 0.0


# ------------------------------------------------------------------ Eq. 18 with Eq. 57

def test_specific_surface_initial_state_hand_value():
    """Eq. 18 at the initial fractions of Tab. 5.1 (eps_S8,0 = 0.095, eps_Li2S,0 = 2.77e-6,
    a_V,0 = 94.908e6 1/m, a = 0.1392, b = 3.310 h) at f_C = 0.5 1/h, 1D (eps_struct = 1):
    a_V0 (1 - (1/1.2)^{3/2} - (2.77e-6 / (0.1392 e^{-3.310 * 0.5}))^{3/2})."""
    t1 = (1.0 / 1.2) ** 1.5
    t2 = (2.77e-6 / (0.1392 * np.exp(-3.310 * 0.5))) ** 1.5
    expect = 94.908e6 * (1.0 - t1 - t2)
    got = float(ch.specific_surface(0.095, 2.77e-6, 0.5, 1.0))
    assert abs(got / expect - 1.0) <= 1e-14
    assert abs(got - 2.2708937e7) <= 1.0       # the same number written out


@pytest.mark.parametrize("eps_struct", [1.0, 0.413, 0.5])
def test_specific_surface_localisation_eq57(eps_struct):
    """Eq. 57 divides a_V,0 and both reference fractions by eps_struct: with the volume fractions
    localised the same way, eps_struct a_V equals the 1D value for any fractions."""
    rng = np.random.default_rng(5)
    for _ in range(20):
        e8 = rng.uniform(0.0, 1.2 * 0.095)
        e2 = rng.uniform(0.0, 0.02)
        fC = rng.uniform(0.05, 2.0)
        one_d = float(ch.specific_surface(e8, e2, fC, 1.0))
        three_d = float(ch.specific_surface(e8 / eps_struct, e2 / eps_struct, fC, eps_struct))
        assert abs(eps_struct * three_d - one_d) <= 1e-14 * 94.908e6


@pytest.mark.parametrize("f_C", [0.05, 0.5, 2.0])
def test_specific_surface_zeros(f_C):
    """a_V vanishes when sulfur has grown to 1.2 eps_S8,0 (S8 term = 1) and when Li2S has reached
    a e^{-b f_C} (Li2S term = 1); beyond, it is clipped at zero (reading 10).  The Li2S zero moves
    with f_C as e^{-b f_C}, so a wrong sign or unit of b misses it."""
    assert float(ch.specific_surface(1.2 * 0.095, 0.0, f_C, 1.0)) == 0.0
    e_li2s = 0.1392 * np.exp(-3.310 * f_C)
    assert abs(float(ch.specific_surface(0.0, e_li2s, f_C, 1.0))) <= 1e-9 * 94.908e6
    assert float(ch.specific_surface(0.0, 0.5 * e_li2s, f_C, 1.0)) > 0.0
    assert float(ch.specific_surface(0.0, 1.5 * e_li2s, f_C, 1.0)) == 0.0


def test_specific_surface_three_halves_power():
    """With Li2S absent, a_V / a_V,0 = 1 - x^{3/2} for x = eps_S8 / (1.2 eps_S8,0)."""
    for x in (0.1, 0.3, 0.64, 0.9):
        got = float(ch.specific_surface(x * 1.2 * 0.095, 0.0, 0.5, 1.0)) / 94.908e6
        assert abs(got - (1.0 - x * np.sqrt(x))) <= 1e-15


# ------------------------------------------------------------------ Tab. 4 rows 1-2, Eq. 5

def _random_point(seed):
    rng = np.random.default_rng(seed)
    U = {m: np.array([rng.uniform(1e-3, 200.0)]) for m in LIQ}
    U["Li"] = np.array([1500.0 * rng.uniform(0.9, 1.1)])
    U["eps_S8s"] = np.array([rng.uniform(0.0, 0.2)])
    U["eps_Li2Ss"] = np.array([rng.uniform(0.0, 0.05)])
    U["PhiL"] = np.array([0.0])
    U["PhiS"] = np.array([2.3])
    return U


@pytest.mark.parametrize("phase", [lis.PORE, lis.STRUCT, lis.SEP])
def test_charge_migration_coefficient_is_kappa_L(phase):
    """Tab. 4 row 2 eliminates the anion by charge neutrality (Sec. 2.5 (i)).  Its Phi^L
    coefficient summed over the transported species must then equal the conductivity of Eq. 5,
    sum over ALL species including the anion of z_j^2 F^2/(RT) D_j^eff c_j, with
    c_A = -sum_j z_j c_j / z_A."""
    model = lis.Model(ch.tradeoff(), order=0, eps_struct=0.4)
    for seed in range(5):
        U = _random_point(seed)
        ph = np.array([phase])
        terms, epsL = lis.coefficients(model, ph, U)
        got = sum(np.real(k) for k, f in terms["PhiL"] if f == "PhiL")
        cS = 8 * U["S8L"] + 8 * U["S8_2"] + 6 * U["S6_2"] + 4 * U["S4_2"] + U["S_2"]
        g = np.maximum(epsL, 0.0) ** 1.5 * np.exp(-7.76e-4 * cS)
        z = {"Li": 1, "S8L": 0, "S8_2": -2, "S6_2": -2, "S4_2": -2, "S_2": -2, "A": -1}
        D0 = {"Li": 9.3e-10, "S8L": 10.0e-10, "S8_2": 5.3e-10, "S6_2": 5.3e-10, "S4_2": 7.6e-10, "S_2": 0.6e-10,
              "A": 9.3e-10}
        c = {m: U[m] for m in LIQ}
        c["A"] = -sum(z[m] * c[m] for m in LIQ) / z["A"]
        F, RT = 96485.332, 8.3145 * 298.15
        kappa_L = sum(z[m] ** 2 * F ** 2 / RT * D0[m] * g * c[m] for m in c)
        assert np.allclose(got, kappa_L, rtol=1e-13, atol=0.0)


def test_charge_diffusion_coefficients_follow_neutrality():
    """Tab. 4 row 2, diffusion part: for any concentration gradients that keep charge neutrality,
    sum_j K^d_j grad c_j equals the full charge-diffusion flux sum over all species (anion
    included) of z_j F D_j^eff grad c_j of Eq. 4.  K^d of Li+ vanishes because D_Li = D_A
    (Tab. 5.2), and S8(L) carries no charge."""
    model = lis.Model(ch.tradeoff(), order=0, eps_struct=0.4)
    U = _random_point(11)
    terms, epsL = lis.coefficients(model, np.array([lis.STRUCT]), U)
    Kd = {f: np.real(k) for k, f in terms["PhiL"] if f != "PhiL"}
    assert float(Kd["Li"][0]) == 0.0
    assert float(Kd["S8L"][0]) == 0.0
    rng = np.random.default_rng(12)
    z = {"Li": 1, "S8L": 0, "S8_2": -2, "S6_2": -2, "S4_2": -2, "S_2": -2}
    D0 = {"Li": 9.3e-10, "S8L": 10.0e-10, "S8_2": 5.3e-10, "S6_2": 5.3e-10, "S4_2": 7.6e-10, "S_2": 0.6e-10}
    cS = 8 * U["S8L"] + 8 * U["S8_2"] + 6 * U["S6_2"] + 4 * U["S4_2"] + U["S_2"]
    g = np.maximum(epsL, 0.0) ** 1.5 * np.exp(-7.76e-4 * cS)
    F = 96485.332
    for _ in range(5):
        grad = {m: rng.normal() for m in LIQ}
        grad_A = sum(z[m] * grad[m] for m in LIQ)            # z_A = -1: grad c_A = sum z_j grad c_j
        full = sum(z[m] * F * D0[m] * g * grad[m] for m in LIQ) + (-1) * F * 9.3e-10 * g * grad_A
        got = sum(Kd[m] * grad[m] for m in LIQ)
        assert np.allclose(got, full, rtol=1e-12, atol=1e-30)


@pytest.mark.parametrize("species", LIQ)
def test_species_flux_vanishes_for_boltzmann_profile(species):
    """Eq. 1 / Tab. 4 row 1: the Nernst-Planck flux D grad c + (z F/RT) D c grad Phi is zero for
    a Boltzmann profile, grad c = -(z F/RT) c grad Phi (any D).  So the coefficient pair the
    oracle returns must satisfy D (-(z F/RT) c) + sigma = 0 -- a wrong sign or a missing c or z
    in sigma breaks it."""
    model = lis.Model(ch.tradeoff(), order=0, eps_struct=0.4)
    U = _random_point(21)
    terms, _ = lis.coefficients(model, np.array([lis.STRUCT]), U)
    (D, f1), (sig, f2) = terms[species]
    assert f1 == species and f2 == "PhiL"
    zc = {"Li": 1, "S8L": 0, "S8_2": -2, "S6_2": -2, "S4_2": -2, "S_2": -2}[species]
    F_RT = 96485.332 / (8.3145 * 298.15)
    grad_phi = 0.37
    flux = D * (-zc * F_RT * U[species] * grad_phi) + sig * grad_phi
    assert abs(float(flux[0])) <= 1e-13 * abs(float(D[0] * U[species][0] * F_RT * grad_phi)) + 1e-300
    assert float(D[0]) > 0.0


def test_solid_conductivity_only_in_structure():
    """Tab. 4 row 4: kappa_S^eff = 1 S/m (Tab. 5.1) in the structure; no solid conduction in
    pores and separator (Sec. 2.5 footnote, Sec. 2.1)."""
    model = lis.Model(ch.tradeoff(), order=0, eps_struct=0.4)
    U = _random_point(31)
    for ph, expect in ((lis.STRUCT, 1.0), (lis.PORE, 0.0), (lis.SEP, 0.0)):
        terms, _ = lis.coefficients(model, np.array([ph]), U)
        assert float(np.real(terms["PhiS"][0][0][0])) == expect


# ------------------------------------------------------------------ Eq. A1

def _case(order, n=(6, 4, 3)):
    from tests.gpu_helpers import structure_with_collector

    phase = structure_with_collector(n, 0.6, 2.0, 1)
    grid = lis.Grid(phase, 1e-6)
    model = lis.Model(ch.tradeoff(), order=order, f_C=0.5, eps_struct=0.4)
    return model, grid


@pytest.mark.parametrize("order", [0, 1])
def test_cell_voltage_of_uniform_state_is_delta_phi0(order):
    """Eq. A1 on the Tab. 6 state (Phi^S = Delta Phi_0 everywhere, Phi^L = 0): U_cell is the
    equilibrium potential of E1 at the Tab. 6 concentrations, U0_1 - (RT/F) ln((a_S8^2-)^{1/2} /
    (a_S8(L))^{1/2}) (Eq. 24 with Delta G_E1 = 0, U0_1 = 2.41 V of Tab. 5.1)."""
    model, grid = _case(order)
    z0 = init.uniform_state(model, grid, init.equilibrium_fields(model))
    U = lis.cell_voltage(model, grid, z0)
    e = ch.equilibrium(298.15)
    nernst = 2.41 - 8.3145 * 298.15 / 96485.332 * np.log(np.sqrt(e["c_S8_2"] / 1000.0) / np.sqrt(e["c_S8L"] / 1000.0))
    assert abs(U - nernst) <= 1e-14


@pytest.mark.parametrize("order", [0, 1])
def test_cell_voltage_is_area_mean_over_collector_structure_faces(order):
    """Eq. A1 is a surface average over the collector (the structure faces at x = 0, reading 5).
    With Phi^S = a(y, z) + b x, linear inside every voxel, the face value at x = 0 is a(y, z)
    (DG1 traces are exact for linear fields; DG0 takes the adjacent cell value, reading 4, which
    is a + b h/2 at the cell centre).  The mean runs over collector faces only, each weighted by
    its area -- never over voxels behind it or the pore faces."""
    model, grid = _case(order)
    z0 = init.uniform_state(model, grid, init.equilibrium_fields(model))
    U = lis.unpack(model, grid, z0)
    rng = np.random.default_rng(8)
    a = rng.uniform(2.0, 2.5, (grid.nz, grid.ny))
    b = 1e3                                              # V/m
    h = grid.h
    xc = (np.arange(grid.nx) + 0.5) * h
    if order == 0:
        U["PhiS"] = a[:, :, None] + b * xc[None, None, :]
        expect = float(np.mean(a[grid.cc] + b * h / 2))
    else:
        gx = np.array([-1.0, 1.0]) / np.sqrt(3.0) * (h / 2)     # Gauss nodes about the centre
        phi = np.empty((2, 2, 2, grid.nz, grid.ny, grid.nx))
        for ix in range(2):
            phi[:, :, ix] = a[None, None, :, :, None] + b * (xc[None, None, None, None, :] + gx[ix])
        U["PhiS"] = phi
        expect = float(np.mean(a[grid.cc]))
    z = lis.pack(model, grid, U)
    got = lis.cell_voltage(model, grid, z)
    assert abs(got - expect) <= 1e-14 * 2.5
    # not a volume mean, not a mean over all faces at x = 0
    assert abs(got - float(np.mean(a))) > 1e-6 or np.all(grid.cc)


# ------------------------------------------------------------------ Sec. 2.8 (Eq. 56)

def _reaction_current(model, grid, z, t):
    """F int a_V sum_E k_E r_E dV over the structure (the electrons the cathode reactions take
    up), evaluated here point by point from the rates."""
    U = lis.unpack(model, grid, z)
    eps = lis._solid_fractions(model, U)
    aV = ch.specific_surface(eps["S8s"], eps["Li2Ss"], model.f_C, model.eps_struct)
    r = ch.rates_mass_action(model.chem, {m: U[m] for m in model.chem.liquid}, U["PhiL"], U["PhiS"], model.T)
    tH = K.smooth_step(t)
    erate = sum(rx.k * r[rx.name] * (tH if rx.smooth else 1.0) for rx in model.chem.reactions if rx.kind == "E")
    Mw = grid.h ** 3 if model.order == 0 else grid.h ** 3 / 8
    st = np.broadcast_to(grid.struct, U["PhiL"].shape)
    return 96485.332 * float(np.sum(Mw * np.where(st, aV * erate, 0.0)))


def test_relaxation_reaches_current_balance_and_freezes_concentrations():
    """The parabolic relaxation of Sec. 2.8 (Delta t = 0.1 s to T_init = 4 s, current ramped by
    T_H of Eq. 56) must end in the steady state of the potential equations: the reaction current
    F int a_V sum k_E r_E equals the applied current j_el A_yz T_H(4 s) (the solid charge
    equation of Tab. 4 integrated over the cathode, no-flux elsewhere), the anode exchange
    current F k_Ano int r_Ano returns the same current through the liquid, and concentrations
    and solid fractions stay at their initial values (they are frozen)."""
    model, grid = _case(0, n=(6, 6, 6))
    z0 = init.uniform_state(model, grid, init.equilibrium_fields(model))
    z = init.relax(model, grid, z0, dt=0.1, t_init=4.0)
    I_app = lis.j_el(model, grid) * grid.ny * grid.nz * grid.h ** 2 * K.smooth_step(4.0)
    I_react = _reaction_current(model, grid, z, 4.0)
    assert abs(I_react / I_app - 1.0) <= 1e-7
    U = lis.unpack(model, grid, z)
    rA = lis.anode_rate(model, U["Li"][:, :, -1], U["PhiL"][:, :, -1])
    I_ano = 96485.332 * 5.0e-3 * float(np.sum(rA)) * grid.h ** 2
    assert abs(I_ano / I_app + 1.0) <= 1e-7              # Li+ + e- -> Li at the anode: rate < 0
    # frozen up to the rounding of 40 Newton updates of the coupled system, measured against the
    # scale of each kind of unknown (Newton's species rows are scaled by c_ref, so a trace species
    # moves by rounding relative to the largest concentration, not to itself)
    lay = lis.layout(model, grid)
    conc = max(np.abs(z0[off:off + n]).max() for f, off, n, st in lay if f in model.chem.liquid)
    solid = max(np.abs(z0[off:off + n]).max() for f, off, n, st in lay if f.startswith("eps_"))
    for f, off, n, st in lay:
        if f not in ("PhiL", "PhiS"):
            scale = conc if f in model.chem.liquid else solid
            assert np.abs(z[off:off + n] - z0[off:off + n]).max() <= 1e-11 * scale, f
    # the relaxed potentials solve the potential rows of the discharge residual at t = 4 s
    R = lis.residual(model, grid, z, z, 4.0, 1.0)
    M = lis.residual_magnitude(model, grid, z, z, 4.0, 1.0)
    for f, off, n, st in lis.layout(model, grid):
        if f in ("PhiL", "PhiS"):
            assert np.all(np.abs(R[off:off + n]) <= 1e-6 * M[off:off + n].max()), f


def test_relaxation_residual_at_equilibrium_before_the_ramp():
    """Relaxation residual (Sec. 2.8) at the Tab. 6 state and t = 0: every reaction rate is zero
    (to rounding), the collector current is ramped to T_H(0) = (1 + tanh(-6)) / 2 of its value
    (Eq. 56), and the anode exchange runs at r_Ano = c_Li / c_ref - 1 = 0.5 because Phi^L = 0
    and U0_Ano = 0 (Eqs. 26-27).  Species rows carry only the storage of a zero change (frozen),
    so they vanish exactly; the Li+ row has no anode term while relaxing."""
    model, grid = _case(0)
    z0 = init.uniform_state(model, grid, init.equilibrium_fields(model))
    R = lis.residual(model, grid, z0, z0, 0.0, 0.1, relax=True)
    M = lis.residual_magnitude(model, grid, z0, z0, 0.0, 0.1)
    U, Um = lis.unpack(model, grid, R), lis.unpack(model, grid, M)
    A = grid.h ** 2
    tH0 = 0.5 * (1.0 + np.tanh(-6.0))
    jcc = lis.j_el(model, grid) * grid.ny * grid.nz / grid.n_cc * tH0
    expect_S = np.zeros_like(np.real(U["PhiS"]))
    expect_S[:, :, 0] = np.where(grid.cc, A * jcc, 0.0)
    tol_S = 1e-12 * Um["PhiS"].max()
    assert np.all(np.abs(np.real(U["PhiS"]) - expect_S) <= tol_S)
    assert A * jcc > 1e3 * tol_S                          # the ramped current is resolved
    expect_L = np.zeros_like(np.real(U["PhiL"]))
    expect_L[:, :, -1] = A * 96485.332 * 5.0e-3 * 0.5
    assert np.all(np.abs(np.real(U["PhiL"]) - expect_L) <= 1e-12 * Um["PhiL"].max())
    for m in model.chem.liquid:
        assert np.all(U[m] == 0.0), m
