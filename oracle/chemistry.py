"""Reactions, constitutive laws and the equilibrium state of the Li-S model.

Test infrastructure (see package docstring).  All functions accept real or
complex numpy arrays (complex-step differentiation); branches test the real part.

Species names: Li (Li+), S8L (S8(L)), S8_2 (S8^2-), S6_2 (S6^2-), S4_2 (S4^2-),
S_2 (S^2-); solids S8s (S8(S)), Li2Ss (Li2S(S)); A is the eliminated anion.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from fractions import Fraction as Fr

import numpy as np

from . import constants as K


def _pos(x):
    """max(x, 0), taking the branch on the real part."""
    return np.where(np.real(x) > 0, x, 0.0)


@dataclass
class Reaction:
    """One row of Tab. 3. ``nu`` maps species to stoichiometric coefficients
    (reactants negative, products positive); each E reaction also consumes one e- (S)."""

    name: str
    kind: str                   # "C" chemical bulk, "E" electrochemical surface
    nu: dict
    k: float                    # k_C,k in mol/(s m^3) or k_E,k in mol/(s m^2)
    K_sp: float = 0.0           # C only
    U0: float = 0.0             # E only
    solid: str = ""             # C only: the solid whose volume fraction scales the rate (Eq. 5)
    smooth: bool = False        # rate multiplied by T_H(t) (reactions with S^2-, Sec. 2.8)


@dataclass
class Chemistry:
    name: str
    liquid: list                # transported liquid species (anion eliminated)
    solid: list                 # solid species with a volume-fraction field
    reactions: list
    frozen_solid: dict = field(default_factory=dict)   # solids held at their initial fraction

    @property
    def fields(self):
        return list(self.liquid) + ["eps_" + s for s in self.solid] + ["PhiL", "PhiS"]

    def is_struct_field(self, f):
        return f.startswith("eps_") or f == "PhiS"


def reaction_table():
    """Tab. 3 (Tradeoff Chemistry) with the rate constants of Tab. 5.1.

    U0 of E5 and E6 is filled in by ``equilibrium`` (Tab. 6)."""
    return [
        Reaction("C1", "C", {"S8s": Fr(-1), "S8L": Fr(1)}, K.K_C1, K_sp=K.K_SP1, solid="S8s"),
        Reaction("C2", "C", {"Li2Ss": Fr(-1), "Li": Fr(2), "S_2": Fr(1)}, K.K_C2, K_sp=K.K_SP2,
                 solid="Li2Ss", smooth=True),
        Reaction("E1", "E", {"S8L": Fr(-1, 2), "S8_2": Fr(1, 2)}, K.K_E[1], U0=K.U0[1]),
        Reaction("E2", "E", {"S8_2": Fr(-3, 2), "S6_2": Fr(2)}, K.K_E[2], U0=K.U0[2]),
        Reaction("E3", "E", {"S6_2": Fr(-1), "S4_2": Fr(3, 2)}, K.K_E[3], U0=K.U0[3]),
        Reaction("E4", "E", {"S4_2": Fr(-1, 6), "S_2": Fr(2, 3)}, K.K_E[4], U0=K.U0[4], smooth=True),
        Reaction("E5", "E", {"S8_2": Fr(-1, 2), "S4_2": Fr(1)}, K.K_E[5], U0=np.nan),
        Reaction("E6", "E", {"S4_2": Fr(-1, 6), "Li": Fr(-4, 3), "Li2Ss": Fr(2, 3)}, K.K_E[6], U0=np.nan),
    ]


def equilibrium(T=K.T_DEFAULT, c_Li=K.C_LI_0):
    """Tab. 6 sequence: equilibrium concentrations, Delta Phi_0, U0_red,5 and U0_red,6.

    Returns a dict with c_<species>, dPhi0, U5, U6 and c_A (charge neutrality, Sec. 2.5 (i))."""
    RT_F = K.R_GAS * T / K.F
    cref = K.C_REF
    U1, U2, U3, U4 = K.U0[1], K.U0[2], K.U0[3], K.U0[4]
    c_S8L = K.K_SP1 * cref
    c_S2 = K.K_SP2 * cref ** 3 / c_Li ** 2
    dPhi0 = ((0.75 * U1 + 0.25 * U2) / 6.0 + U3 / 12.0 + 0.75 * U4
             + RT_F * np.log((c_S8L / cref) ** (1.0 / 16.0) / (c_S2 / cref) ** 0.5))
    c_S8_2 = c_S8L * np.exp(-2.0 * (dPhi0 - U1) / RT_F)
    c_S6_2 = cref * (c_S8L / cref) ** 0.75 * np.exp(-2.0 * (dPhi0 - (0.75 * U1 + 0.25 * U2)) / RT_F)
    c_S4_2 = cref * (c_S2 / cref) ** 4 * np.exp(6.0 * (dPhi0 - U4) / RT_F)
    U5 = dPhi0 - RT_F * np.log((c_S8_2 / cref) ** 0.5 / (c_S4_2 / cref))
    U6 = dPhi0 - RT_F * np.log((c_S4_2 / cref) ** (1.0 / 6.0) * (c_Li / cref) ** (4.0 / 3.0))
    conc = {"Li": c_Li, "S8L": c_S8L, "S8_2": c_S8_2, "S6_2": c_S6_2, "S4_2": c_S4_2, "S_2": c_S2}
    c_A = sum(K.Z[m] * v for m, v in conc.items()) / (-K.Z["A"])
    out = {"c_" + m: v for m, v in conc.items()}
    out.update(dPhi0=dPhi0, U5=U5, U6=U6, c_A=c_A)
    return out


def tradeoff(T=K.T_DEFAULT):
    """The paper's Tradeoff Chemistry (Fig. 2c, Tab. 3): 6 liquid species, 2 solids, 8 reactions."""
    eq = equilibrium(T)
    rx = reaction_table()
    for r in rx:
        if r.name == "E5":
            r.U0 = eq["U5"]
        if r.name == "E6":
            r.U0 = eq["U6"]
    return Chemistry("tradeoff", ["Li", "S8L", "S8_2", "S6_2", "S4_2", "S_2"], ["S8s", "Li2Ss"], rx)


def reduced3(T=K.T_DEFAULT):
    """Three-species chemistry of the small DG0 workload: Li+, S8(L), S8^2-, reaction E1 only,
    solid volume fractions frozen at their initial values (no solid fields)."""
    rx = [r for r in reaction_table() if r.name == "E1"]
    return Chemistry("reduced3", ["Li", "S8L", "S8_2"], [], rx,
                     frozen_solid={"S8s": K.EPS_S8_0, "Li2Ss": K.EPS_LI2S_0})


# ----------------------------------------------------------------------------- pointwise laws

def activities(chem, c):
    """<a_m> = <c_m>/c_ref for liquid species (Eq. 20 text); negative values clipped to 0."""
    return {m: _pos(c[m]) / K.C_REF for m in chem.liquid}


def net_activities(rx, a):
    """<a>_reac,k and <a>_prod,k of Eq. 20 (solids and e- have activity 1)."""
    ar, ap = 1.0, 1.0
    for m, nu in rx.nu.items():
        if m not in a:
            continue
        if nu < 0:
            ar = ar * a[m] ** float(-nu)
        else:
            ap = ap * a[m] ** float(nu)
    return ar, ap


def rates_mass_action(chem, c, phiL, phiS, T=K.T_DEFAULT):
    """Reaction rates r_V,k / r_A,k in the mass-action form.

    C: r = <a>_r sqrt(K_sp) - <a>_p / sqrt(K_sp)         (Eqs. 19-21 combined, alpha = 1/2)
    E: r = <a>_r exp(-x) - <a>_p exp(x),  x = F (Phi_S - Phi_L - U0) / (2 R T)  (Eqs. 22-24, n_e = 1)
    These equal the sinh/ln forms below for positive activities and stay finite at zero activity."""
    a = activities(chem, c)
    out = {}
    for rx in chem.reactions:
        ar, ap = net_activities(rx, a)
        if rx.kind == "C":
            s = np.sqrt(rx.K_sp)
            out[rx.name] = ar * s - ap / s
        else:
            x = K.F * (phiS - phiL - rx.U0) / (2.0 * K.R_GAS * T)
            out[rx.name] = ar * np.exp(-x) - ap * np.exp(x)
    return out


def rates_literal(chem, c, phiL, phiS, T=K.T_DEFAULT):
    """Rates written exactly as Eqs. 19_simp, 21, 22, 23, 24 (positive activities only)."""
    a = activities(chem, c)
    RT = K.R_GAS * T
    out = {}
    for rx in chem.reactions:
        ar, ap = net_activities(rx, a)
        Q = ap / ar
        if rx.kind == "C":
            dG = RT * np.log(Q / rx.K_sp)
        else:
            U_eq = rx.U0 - RT / K.F * np.log(Q)
            dG = K.F * (phiS - phiL - U_eq)
        out[rx.name] = -2.0 * np.sqrt(ar * ap) * np.sinh(dG / (2.0 * RT))
    return out


def specific_surface(eS8, eLi2S, f_C, eps_struct):
    """a_V of Eq. 18 with the 3D localisation of Eq. 57 (eps_struct = 1 gives the 1D model).

    Negative volume fractions are clipped to 0 and a negative result to 0."""
    t1 = (_pos(eS8) / (1.2 * K.EPS_S8_0 / eps_struct)) ** 1.5
    t2 = (_pos(eLi2S) / (K.AV_A * np.exp(-K.AV_B * f_C) / eps_struct)) ** 1.5
    return K.A_V0 / eps_struct * _pos(1.0 - t1 - t2)


def cbd_fraction(eps_struct):
    """Inert carbon-binder volume fraction inside a structure voxel, Eq. 57: (x_Cathode - x_Sulfur)/eps_struct."""
    return (K.X_CATHODE - K.X_SULFUR) / eps_struct


def sulfur_concentration(c):
    """c_S^L of Sec. 2.2 (dissolved sulfur atoms, mol/m^3)."""
    return sum(K.SULFUR[m] * c[m] for m in c if K.SULFUR.get(m, 0))


def transport_factor(epsL, c):
    """g = (eps_L)^{3/2} eta(0)/eta(c_S): Bruggeman (Eq. 18 final, tau = eps^{-1/2}) times Stokes-Einstein (Eqs. 2-3)."""
    cS = sulfur_concentration(c)
    return _pos(epsL) ** 1.5 * np.exp(-K.VISC_EXP * cS)


def rates_magnitude(chem, c, phiL, phiS, T=K.T_DEFAULT):
    """|forward| + |backward| term of each mass-action rate (size of the terms that cancel)."""
    a = activities(chem, c)
    out = {}
    for rx in chem.reactions:
        ar, ap = net_activities(rx, a)
        if rx.kind == "C":
            s = np.sqrt(rx.K_sp)
            out[rx.name] = np.abs(ar * s) + np.abs(ap / s)
        else:
            x = K.F * (phiS - phiL - rx.U0) / (2.0 * K.R_GAS * T)
            out[rx.name] = np.abs(ar * np.exp(-x)) + np.abs(ap * np.exp(x))
    return out


def sources(chem, c, eps_solid, phiL, phiS, tH, aV, T=K.T_DEFAULT, mag=False):
    """Volumetric sources (mol m^-3 s^-1) and charge sources (A m^-3) at structure points.

    Species i:  k_C R_C,i + a_V k_E R_E,i / F = sum_C nu_ik eps_s(k) k_C,k r_k + a_V sum_E nu_ik k_E,k r_k  (Eqs. 5, 6, 16, 17)
    Liquid charge:  sum_j z_j a_V k_E R_E,j  (Tab. 4 row 2);  solid charge: z_e a_V k_E R_E,e (Eq. 17b).
    Reactions flagged ``smooth`` are multiplied by T_H (Sec. 2.8)."""
    r = rates_magnitude(chem, c, phiL, phiS, T) if mag else rates_mass_action(chem, c, phiL, phiS, T)
    names = list(chem.liquid) + list(chem.solid)
    S = {m: 0.0 for m in names}
    SE = {m: 0.0 for m in chem.liquid}
    e_rate = 0.0                                  # sum_E k_E,k r_k T_k
    for rx in chem.reactions:
        rate = r[rx.name] * (tH if rx.smooth else 1.0)
        sg = (lambda v: abs(float(v))) if mag else float
        if rx.kind == "C":
            w = eps_solid[rx.solid] * rx.k * rate
            if mag:
                w = np.abs(w)
            for m, nu in rx.nu.items():
                if m in S:
                    S[m] = S[m] + sg(nu) * w
        else:
            w = aV * rx.k * rate
            if mag:
                w = np.abs(w)
            for m, nu in rx.nu.items():
                if m in S:
                    S[m] = S[m] + sg(nu) * w
                if m in SE:
                    SE[m] = SE[m] + sg(nu) * w
            e_rate = e_rate + rx.k * rate
    if mag:
        q_liquid = K.F * sum(abs(K.Z[m]) * SE[m] for m in chem.liquid)
        return S, q_liquid, np.abs(aV) * K.F * e_rate
    q_liquid = K.F * sum(K.Z[m] * SE[m] for m in chem.liquid)
    nu_e, z_e = -1.0, -1.0
    q_solid = z_e * aV * K.F * nu_e * e_rate
    return S, q_liquid, q_solid
