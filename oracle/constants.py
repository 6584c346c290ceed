"""Physical parameters of the Li-S model, as printed in the paper.

Test infrastructure (see package docstring).  Values are quoted with their table.
"""
import math

# Sec. 2.2, Eq. 1 text: Faraday constant, molar gas constant, reference concentration (Sec. 2.4, Eq. 20)
F = 96485.332          # C/mol
R_GAS = 8.3145         # J/(mol K)
# Sec. 2.2 prints T = 298 K; only 298.15 K reproduces the equilibrium column of Tab. 5.2.
T_DEFAULT = 298.15     # K
C_REF = 1000.0         # mol/m^3

# Eq. 2: viscosity exponent (m^3/mol)
VISC_EXP = 7.76e-4

# Tab. 5.2: diffusion coefficients at infinite dilution (m^2/s)
D0 = {
    "Li": 9.3e-10,
    "A": 9.3e-10,
    "S_2": 0.6e-10,
    "S4_2": 7.6e-10,
    "S6_2": 5.3e-10,
    "S8_2": 5.3e-10,
    "S8L": 10.0e-10,
}
# charge numbers (species names)
Z = {"Li": 1, "A": -1, "S_2": -2, "S4_2": -2, "S6_2": -2, "S8_2": -2, "S8L": 0}
# sulfur atoms per species, Sec. 2.2: c_S = c_S2- + 4 c_S4 + 6 c_S6 + 8 c_S8^2- + 8 c_S8(L)
SULFUR = {"Li": 0, "A": 0, "S_2": 1, "S4_2": 4, "S6_2": 6, "S8_2": 8, "S8L": 8}

# Tab. 5.1: cathode kinetics
K_SP1 = 0.006
K_C1 = 120.0           # mol/(s m^3)
K_SP2 = 8e-15
K_C2 = 3e-3            # mol/(s m^3)
U0 = {1: 2.41, 2: 2.32, 3: 2.31, 4: 1.985}   # V (E5, E6 follow from Tab. 6)
K_E = {1: 2.53e-6, 2: 3.54e-8, 3: 1.49e-10, 4: 2.05e-7, 5: 9.11e-10, 6: 1.37e-15}  # mol/(s m^2)

# Tab. 5.1: solid phase
A_V0 = 94.908e6        # 1/m
RHO_S8 = 2070.4        # kg/m^3
M_S8 = 0.2565          # kg/mol
EPS_S8_0 = 0.095
RHO_LI2S = 1659.0
M_LI2S = 0.0459
EPS_LI2S_0 = 2.77e-6
AV_A = 0.1392          # Eq. 18 parameter a (-)
AV_B = 3.310           # Eq. 18 parameter b (h)
KAPPA_S = 1.0          # S/m
K_ANO = 5.0e-3         # mol/(s m^2), anode
U0_ANO = 0.0

# Tab. 5.2: initial Li+ concentration
C_LI_0 = 1500.0

# Tab. 2: cathode volume fractions (cathode total 0.168, sulfur 0.0956)
X_CATHODE = 0.168
X_SULFUR = 0.0956
# Sec. 2.1 / Sec. 2.5: separator porosity
EPS_SEP = 0.4

# App. B: theoretical capacity c_theo = n_e F / M_S8 with n_e = 16 (C/kg)
N_E_S8 = 16


def c_theo():
    """Theoretical capacity of S8 in C/kg (App. B)."""
    return N_E_S8 * F / M_S8


def c_theo_ah_per_kg():
    return c_theo() / 3600.0


def sulfur_loading(L_cat):
    """m_A,S8 = rho_S8 eps_S8,0 L_Cat in kg/m^2 (App. B)."""
    return RHO_S8 * EPS_S8_0 * L_cat


def j_el_from_rate(f_C_per_h, L_cat):
    """Galvanostatic current density j_el = f_C c_theo m_A,S8 (App. B), f_C in 1/h, result A/m^2."""
    return (f_C_per_h / 3600.0) * c_theo() * sulfur_loading(L_cat)


def thermal_voltage(T=T_DEFAULT):
    return R_GAS * T / F


def smooth_step(t):
    """T_H(t) = (1 + tanh(6 (t - 1 s))) / 2, Eq. 56."""
    return 0.5 * (1.0 + math.tanh(6.0 * (t - 1.0)))
