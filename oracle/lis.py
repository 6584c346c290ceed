"""Residual of the coarse-grained Li-S system (Tab. 4) on a masked voxel grid, DG0 and DG1.

Test infrastructure (see package docstring).

Unknowns (Sec. 2.7, N_var = 10 for the Tradeoff Chemistry): liquid concentrations
<c_i^L> (all cells), solid volume fractions eps_S8, eps_Li2S (structure cells),
Phi^L (all cells), Phi^S (structure cells).  Phases: 0 macro-pore (eps_L = 1, no
reactions), 1 coarse-grained structure (Eq. 57 localisation, reactions, kappa_S),
2 homogeneous separator (eps_L = 0.4, no reactions, no solid conduction; Sec. 2.1).

State-vector layout (shared interface with the C library, defined here independently):
fields are stored one after another in ``Chemistry.fields`` order; a liquid/Phi^L field
has one value per cell (cell index i + nx*(j + ny*k)), a solid/Phi^S field one value per
structure cell in increasing cell index.  DG1 multiplies each field by 8 nodes stored
node-major: field offset + node*len + cell, node = a + 2b + 4c for the x, y, z node indices.

Boundary conditions (Tab. 4): Neumann current j_el at the current collector (x = 0) on
structure faces, rescaled so that the total current is j_el * (ny nz h^2); Butler-Volmer
Li+ exchange at the anode face (x = nx) with Phi^S_Ano = 0 and U0_Ano = 0 (Eqs. 25-27);
no flux elsewhere.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import chemistry as ch
from . import constants as K
from . import dg

PORE, STRUCT, SEP = 0, 1, 2


@dataclass
class Model:
    chem: ch.Chemistry
    order: int = 0                 # 0: DG0, 1: DG1 (Q1)
    T: float = K.T_DEFAULT
    f_C: float = 0.5               # discharge rate in 1/h
    eps_struct: float = 0.4        # structure volume fraction of the cathode (1 - porosity), Eq. 57
    j_el: float | None = None      # A/m^2; None: from f_C (App. B)
    penalty: float = 1.0           # interior-penalty factor (Eq. 46)
    smooth: bool = True            # T_H regularisation of the S^2- reactions (Sec. 2.8)


class Grid:
    def __init__(self, phase, h):
        self.phase = np.asarray(phase, dtype=np.uint8)
        self.nz, self.ny, self.nx = self.phase.shape
        self.h = float(h)
        self.struct = self.phase == STRUCT
        self.sep = self.phase == SEP
        self.struct_idx = np.flatnonzero(self.struct.ravel())
        self.n_cell = self.phase.size
        self.n_struct = self.struct_idx.size
        self.cc = self.struct[:, :, 0]
        self.n_cc = int(self.cc.sum())
        sep_layers = np.all(self.sep, axis=(0, 1))
        self.n_sep = int(sep_layers.sum())
        self.L_cat = (self.nx - self.n_sep) * self.h


def j_el(model, grid):
    if model.j_el is not None:
        return model.j_el
    return K.j_el_from_rate(model.f_C, grid.L_cat)


def layout(model, grid):
    """[(field, offset, length, on_structure_only)]; lengths include the 8 DG1 nodes."""
    nn = 8 if model.order == 1 else 1
    out, off = [], 0
    for f in model.chem.fields:
        st = model.chem.is_struct_field(f)
        n = (grid.n_struct if st else grid.n_cell) * nn
        out.append((f, off, n, st))
        off += n
    return out


def n_dof(model, grid):
    lay = layout(model, grid)
    return lay[-1][1] + lay[-1][2]


def _shape(model, grid):
    base = (grid.nz, grid.ny, grid.nx)
    return (2, 2, 2) + base if model.order == 1 else base


def unpack(model, grid, z):
    """Flat state -> dict of dense arrays (solid fields zero outside the structure)."""
    shp = _shape(model, grid)
    out = {}
    for f, off, n, st in layout(model, grid):
        seg = z[off:off + n]
        if model.order == 1:
            seg = seg.reshape(8, -1)
            if st:
                full = np.zeros((8, grid.n_cell), dtype=z.dtype)
                full[:, grid.struct_idx] = seg
                seg = full
            out[f] = seg.reshape(shp)
        else:
            if st:
                full = np.zeros(grid.n_cell, dtype=z.dtype)
                full[grid.struct_idx] = seg
                seg = full
            out[f] = seg.reshape(shp)
    return out


def pack(model, grid, d, dtype=float):
    parts = []
    for f, off, n, st in layout(model, grid):
        a = np.asarray(d[f])
        if model.order == 1:
            a = a.reshape(8, grid.n_cell)
            parts.append((a[:, grid.struct_idx] if st else a).ravel())
        else:
            a = a.ravel()
            parts.append(a[grid.struct_idx] if st else a)
    return np.concatenate(parts).astype(np.result_type(dtype, *parts))


# --------------------------------------------------------------------------- point physics

def _solid_fractions(model, U):
    chem = model.chem
    out = {}
    for s in ("S8s", "Li2Ss"):
        if s in chem.solid:
            out[s] = U["eps_" + s]
        else:
            out[s] = chem.frozen_solid[s] / model.eps_struct
    return out


def liquid_fraction(model, phase, eps_solid):
    """eps_L = 1 - sum of solid fractions (Sec. 2.5 (ii)) in structure, 0.4 in separator, 1 in pores."""
    es = model.eps_struct
    epsL_struct = 1.0 - ch.cbd_fraction(es) - eps_solid["S8s"] - eps_solid["Li2Ss"]
    return np.where(phase == STRUCT, epsL_struct, np.where(phase == SEP, K.EPS_SEP, 1.0))


def coefficients(model, phase, U):
    """Transport coefficients at points (cells, nodes or face points).

    Returns {equation: [(coefficient, potential-field-name), ...]} following Tab. 4:
      species i:   D_i^eff grad c_i + z_i F/(RT) D_i^eff c_i grad Phi^L
      Phi^L:       sum_j z_j F (D_j^eff - D_A^eff) grad c_j + z_j F^2/(RT)(z_j D_j^eff - z_A D_A^eff) c_j grad Phi^L
      Phi^S:       kappa_S grad Phi^S (kappa_S only inside the structure)"""
    chem = model.chem
    RT = K.R_GAS * model.T
    eps_s = _solid_fractions(model, U)
    epsL = liquid_fraction(model, phase, eps_s)
    c = {m: U[m] for m in chem.liquid}
    g = ch.transport_factor(epsL, c)
    DA = K.D0["A"] * g
    zA = K.Z["A"]
    terms = {}
    phiL_terms = []
    for m in chem.liquid:
        Dm = K.D0[m] * g
        sig = K.Z[m] * K.F / RT * Dm * c[m]
        terms[m] = [(Dm, m), (sig, "PhiL")]
        phiL_terms.append((K.Z[m] * K.F * (Dm - DA), m))
        phiL_terms.append((K.Z[m] * K.F ** 2 / RT * (K.Z[m] * Dm - zA * DA) * c[m], "PhiL"))
    terms["PhiL"] = phiL_terms
    terms["PhiS"] = [(np.where(phase == STRUCT, K.KAPPA_S, 0.0) * np.ones_like(g), "PhiS")]
    return terms, epsL


def point_sources(model, phase, U, tH):
    """Sources at points, zero outside the structure (reactions only in the cathode structure, Sec. 2.6)."""
    chem = model.chem
    eps_s = _solid_fractions(model, U)
    aV = ch.specific_surface(eps_s["S8s"], eps_s["Li2Ss"], model.f_C, model.eps_struct)
    c = {m: U[m] for m in chem.liquid}
    S, qL, qS = ch.sources(chem, c, eps_s, U["PhiL"], U["PhiS"], tH, aV, model.T)
    st = phase == STRUCT
    S = {m: np.where(st, v, 0.0) for m, v in S.items()}
    return S, np.where(st, qL, 0.0), np.where(st, qS, 0.0)


def anode_rate(model, cLi, phiL):
    """r_A,Ano for Li+ + e- <-> Li(S) with Phi^S_Ano = 0, U0_Ano = 0 (Eqs. 22-24, 26):
    r = a_Li exp(-x) - exp(x), x = F (0 - Phi^L - 0) / (2RT)."""
    x = K.F * (0.0 - phiL - K.U0_ANO) / (2.0 * K.R_GAS * model.T)
    return ch._pos(cLi) / K.C_REF * np.exp(-x) - np.exp(x)


# --------------------------------------------------------------------------- residual

def residual(model, grid, z, zn, t, dt, relax=False):
    """R(z; z^n, t, dt) of the implicit Euler step (Eq. 50) in the DG weak form.

    relax=True gives the parabolic relaxation of Sec. 2.8: concentrations and solid fractions
    frozen at z^n, d_t Phi terms with coefficient 1 added to both potential equations and the
    current ramped by T_H(t)."""
    if model.order == 0:
        return _residual_dg0(model, grid, z, zn, t, dt, relax)
    return _residual_dg1(model, grid, z, zn, t, dt, relax)


def _storage_terms(model, U, Un, phase, Mw, dt, relax):
    chem = model.chem
    R = {}
    eps_s, eps_sn = _solid_fractions(model, U), _solid_fractions(model, Un)
    epsL, epsLn = liquid_fraction(model, phase, eps_s), liquid_fraction(model, phase, eps_sn)
    for m in chem.liquid:
        if relax:
            R[m] = Mw * (U[m] - Un[m]) / dt
        else:
            R[m] = Mw * (epsL * U[m] - epsLn * Un[m]) / dt
    rho_M = {"S8s": K.RHO_S8 / K.M_S8, "Li2Ss": K.RHO_LI2S / K.M_LI2S}
    for s in chem.solid:
        f = "eps_" + s
        R[f] = Mw * rho_M[s] * (U[f] - Un[f]) / dt * (phase == STRUCT)
    if relax:
        R["PhiL"] = Mw * (U["PhiL"] - Un["PhiL"]) / dt
        R["PhiS"] = Mw * (U["PhiS"] - Un["PhiS"]) / dt * (phase == STRUCT)
    else:
        R["PhiL"] = 0.0 * U["PhiL"]
        R["PhiS"] = 0.0 * U["PhiS"]
    return R


def _smooth_factor(model, t):
    return K.smooth_step(t) if model.smooth else 1.0


def _residual_dg0(model, grid, z, zn, t, dt, relax):
    chem = model.chem
    h = grid.h
    V, A = h ** 3, h ** 2
    U, Un = unpack(model, grid, z), unpack(model, grid, zn)
    phase = grid.phase
    R = _storage_terms(model, U, Un, phase, V, dt, relax)
    terms, _ = coefficients(model, phase, U)
    S, qL, qS = point_sources(model, phase, U, _smooth_factor(model, t))
    eqs = list(chem.liquid) + ["PhiL", "PhiS"]
    for e in eqs:
        if relax and e in chem.liquid:
            continue
        for Kc, f in terms[e]:
            R[e] = R[e] + dg.dg0_faces(Kc, U[f], h)
    if not relax:
        for m in chem.liquid:
            R[m] = R[m] - V * S[m]
        for s in chem.solid:
            R["eps_" + s] = R["eps_" + s] - V * S[s]
    R["PhiL"] = R["PhiL"] - V * qL
    R["PhiS"] = R["PhiS"] - V * qS
    # anode (x = nx face of the last layer), Eqs. 27
    rA = anode_rate(model, U["Li"][:, :, -1], U["PhiL"][:, :, -1])
    if not relax:
        R["Li"][:, :, -1] += A * K.K_ANO * rA
    R["PhiL"][:, :, -1] += A * K.F * K.K_ANO * rA
    # current collector (x = 0 face, structure cells), Eq. 25 with f^N = j_el
    jcc = _cc_current(model, grid, t, relax)
    R["PhiS"][:, :, 0] += np.where(grid.cc, A * jcc, 0.0)
    return pack(model, grid, R, dtype=z.dtype)


def _cc_current(model, grid, t, relax):
    if grid.n_cc == 0:
        raise ValueError("no structure cell touches the current collector")
    j = j_el(model, grid) * (grid.ny * grid.nz) / grid.n_cc
    if relax:
        j = j * K.smooth_step(t)
    return j


def _face_coefficients(model, grid, U):
    """Coefficients evaluated from the traced fields on both faces of every cell, per direction."""
    out = {}
    for d in ("x", "y", "z"):
        per_side = {}
        for side in (+1, -1):
            Ut = {f: dg.trace(v, d, side) for f, v in U.items()}
            ph = np.broadcast_to(grid.phase, Ut["PhiL"].shape)
            terms, _ = coefficients(model, ph, Ut)
            per_side[side] = terms
        out[d] = per_side
    return out


def _residual_dg1(model, grid, z, zn, t, dt, relax):
    chem = model.chem
    h = grid.h
    Mw = h ** 3 / 8.0
    U, Un = unpack(model, grid, z), unpack(model, grid, zn)
    phase = np.broadcast_to(grid.phase, U["PhiL"].shape)
    R = _storage_terms(model, U, Un, phase, Mw, dt, relax)
    terms, _ = coefficients(model, phase, U)
    fterms = _face_coefficients(model, grid, U)
    S, qL, qS = point_sources(model, phase, U, _smooth_factor(model, t))
    eqs = list(chem.liquid) + ["PhiL", "PhiS"]
    for e in eqs:
        if relax and e in chem.liquid:
            continue
        for it, (Kn, f) in enumerate(terms[e]):
            Kf = {d: (fterms[d][+1][e][it][0], fterms[d][-1][e][it][0]) for d in ("x", "y", "z")}
            R[e] = R[e] + dg.dg1_volume(Kn, U[f], h) + dg.dg1_faces(Kf, U[f], h, model.penalty)
    if not relax:
        for m in chem.liquid:
            R[m] = R[m] - Mw * S[m]
        for s in chem.solid:
            R["eps_" + s] = R["eps_" + s] - Mw * S[s]
    R["PhiL"] = R["PhiL"] - Mw * qL
    R["PhiS"] = R["PhiS"] - Mw * qS
    # anode: face xi = +1 in x of the last layer
    last = np.zeros((grid.nz, grid.ny, grid.nx), dtype=bool)
    last[:, :, -1] = True
    cLi_t, phiL_t = dg.trace(U["Li"], "x", +1), dg.trace(U["PhiL"], "x", +1)
    rA = np.where(last, anode_rate(model, cLi_t, phiL_t), 0.0)
    if not relax:
        R["Li"] = R["Li"] + dg.dg1_boundary_flux(U["Li"].shape, "x", +1, K.K_ANO * rA, h, dtype=z.dtype)
    R["PhiL"] = R["PhiL"] + dg.dg1_boundary_flux(U["PhiL"].shape, "x", +1, K.F * K.K_ANO * rA, h, dtype=z.dtype)
    # current collector: face xi = -1 in x of structure cells in the first layer
    first = np.zeros((grid.nz, grid.ny, grid.nx), dtype=bool)
    first[:, :, 0] = True
    fN = np.where(first & grid.struct, _cc_current(model, grid, t, relax), 0.0)
    R["PhiS"] = R["PhiS"] + dg.dg1_boundary_flux(U["PhiS"].shape, "x", -1, fN, h, dtype=z.dtype)
    return pack(model, grid, R, dtype=z.dtype)


# --------------------------------------------------------------------------- battery quantities

def cell_voltage(model, grid, z):
    """U_cell = |A_CC|^-1 int_{A_CC} <Phi^S> do (Eq. A1) over the structure faces at x = 0 (Phi^S_Ano = 0)."""
    U = unpack(model, grid, z)
    if model.order == 0:
        return float(np.real(U["PhiS"][:, :, 0][grid.cc]).mean())
    tr = dg.trace(U["PhiS"], "x", -1)[..., 0]            # (2, 2, nz, ny) face points
    return float(np.real(tr[:, :, grid.cc]).mean())


def cell_means(model, grid, z):
    """Volume integrals over cathode + separator (Eq. A3 numerators): liquid-phase amounts
    int eps_L c_i, solid amounts int (rho/M) eps_s, and the liquid charge int eps_L sum z_j F c_j."""
    chem = model.chem
    U = unpack(model, grid, z)
    phase = grid.phase if model.order == 0 else np.broadcast_to(grid.phase, U["PhiL"].shape)
    Mw = grid.h ** 3 if model.order == 0 else grid.h ** 3 / 8.0
    eps_s = _solid_fractions(model, U)
    epsL = liquid_fraction(model, phase, eps_s)
    out = {}
    for m in chem.liquid:
        out[m] = float(np.sum(Mw * epsL * U[m]))
    rho_M = {"S8s": K.RHO_S8 / K.M_S8, "Li2Ss": K.RHO_LI2S / K.M_LI2S}
    for s in chem.solid:
        out[s] = float(np.sum(Mw * rho_M[s] * U["eps_" + s] * (phase == STRUCT)))
    out["charge"] = float(np.sum(Mw * epsL * K.F * sum(K.Z[m] * U[m] for m in chem.liquid)))
    out["sulfur"] = sum(K.SULFUR[m] * out[m] for m in chem.liquid) + \
        (8 * out["S8s"] if "S8s" in out else 0.0) + (out["Li2Ss"] if "Li2Ss" in out else 0.0)
    out["lithium"] = out["Li"] + (2 * out["Li2Ss"] if "Li2Ss" in out else 0.0)
    return out


# --------------------------------------------------------------------------- rounding scale

def residual_magnitude(model, grid, z, zn, t, dt):
    """Per-row sum of the absolute values of the terms that make up ``residual`` (storage parts,
    every face flux, forward and backward reaction terms, boundary terms): the size against
    which rounding differences between two implementations of the residual are measured."""
    chem = model.chem
    h = grid.h
    dg1 = model.order == 1
    Mw = h ** 3 / 8.0 if dg1 else h ** 3
    U, Un = unpack(model, grid, z), unpack(model, grid, zn)
    phase = np.broadcast_to(grid.phase, U["PhiL"].shape) if dg1 else grid.phase
    eps_s, eps_sn = _solid_fractions(model, U), _solid_fractions(model, Un)
    epsL, epsLn = liquid_fraction(model, phase, eps_s), liquid_fraction(model, phase, eps_sn)
    R = {}
    for m in chem.liquid:
        R[m] = Mw * (np.abs(epsL * U[m]) + np.abs(epsLn * Un[m])) / dt
    rho_M = {"S8s": K.RHO_S8 / K.M_S8, "Li2Ss": K.RHO_LI2S / K.M_LI2S}
    for s in chem.solid:
        f = "eps_" + s
        R[f] = Mw * rho_M[s] * (np.abs(U[f]) + np.abs(Un[f])) / dt * (phase == STRUCT)
    R["PhiL"] = 0.0 * np.abs(U["PhiL"])
    R["PhiS"] = 0.0 * np.abs(U["PhiS"])
    terms, _ = coefficients(model, phase, U)
    if dg1:
        fterms = _face_coefficients(model, grid, U)
    for e in list(chem.liquid) + ["PhiL", "PhiS"]:
        for it, (Kn, f) in enumerate(terms[e]):
            if dg1:
                Kf = {d: (fterms[d][+1][e][it][0], fterms[d][-1][e][it][0]) for d in ("x", "y", "z")}
                R[e] = R[e] + dg.dg1_volume(Kn, U[f], h, mag=True) + dg.dg1_faces(Kf, U[f], h, model.penalty, mag=True)
            else:
                R[e] = R[e] + dg.dg0_faces(Kn, U[f], h, mag=True)
    eps = _solid_fractions(model, U)
    aV = ch.specific_surface(eps["S8s"], eps["Li2Ss"], model.f_C, model.eps_struct)
    c = {m: U[m] for m in chem.liquid}
    S, qL, qS = ch.sources(chem, c, eps, U["PhiL"], U["PhiS"], _smooth_factor(model, t), aV, model.T, mag=True)
    st = phase == STRUCT
    for m in chem.liquid:
        R[m] = R[m] + Mw * np.where(st, S[m], 0.0)
    for s in chem.solid:
        R["eps_" + s] = R["eps_" + s] + Mw * np.where(st, S[s], 0.0)
    R["PhiL"] = R["PhiL"] + Mw * np.where(st, qL, 0.0)
    R["PhiS"] = R["PhiS"] + Mw * np.where(st, qS, 0.0)
    x = lambda phiL: K.F * (0.0 - phiL) / (2.0 * K.R_GAS * model.T)
    A = h * h
    if dg1:
        cLi_t, phiL_t = dg.trace(U["Li"], "x", +1), dg.trace(U["PhiL"], "x", +1)
        last = np.zeros((grid.nz, grid.ny, grid.nx), dtype=bool)
        last[:, :, -1] = True
        rm = np.where(last, np.abs(cLi_t) / K.C_REF * np.exp(-x(phiL_t)) + np.exp(x(phiL_t)), 0.0)
        R["Li"] = R["Li"] + dg.dg1_boundary_flux(U["Li"].shape, "x", +1, K.K_ANO * rm, h, mag=True)
        R["PhiL"] = R["PhiL"] + dg.dg1_boundary_flux(U["Li"].shape, "x", +1, K.F * K.K_ANO * rm, h, mag=True)
        first = np.zeros((grid.nz, grid.ny, grid.nx), dtype=bool)
        first[:, :, 0] = True
        fN = np.where(first & grid.struct, abs(_cc_current(model, grid, t, False)), 0.0)
        R["PhiS"] = R["PhiS"] + dg.dg1_boundary_flux(U["PhiS"].shape, "x", -1, fN, h, mag=True)
    else:
        cL, pL = U["Li"][:, :, -1], U["PhiL"][:, :, -1]
        rm = np.abs(cL) / K.C_REF * np.exp(-x(pL)) + np.exp(x(pL))
        R["Li"][:, :, -1] += A * K.K_ANO * rm
        R["PhiL"][:, :, -1] += A * K.F * K.K_ANO * rm
        R["PhiS"][:, :, 0] += np.where(grid.cc, A * abs(_cc_current(model, grid, t, False)), 0.0)
    return pack(model, grid, R)
