"""Consistent initial state (Sec. 2.8): Tab. 6 equilibrium, then parabolic relaxation.

Test infrastructure (see package docstring).
"""
from __future__ import annotations

import numpy as np

from . import chemistry as ch
from . import constants as K
from . import lis
from . import newton

# Initial concentrations of the three-species chemistry (Li+, S8(L), S8^2-), mol/m^3.
REDUCED3_C0 = {"Li": 1000.0, "S8L": 10.0, "S8_2": 100.0}


def equilibrium_fields(model):
    """Uniform field values of the equilibrium state: {field: value}.

    Tradeoff chemistry: Tab. 6 with <Phi^L>_0 = 0 and <Phi^S>_0 = Delta Phi_0 (gauge choice,
    Sec. 2.8), eps_S8 = eps_S8,0/eps_struct, eps_Li2S = eps_Li2S,0/eps_struct (Eq. 57).
    Three-species chemistry: REDUCED3_C0 with Phi^S at the Nernst potential of E1 (Eq. 24)."""
    chem = model.chem
    if chem.name == "tradeoff":
        eq = ch.equilibrium(model.T)
        vals = {m: eq["c_" + m] for m in chem.liquid}
        vals["eps_S8s"] = K.EPS_S8_0 / model.eps_struct
        vals["eps_Li2Ss"] = K.EPS_LI2S_0 / model.eps_struct
        vals["PhiL"] = 0.0
        vals["PhiS"] = eq["dPhi0"]
        return vals
    vals = dict(REDUCED3_C0)
    rx = chem.reactions[0]
    a = {m: vals[m] / K.C_REF for m in chem.liquid}
    ar, ap = ch.net_activities(rx, a)
    vals["PhiL"] = 0.0
    vals["PhiS"] = rx.U0 - K.R_GAS * model.T / K.F * np.log(ap / ar)
    return vals


def uniform_state(model, grid, vals):
    z = np.empty(lis.n_dof(model, grid))
    for f, off, n, st in lis.layout(model, grid):
        z[off:off + n] = vals[f]
    return z


def perturb(model, grid, z, noise, fields=None):
    """z * (1 + 0.01 noise) on the concentration fields (or the listed fields)."""
    out = z.copy()
    fields = model.chem.liquid if fields is None else fields
    for f, off, n, st in lis.layout(model, grid):
        if f in fields:
            out[off:off + n] = z[off:off + n] * (1.0 + 0.01 * noise[off:off + n])
    return out


def relax(model, grid, z0, dt=0.1, t_init=4.0, rtol=1e-10):
    """Parabolic relaxation: implicit Euler with dt = 0.1 s up to T_init = 4 s on the potential
    equations with d_t Phi terms, concentrations frozen and current ramped by T_H (Eq. 56)."""
    z = z0.copy()
    n = int(round(t_init / dt))
    t = 0.0
    for _ in range(n):
        z, info = newton.newton(model, grid, z, t + dt, dt, relax=True, rtol=rtol)
        if not info.converged:
            raise RuntimeError("relaxation step failed: " + info.reason)
        t += dt
    return z
