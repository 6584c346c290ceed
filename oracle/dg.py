"""Generic discontinuous-Galerkin operators on a uniform voxel grid (Sec. 2.6, App. A).

Test infrastructure (see package docstring).

Weak form of  d_t psi = div(K grad psi) + S  (Eq. 42) per Eq. 43 with the
interior-penalty flux of Eqs. 46-47:

  int d_t psi v  +  int K grad psi . grad v  -  sum_faces int {K grad psi}.[[v]]
                 +  sum_faces int {K}_H [[psi]].[[v]] / h  +  sum_bnd int f^N v  =  int S v

Conventions used throughout the oracle
  * DG0 arrays have shape (nz, ny, nx) (x fastest in memory); cell volume V = h^3, face area A = h^2.
  * DG1 arrays have shape (2, 2, 2, nz, ny, nx): nodal values of a Q1 Lagrange basis on the
    2-point Gauss-Legendre nodes +-1/sqrt(3) of each cell, node axes ordered (z, y, x).
    Volume and face integrals use the same Gauss points, so the mass matrix is diagonal
    (h^3/8 per node), face quadrature points lie on nodal lines, and traces come from
    the 1D extrapolation weights (1 +- sqrt(3))/2.
  * {K grad psi} on interior faces is taken as {K}_H {grad psi}: the diffusivity-weighted
    average whose weights K+/(K-+K+), K-/(K-+K+) reduce to the arithmetic average of
    Eq. 46 when K is continuous and vanish with {K}_H when one side's K is zero, as the
    footnote to Eq. 45 requires of the solid charge transport into pores and separator.
  * Residual sign: R = storage + face/boundary terms - sources, i.e. the left minus the
    right side of the weak form, volume-integrated (units of the equation times m^3).
"""
from __future__ import annotations

import numpy as np

SQ3 = np.sqrt(3.0)
ALPHA = 0.5 * (1.0 + SQ3)   # trace weight of the node next to the face
BETA = 0.5 * (1.0 - SQ3)    # trace weight of the far node

# direction -> (DG0 cell axis, DG1 node axis, DG1 cell axis)
AXES = {"x": (2, 2, 5), "y": (1, 1, 4), "z": (0, 0, 3)}


def harmonic(a, b):
    """{D}_H = 2 D- D+ / (D- + D+) (Eq. 45); 0 when D- D+ <= 0 (a zero or sign-changing coefficient)."""
    prod = a * b
    ok = np.real(prod) > 0
    den = np.where(ok, a + b, 1.0)
    return np.where(ok, 2.0 * prod / den, 0.0)


def _sl(ndim, axis, s):
    idx = [slice(None)] * ndim
    idx[axis] = s
    return tuple(idx)


# ------------------------------------------------------------------------------------ DG0

def dg0_faces(Kc, psi, h, mag=False):
    """Interior-face part of Eq. 48 per cell: sum_Q A {K}_H (psi_P - psi_Q) / h, A = h^2.

    Kc, psi: (nz, ny, nx).  Each face is evaluated once and added to both cells.
    mag=True sums |flux| instead (the size of the terms, used for rounding tolerances)."""
    out = np.zeros(np.broadcast(Kc, psi).shape, dtype=np.result_type(Kc, psi, float))
    for d in ("x", "y", "z"):
        ax = AXES[d][0]
        n = out.shape[ax]
        if n < 2:
            continue
        lo, hi = _sl(3, ax, slice(0, n - 1)), _sl(3, ax, slice(1, n))
        flux = h * harmonic(Kc[lo], Kc[hi]) * (psi[lo] - psi[hi])
        if mag:
            flux = np.abs(flux)
        out[lo] += flux
        out[hi] -= -flux if mag else flux
    return out


def dg0_dirichlet(Kb, psi_b, psi_D, h):
    """Boundary mirror term of Eq. B1 for p = 0: A K (psi - psi_D) / (h/2)."""
    return h * h * Kb * (psi_b - psi_D) / (0.5 * h)


# ------------------------------------------------------------------------------------ DG1

def node(arr, d, a):
    """Nodal values with index a (0: xi = -1/sqrt3, 1: xi = +1/sqrt3) along direction d."""
    return np.take(arr, a, axis=AXES[d][1])


def trace(arr, d, side):
    """Values of the Q1 polynomial on the cell face xi = +1 (side=+1) or xi = -1 (side=-1)
    along direction d, at the face Gauss points (node axis d removed)."""
    v0, v1 = node(arr, d, 0), node(arr, d, 1)
    if side > 0:
        return ALPHA * v1 + BETA * v0
    return ALPHA * v0 + BETA * v1


def normal_grad(arr, d, h):
    """d psi / d x_d at the nodes of a line (constant along the line for Q1): sqrt(3)(psi_1 - psi_0)/h."""
    return SQ3 * (node(arr, d, 1) - node(arr, d, 0)) / h


def _scatter_nodes(out, d, val_at_1, val_at_0):
    na = AXES[d][1]
    out[_sl(out.ndim, na, 1)] += val_at_1
    out[_sl(out.ndim, na, 0)] += val_at_0


def dg1_volume(Kn, psi, h, mag=False):
    """int K grad psi . grad phi_m over each cell with 2x2x2 Gauss quadrature (collocated K).

    Per direction the term factorises into lines of two nodes:
    +-(3h/8)(K_0 + K_1)(psi_1 - psi_0) for the node at +-1/sqrt3."""
    out = np.zeros(np.broadcast(Kn, psi).shape, dtype=np.result_type(Kn, psi, float))
    for d in ("x", "y", "z"):
        flux = (3.0 * h / 8.0) * (node(Kn, d, 0) + node(Kn, d, 1)) * (node(psi, d, 1) - node(psi, d, 0))
        if mag:
            flux = np.abs(flux)
        _scatter_nodes(out, d, flux, flux if mag else -flux)
    return out


def dg1_faces(Kf, psi, h, penalty=1.0, mag=False):
    """Interior-face terms of Eq. 46 on every interior face, 2x2 Gauss points per face.

    Kf[d] = (K_plus_side, K_minus_side): the coefficient evaluated from the traced fields on
    each cell's xi = +1 and xi = -1 face of direction d, arrays shaped like ``trace``.
      -int {K}_H {d_n psi} [[v]]  +  penalty int {K}_H [[psi]].[[v]] / h
    The face weight is (h/2)^2 per point; test-function traces are ALPHA (near node), BETA (far)."""
    out = np.zeros(psi.shape, dtype=np.result_type(psi, *[k for pair in Kf.values() for k in pair], float))
    wf = 0.25 * h * h
    for d in ("x", "y", "z"):
        ca = AXES[d][2] - 1        # cell axis after removing the node axis of d
        Kp, Km = Kf[d]
        tp, tm = trace(psi, d, +1), trace(psi, d, -1)
        gr = normal_grad(psi, d, h)
        n = tp.shape[ca]
        if n < 2:
            continue
        nd = tp.ndim
        L, Rr = _sl(nd, ca, slice(0, n - 1)), _sl(nd, ca, slice(1, n))
        H = harmonic(Kp[L], Km[Rr])
        avg = H * 0.5 * (gr[L] + gr[Rr])
        pen = penalty * H * (tp[L] - tm[Rr]) / h
        fP = wf * (-avg + pen)           # enters cell P (left) as f * v-
        fQ = wf * (avg - pen)            # enters cell Q (right) as f * v+
        if mag:
            fP = wf * (np.abs(avg) + np.abs(pen))
            fQ = fP
        accP = np.zeros_like(tp, dtype=out.dtype)
        accQ = np.zeros_like(tp, dtype=out.dtype)
        accP[L] = fP
        accQ[Rr] = fQ
        # P: near node is a=1, far node a=0; Q: near node a=0, far node a=1
        if mag:
            _scatter_nodes(out, d, ALPHA * accP + abs(BETA) * accQ, abs(BETA) * accP + ALPHA * accQ)
        else:
            _scatter_nodes(out, d, ALPHA * accP + BETA * accQ, BETA * accP + ALPHA * accQ)
    return out


def dg1_boundary_flux(shape_like, d, side, fN, h, dtype=float, mag=False):
    """int_{face} f^N v for the face xi = side of direction d (f^N given at the face points,
    zero where the face is not a boundary face)."""
    out = np.zeros(shape_like, dtype=dtype)
    wf = 0.25 * h * h
    if mag:
        fN = np.abs(fN)
        _scatter_nodes(out, d, ALPHA * wf * fN, ALPHA * wf * fN)
        return out
    if side > 0:
        _scatter_nodes(out, d, ALPHA * wf * fN, BETA * wf * fN)
    else:
        _scatter_nodes(out, d, BETA * wf * fN, ALPHA * wf * fN)
    return out


def dg1_dirichlet(Kb, psi, psi_D, d, side, h):
    """Mirror term of Eq. B1 for p = 1 on the face xi = side of direction d of every cell:
    int (-(K grad psi).n v + K (psi - psi_D) v / (h/2)); restrict with a mask afterwards."""
    n_sign = float(side)
    tr = trace(psi, d, side)
    gr = normal_grad(psi, d, h)
    fN = -Kb * gr * n_sign + Kb * (tr - psi_D) / (0.5 * h)
    return dg1_boundary_flux(psi.shape, d, side, fN, h, dtype=np.result_type(psi, Kb, float))
