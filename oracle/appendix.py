"""App. A benchmarks of the spatial DG discretisation, in 1D (grids of shape (1, 1, nx)).

Test infrastructure (see package docstring).  The residuals reuse the generic operators of
``oracle.dg`` (the same ones the Li-S residual is built from), with the Dirichlet mirror
terms of Eq. B1.

A1 (Eqs. B2-B3): diffusion across a discontinuity, no-flux ends.  The analytic solution is
   written with erf(x / (2 sqrt(D t))): Eq. B3 prints erf(x / (4 D t)), which is not
   dimensionless; the Laplace-transform solution it cites has 2 sqrt(D t).  Eq. B3 holds on
   an infinite line; on the paper's finite domain it is off by ~5e-4 (rms) at t = 0.8 s,
   which hides the discretisation error, so the error is evaluated at t = 0.1 s, where the
   diffusion length 2 sqrt(D_R t) = 0.02 m is far from the ends at +-0.1 m.
A3 (Eqs. B7-B9): the Cherniha predator-prey system with lambda_2 = 0 (an elliptic constraint
   like the potential equations), Dirichlet ends.  Time integration uses Richardson
   extrapolation of implicit Euler (Eq. 54) so that the spatial order is not masked by the
   first-order time error at affordable step counts.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla
from scipy.special import erf

from . import dg

CS = 1e-30


def _cell_centres(n, x0, x1):
    h = (x1 - x0) / n
    return x0 + h * (np.arange(n) + 0.5), h


def node_coords(n, x0, x1):
    """x of the two Gauss nodes per cell, shape (2, n)."""
    xc, h = _cell_centres(n, x0, x1)
    off = h / (2.0 * np.sqrt(3.0))
    return np.stack([xc - off, xc + off]), h


def l2_error(order, vals, n, x0, x1, exact):
    """(1/L int (u_h - u)^2 dx)^(1/2) with a 5-point Gauss rule per cell, u_h the DG polynomial
    (piecewise constant for DG0, linear through the two Gauss nodes for DG1) -- the norm of
    Eqs. B4, B6, B9."""
    L = x1 - x0
    h = L / n
    gx, gw = np.polynomial.legendre.leggauss(5)
    xc = x0 + h * (np.arange(n) + 0.5)
    tot = 0.0
    for xi, w in zip(gx, gw):
        x = xc + 0.5 * h * xi
        if order == 0:
            uh = vals.reshape(n)
        else:
            v = vals.reshape(2, n)
            s = np.sqrt(3.0)
            l0 = (xi - 1.0 / s) / (-2.0 / s)
            l1 = (xi + 1.0 / s) / (2.0 / s)
            uh = l0 * v[0] + l1 * v[1]
        tot += np.sum(0.5 * h * w * (uh - exact(x)) ** 2)
    return float(np.sqrt(tot / L))


def to_dg1(vals2):
    """(2, n) nodal values along x -> DG1 array (2, 2, 2, 1, 1, n) constant in y and z."""
    n = vals2.shape[1]
    out = np.empty((2, 2, 2, 1, 1, n), dtype=vals2.dtype)
    out[...] = vals2.reshape(1, 1, 2, 1, 1, n)
    return out


def _jacobian_1d(res, u, nper):
    """Complex-step Jacobian of a 1D residual whose cells couple to neighbours only:
    colour cells by index mod 3, one JVP per (colour, local dof)."""
    N = u.size
    ncell = N // nper
    rows, cols, vals = [], [], []
    cell_of = np.arange(N) // nper
    loc_of = np.arange(N) % nper
    for c in range(3):
        for l in range(nper):
            v = np.zeros(N)
            sel = (cell_of % 3 == c) & (loc_of == l)
            v[sel] = 1.0
            Jv = np.imag(res(u + 1j * CS * v)) / CS
            # row in cell P couples to the seeded cell among P-1, P, P+1
            for d in (-1, 0, 1):
                q = cell_of + d
                ok = (q >= 0) & (q < ncell) & (q % 3 == c) & (Jv != 0)
                r = np.flatnonzero(ok)
                rows.append(r)
                cols.append(q[r] * nper + l)
                vals.append(Jv[r])
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N))


def _newton(res, u0, tol=1e-13, max_it=30):
    """Newton until the update is below tol relative to the state."""
    u = u0.copy()
    for _ in range(max_it):
        r = np.real(res(u))
        J = _jacobian_1d(res, u, _newton.nper)
        du = spla.spsolve(J.tocsc(), -r)
        u = u + du
        if np.linalg.norm(du) <= tol * (1.0 + np.linalg.norm(u)):
            return u
    raise RuntimeError("App. A Newton did not converge")


# --------------------------------------------------------------------------------------- A1

A1 = dict(L=0.2, T=1.0, DL=1e-4, DR=1e-3, cL=0.0, cR=1.0, t_eval=0.1, dt=1e-4)


def a1_exact(x, t, p=A1):
    DL, DR, cL, cR = p["DL"], p["DR"], p["cL"], p["cR"]
    cm = (np.sqrt(DL) * cL + np.sqrt(DR) * cR) / (np.sqrt(DL) + np.sqrt(DR))
    left = cL + (cm - cL) * (1.0 - erf(-x / (2.0 * np.sqrt(DL * t))))
    right = cm + (cR - cm) * erf(x / (2.0 * np.sqrt(DR * t)))
    return np.where(x < 0, left, right)


def a1_solve(order, n, p=A1, t_eval=None, dt=None):
    """Implicit Euler of Eq. B2; the problem is linear, so one LU serves all steps.
    Returns the L2 error of Eq. B4 at t_eval (Gauss quadrature on the nodes)."""
    t_eval = p["t_eval"] if t_eval is None else t_eval
    dt = p["dt"] if dt is None else dt
    L = p["L"]
    if order == 0:
        xc, h = _cell_centres(n, -L / 2, L / 2)
        D = np.where(xc < 0, p["DL"], p["DR"]).reshape(1, 1, n)
        c0 = np.where(xc < 0, p["cL"], p["cR"]).reshape(1, 1, n)
        M = h ** 3

        def op(c):
            return dg.dg0_faces(D, c.reshape(1, 1, n), h).ravel()
        xq = xc.reshape(1, n)
        wq = np.full((1, n), h)
    else:
        xn, h = node_coords(n, -L / 2, L / 2)
        side = np.where((xn[0] + xn[1]) / 2 < 0, 0, 1)
        D2 = np.where(side == 0, p["DL"], p["DR"]) * np.ones((2, 1))
        D = to_dg1(D2)
        c0 = to_dg1(np.where(side == 0, p["cL"], p["cR"]) * np.ones((2, 1)))
        M = h ** 3 / 8.0
        Kf = {}
        for d in ("x", "y", "z"):
            Kf[d] = (dg.trace(D, d, +1), dg.trace(D, d, -1))

        def op(c):
            cc = c.reshape(D.shape)
            return (dg.dg1_volume(D, cc, h) + dg.dg1_faces(Kf, cc, h)).ravel()
        xq = xn
        wq = np.full((2, n), h / 2.0)
    c0 = c0.ravel().astype(float)
    N = c0.size
    nper = N // n
    # cell-major ordering for the colouring: position i*nper + k holds node-major entry k*n + i
    perm = np.arange(N).reshape(nper, n).T.ravel()
    inv = np.empty_like(perm)
    inv[perm] = np.arange(N)

    def res(ucm):
        return op(ucm[inv])[perm]
    Kcm = _jacobian_1d(res, np.zeros(N), nper)
    K = Kcm[inv][:, inv]
    A = (sp.identity(N) * (M / dt) + K).tocsc()
    lu = spla.splu(A)
    c = c0.copy()
    nsteps = int(round(t_eval / dt))
    for _ in range(nsteps):
        c = lu.solve(M / dt * c)
    if order == 1:
        vals = c.reshape(D.shape)[0, 0]          # (2, 1, 1, n) -> x nodes
        vals = vals.reshape(2, n)
    else:
        vals = c.reshape(1, n)
    return l2_error(order, vals, n, -L / 2, L / 2, lambda x: a1_exact(x, t_eval, p))


# --------------------------------------------------------------------------------------- A3

A3 = dict(A1=1.0, A2=2.0, lam1=11.0, lam2=0.0, B=0.1, C=0.1, K=0.2)


def a3_beta(p=A3):
    return (p["A1"] - p["A2"]) / (p["lam1"] - p["lam2"])


def a3_length(p=A3):
    return np.pi / np.sqrt(-a3_beta(p) * p["lam1"])


def a3_exact(x, t, p=A3):
    b = a3_beta(p)
    s = np.sin(np.sqrt(-b * p["lam1"]) * x) * np.exp(b * t)
    c1 = p["A1"] / p["B"] + p["K"] / ((p["A1"] - p["A2"]) * p["B"]) * s
    c2 = p["K"] / ((p["A2"] - p["A1"]) * p["C"]) * s
    return c1, c2


def a3_solve(order, n, t_eval=2.0, dt=0.1, p=A3):
    """Eq. B7 with Dirichlet ends (mirror terms, Eq. B1); returns the error of Eq. B9 at t_eval."""
    L = a3_length(p)
    D1 = 1.0
    if order == 0:
        xc, h = _cell_centres(n, 0.0, L)
        shp = (1, 1, n)
        M = h ** 3
        xq, wq = xc.reshape(1, n), np.full((1, n), h)
        c1, c2 = a3_exact(xc, 0.0, p)
        u0 = np.concatenate([c1, c2])
        Kc = np.ones(shp)
    else:
        xn, h = node_coords(n, 0.0, L)
        shp = (2, 2, 2, 1, 1, n)
        M = h ** 3 / 8.0
        xq, wq = xn, np.full((2, n), h / 2.0)
        c1, c2 = a3_exact(xn, 0.0, p)
        u0 = np.concatenate([to_dg1(c1).ravel(), to_dg1(c2).ravel()])
        Kc = np.ones(shp)
        Kf = {d: (dg.trace(Kc, d, +1), dg.trace(Kc, d, -1)) for d in ("x", "y", "z")}
    ncomp = int(np.prod(shp))
    c1D = p["A1"] / p["B"]

    def spatial(u):
        a, b = u[:ncomp].reshape(shp), u[ncomp:].reshape(shp)
        out = []
        for f, fD in ((a, c1D), (b, 0.0)):
            if order == 0:
                r = dg.dg0_faces(D1 * Kc, f, h)
                r[..., 0] += dg.dg0_dirichlet(D1, f[..., 0], fD, h)
                r[..., -1] += dg.dg0_dirichlet(D1, f[..., -1], fD, h)
            else:
                r = dg.dg1_volume(D1 * Kc, f, h) + dg.dg1_faces(Kf, f, h)
                first = np.zeros(shp[3:], dtype=bool)
                first[..., 0] = True
                last = np.zeros(shp[3:], dtype=bool)
                last[..., -1] = True
                r = r + dg.dg1_dirichlet(D1 * dg.trace(Kc, "x", -1) * first, f, fD, "x", -1, h)
                r = r + dg.dg1_dirichlet(D1 * dg.trace(Kc, "x", +1) * last, f, fD, "x", +1, h)
            out.append(r)
        ra, rb = out
        ra = ra - M * a * (p["A1"] - p["B"] * a - p["C"] * b)
        rb = rb - M * b * (p["A2"] - p["B"] * a - p["C"] * b)
        return ra, rb

    # dofs per cell: interleave is not needed; colour by cell works on each half separately
    nper_half = ncomp // n
    u = u0.copy()

    def step_wrapped(u, dtt):
        # reorder to cell-major so that the cell colouring applies: (n, 2*nper_half)
        perm = np.concatenate([np.arange(ncomp).reshape(-1, n).T, ncomp + np.arange(ncomp).reshape(-1, n).T], axis=1).ravel()
        inv = np.empty_like(perm)
        inv[perm] = np.arange(perm.size)

        def res_cm(vcm):
            v = vcm[inv]
            ra, rb = spatial(v)
            a, a_old = v[:ncomp], u[:ncomp]
            b, b_old = v[ncomp:], u[ncomp:]
            ra = ra.ravel() + M * p["lam1"] * (a - a_old) / dtt
            rb = rb.ravel() + M * p["lam2"] * (b - b_old) / dtt
            return np.concatenate([ra, rb])[perm]
        _newton.nper = 2 * nper_half
        ucm = _newton(res_cm, u[perm])
        return ucm[inv]

    nsteps = int(round(t_eval / dt))
    for _ in range(nsteps):
        uC = step_wrapped(u, dt)
        uF = step_wrapped(step_wrapped(u, dt / 2), dt / 2)
        u = 2.0 * uF - uC
    a, b = u[:ncomp].reshape(shp), u[ncomp:].reshape(shp)
    if order == 1:
        a, b = a[0, 0].reshape(2, n), b[0, 0].reshape(2, n)
    else:
        a, b = a.reshape(1, n), b.reshape(1, n)
    return (l2_error(order, a, n, 0.0, L, lambda x: a3_exact(x, t_eval, p)[0])
            + l2_error(order, b, n, 0.0, L, lambda x: a3_exact(x, t_eval, p)[1]))


def order_fit(ns, errs):
    """Least-squares slope of log(err) against log(1/n)."""
    x = np.log(1.0 / np.asarray(ns, float))
    y = np.log(np.asarray(errs, float))
    return float(np.polyfit(x, y, 1)[0])
