"""Complex-step Jacobian-vector products, coloured Jacobian assembly and Newton's method.

Test infrastructure (see package docstring).

JVP: J(z) v = Im R(z + i eps v) / eps with eps = 1e-30 (complex-step differentiation,
Squire & Trapp 1998): an exact directional derivative up to rounding, with no
subtractive cancellation, for any residual written with complex-analytic operations.

Newton (the role of PETSc ``newtonls`` in Sec. 2.7): exact linear solves with SuperLU,
backtracking line search on the scaled residual norm ||S R||_2 (Armijo 1e-4, step
halving, at most 10 cuts), convergence when ||S R||_2 <= max(rtol ||S R(z^n)||_2, atol sqrt(N))
(atol = 1e-12: an RMS scaled residual just above its rounding level, for steps that start almost converged),
or when the line search can no longer reduce ||S R||_2 and ||S R||_2 <= stall_rtol ||S R(z^n)||_2
(stall_rtol = 1e-8, PETSc's default relative tolerance: at large dt the rounding level of the scaled
residual lies above rtol ||S R(z^n)||_2); failure on the iteration limit, a failed line search above
that level or non-finite values.
Row scales S: Delta t / (M c_ref) for species and solid rows, Delta t / (M F c_ref)
for the two charge rows, M the cell (DG0) or node (DG1) volume.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import constants as K
from . import lis

CS_EPS = 1e-30


def jvp(model, grid, z, zn, t, dt, v, relax=False):
    zc = z.astype(complex) + 1j * CS_EPS * v
    return np.imag(lis.residual(model, grid, zc, zn.astype(complex), t, dt, relax)) / CS_EPS


def row_scales(model, grid, dt):
    M = grid.h ** 3 if model.order == 0 else grid.h ** 3 / 8.0
    s = np.empty(lis.n_dof(model, grid))
    for f, off, n, st in lis.layout(model, grid):
        if f in ("PhiL", "PhiS"):
            s[off:off + n] = dt / (M * K.F * K.C_REF)
        else:
            s[off:off + n] = dt / (M * K.C_REF)
    return s


def _dof_maps(model, grid):
    """Per field: (offset, len per node, struct-only, cell -> local index or -1)."""
    nn = 8 if model.order == 1 else 1
    maps = []
    comp = -np.ones(grid.n_cell, dtype=np.int64)
    comp[grid.struct_idx] = np.arange(grid.n_struct)
    for f, off, n, st in lis.layout(model, grid):
        loc = comp if st else np.arange(grid.n_cell)
        maps.append((f, off, n // nn, st, loc))
    return maps, nn


def assemble_jacobian(model, grid, z, zn, t, dt, relax=False):
    """Sparse J = dR/dz, column groups by the 7-colouring (i + 2j + 3k) mod 7 of the cells:
    two cells of one colour never share a face-neighbour stencil, so one complex-step JVP
    per (colour, field, node) recovers those columns exactly."""
    nz, ny, nx = grid.nz, grid.ny, grid.nx
    kk, jj, ii = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    color = ((ii + 2 * jj + 3 * kk) % 7).ravel()
    ci, cj, ck = ii.ravel(), jj.ravel(), kk.ravel()
    maps, nn = _dof_maps(model, grid)
    N = lis.n_dof(model, grid)
    # row -> cell
    row_cell = np.empty(N, dtype=np.int64)
    for f, off, ln, st, loc in maps:
        cells = grid.struct_idx if st else np.arange(grid.n_cell)
        for nd in range(nn):
            row_cell[off + nd * ln: off + (nd + 1) * ln] = cells
    # offset value (dx + 2dy + 3dz) -> offset vector
    offs = {0: (0, 0, 0), 1: (1, 0, 0), -1: (-1, 0, 0), 2: (0, 1, 0), -2: (0, -1, 0), 3: (0, 0, 1), -3: (0, 0, -1)}
    rows, cols, vals = [], [], []
    pc = color[row_cell]
    pi, pj, pk = ci[row_cell], cj[row_cell], ck[row_cell]
    for c in range(7):
        need = (c - pc) % 7
        need = np.where(need > 3, need - 7, need)
        dvec = np.array([offs[int(v)] for v in range(-3, 4)])
        dx, dy, dz = dvec[need + 3, 0], dvec[need + 3, 1], dvec[need + 3, 2]
        qi, qj, qk = pi + dx, pj + dy, pk + dz
        inb = (qi >= 0) & (qi < nx) & (qj >= 0) & (qj < ny) & (qk >= 0) & (qk < nz)
        qcell = np.where(inb, qi + nx * (qj + ny * qk), 0)
        for f, off, ln, st, loc in maps:
            seeded_cells = np.flatnonzero((color == c) & (loc >= 0))
            if seeded_cells.size == 0:
                continue
            qloc = np.where(inb, loc[qcell], -1)
            for nd in range(nn):
                v = np.zeros(N)
                v[off + nd * ln + loc[seeded_cells]] = 1.0
                Jv = jvp(model, grid, z, zn, t, dt, v, relax)
                ok = inb & (qloc >= 0) & (Jv != 0.0)
                r = np.flatnonzero(ok)
                rows.append(r)
                cols.append(off + nd * ln + qloc[r])
                vals.append(Jv[r])
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = np.concatenate(vals)
    return sp.csr_matrix((vals, (rows, cols)), shape=(N, N))


def _abs_jac_group(args):
    """|J| w restricted to the columns seeded in one (colour, field, node) group (see
    ``abs_jacobian_times``); a top-level function so that a spawn pool can run it."""
    model, grid, z, zn, t, dt, w, relax, c = args
    nz, ny, nx = grid.nz, grid.ny, grid.nx
    kk, jj, ii = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    color = ((ii + 2 * jj + 3 * kk) % 7).ravel()
    ci, cj, ck = ii.ravel(), jj.ravel(), kk.ravel()
    maps, nn = _dof_maps(model, grid)
    N = lis.n_dof(model, grid)
    row_cell = np.empty(N, dtype=np.int64)
    for f, off, ln, st, loc in maps:
        cells = grid.struct_idx if st else np.arange(grid.n_cell)
        for nd in range(nn):
            row_cell[off + nd * ln: off + (nd + 1) * ln] = cells
    offs = np.array([(0, 0, -1), (0, -1, 0), (-1, 0, 0), (0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)])
    pc = color[row_cell]
    need = (c - pc) % 7
    need = np.where(need > 3, need - 7, need)
    qi, qj, qk = ci[row_cell] + offs[need + 3, 0], cj[row_cell] + offs[need + 3, 1], ck[row_cell] + offs[need + 3, 2]
    inb = (qi >= 0) & (qi < nx) & (qj >= 0) & (qj < ny) & (qk >= 0) & (qk < nz)
    qcell = np.where(inb, qi + nx * (qj + ny * qk), 0)
    out = np.zeros(N)
    for f, off, ln, st, loc in maps:
        seeded = np.flatnonzero((color == c) & (loc >= 0))
        if seeded.size == 0:
            continue
        qloc = np.where(inb, loc[qcell], -1)
        for nd in range(nn):
            v = np.zeros(N)
            v[off + nd * ln + loc[seeded]] = 1.0
            Jv = jvp(model, grid, z, zn, t, dt, v, relax)
            ok = inb & (qloc >= 0)
            r = np.flatnonzero(ok)
            out[r] += np.abs(Jv[r]) * np.abs(w[off + nd * ln + qloc[r]])
    return out


def abs_jacobian_times(model, grid, z, zn, t, dt, w, relax=False, workers=1):
    """|J| |w| (entrywise absolute Jacobian times |w|) by the colouring of ``assemble_jacobian``:
    each seeded complex-step product gives, in every row, the one Jacobian entry of that row's
    seeded column.  workers > 1 spreads the seven colours over a spawn process pool."""
    tasks = [(model, grid, z, zn, t, dt, w, relax, c) for c in range(7)]
    if workers <= 1:
        parts = [_abs_jac_group(a) for a in tasks]
    else:
        import multiprocessing as mp

        with mp.get_context("spawn").Pool(min(workers, 7)) as pool:
            parts = pool.map(_abs_jac_group, tasks)
    return np.sum(parts, axis=0)


@dataclass
class NewtonInfo:
    converged: bool
    iterations: int
    norm0: float
    norm: float
    reason: str = ""


def newton(model, grid, zn, t, dt, z0=None, rtol=1e-10, max_it=25, relax=False, max_cuts=10, atol=1e-12,
           stall_rtol=1e-8):
    """Solve R(z; z^n, t, dt) = 0 for z = z^{n+1} starting from z0 (default z^n)."""
    S = row_scales(model, grid, dt)
    z = (zn if z0 is None else z0).astype(float).copy()
    Rz = lis.residual(model, grid, z, zn, t, dt, relax)
    nrm = float(np.linalg.norm(S * Rz))
    n0 = nrm
    if not np.isfinite(nrm):
        return z, NewtonInfo(False, 0, n0, nrm, "nonfinite")
    it = 0
    floor = atol * np.sqrt(z.size)
    while True:
        if nrm <= max(rtol * n0, floor) or nrm == 0.0:
            return z, NewtonInfo(True, it, n0, nrm)
        if it >= max_it:
            return z, NewtonInfo(False, it, n0, nrm, "max_it")
        J = assemble_jacobian(model, grid, z, zn, t, dt, relax)
        delta = spla.spsolve(J.tocsc(), -Rz)
        if not np.all(np.isfinite(delta)):
            return z, NewtonInfo(False, it, n0, nrm, "nonfinite")
        lam = 1.0
        for _ in range(max_cuts + 1):
            zt = z + lam * delta
            Rt = lis.residual(model, grid, zt, zn, t, dt, relax)
            nt = float(np.linalg.norm(S * Rt))
            if np.isfinite(nt) and nt <= (1.0 - 1e-4 * lam) * nrm:
                break
            lam *= 0.5
        else:
            # no decrease possible: stagnation at the rounding level of the scaled residual counts
            # as converged within stall_rtol (PETSc's default relative tolerance), else a failure
            if np.isfinite(nrm) and nrm <= stall_rtol * n0:
                return z, NewtonInfo(True, it, n0, nrm)
            return z, NewtonInfo(False, it, n0, nrm, "line_search")
        z, Rz, nrm = zt, Rt, nt
        it += 1


def implicit_euler_step(model, grid, zn, t, dt, **kw):
    """z^{n+1} with (z^{n+1} - z^n)/dt = F(z^{n+1}) (Eq. 50); T_H taken at t^{n+1}."""
    return newton(model, grid, zn, t + dt, dt, **kw)
