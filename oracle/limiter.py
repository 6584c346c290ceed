"""Vertex-based slope limiter for the DG1 (Q1) liquid species (App. B, after Kuzmin 2010).

Test infrastructure (see package docstring).

The paper observes that its DG1 scheme is not positivity-preserving (Sec. 2.6) and, in the 1D tests
of App. B, applies Kuzmin's vertex-based slope limiter after each step.  For the Q1 voxel
discretisation the rule reads, per voxel e and liquid species, on the conserved density
q = eps_L c (so that the limiter conserves every species exactly):

  * q_e is the voxel mean of q (the mean of the 8 nodal values: the Gauss nodes carry equal weight);
  * at every grid vertex v, q_v^max / q_v^min are the largest / smallest mean of the voxels that
    share v (only the voxels inside the domain);
  * at each of the 8 corners of e, the Q1 field's value u_c (extrapolated from the nodes with the
    1D weights (1 +- sqrt3)/2) gives alpha_c = min(1, (q_v^max - q_e)/(u_c - q_e)) if u_c > q_e,
    min(1, (q_v^min - q_e)/(u_c - q_e)) if u_c < q_e, and 1 if u_c = q_e;
  * alpha_e = min over the corners, and every node is replaced by q_e + alpha_e (q_n - q_e).

The limited nodal concentration is c_n = q_n / eps_L,n.  Corner values of the limited field lie in
the range of the surrounding means, and the Gauss nodes are convex combinations of the corners, so
non-negative means give non-negative nodal values.
"""
from __future__ import annotations

import numpy as np

from . import dg
from . import lis

# W[c, a]: weight of node a (0: xi = -1/sqrt3, 1: +1/sqrt3) in the Q1 value at corner c (0: xi = -1, 1: +1)
_W = np.array([[dg.ALPHA, dg.BETA], [dg.BETA, dg.ALPHA]])


def corner_values(u):
    """(2,2,2,nz,ny,nx) nodal Q1 values -> (2,2,2,nz,ny,nx) values at the cell corners (cz, cy, cx)."""
    return np.einsum("ia,jb,kc,abc...->ijk...", _W, _W, _W, u)


def vertex_bounds(mean):
    """Largest and smallest voxel mean around every grid vertex: two (nz+1, ny+1, nx+1) arrays."""
    nz, ny, nx = mean.shape
    hi = np.full((nz + 2, ny + 2, nx + 2), -np.inf)
    lo = np.full((nz + 2, ny + 2, nx + 2), np.inf)
    hi[1:-1, 1:-1, 1:-1] = mean
    lo[1:-1, 1:-1, 1:-1] = mean
    vmax = np.full((nz + 1, ny + 1, nx + 1), -np.inf)
    vmin = np.full((nz + 1, ny + 1, nx + 1), np.inf)
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                sl = (slice(dz, dz + nz + 1), slice(dy, dy + ny + 1), slice(dx, dx + nx + 1))
                vmax = np.maximum(vmax, hi[sl])
                vmin = np.minimum(vmin, lo[sl])
    return vmax, vmin


def limit_field(q):
    """Limit one Q1 field q (2,2,2,nz,ny,nx); returns (limited q, alpha per voxel)."""
    mean = q.mean(axis=(0, 1, 2))
    vmax, vmin = vertex_bounds(mean)
    nz, ny, nx = mean.shape
    uc = corner_values(q)
    alpha = np.ones_like(mean)
    for cz in (0, 1):
        for cy in (0, 1):
            for cx in (0, 1):
                d = uc[cz, cy, cx] - mean
                bmax = vmax[cz:cz + nz, cy:cy + ny, cx:cx + nx] - mean
                bmin = vmin[cz:cz + nz, cy:cy + ny, cx:cx + nx] - mean
                with np.errstate(divide="ignore", invalid="ignore"):
                    a = np.where(d > 0, np.minimum(1.0, bmax / d), np.where(d < 0, np.minimum(1.0, bmin / d), 1.0))
                alpha = np.minimum(alpha, a)
    return mean + alpha * (q - mean), alpha


def node_liquid_fraction(model, grid, U):
    """eps_L at every DG1 node, shape (2,2,2,nz,ny,nx)."""
    return lis.liquid_fraction(model, grid.phase[None, None, None], lis._solid_fractions(model, U))


def kuzmin_limit(model, grid, z):
    """Apply the limiter to every liquid species of a DG1 state z; returns the new flat state."""
    if model.order != 1:
        raise ValueError("the slope limiter acts on DG1 states")
    U = lis.unpack(model, grid, z)
    eL = node_liquid_fraction(model, grid, U)
    out = dict(U)
    for f in model.chem.liquid:
        q, _ = limit_field(eL * U[f])
        out[f] = q / eL
    return lis.pack(model, grid, out, dtype=z.dtype)


def limit_field_loops(q):
    """The same rule in plain loops over voxels and corners (for small grids)."""
    _, _, _, nz, ny, nx = q.shape
    mean = q.mean(axis=(0, 1, 2))
    out = q.copy()
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                alpha = 1.0
                for cz in (0, 1):
                    for cy in (0, 1):
                        for cx in (0, 1):
                            uc = 0.0
                            for az in (0, 1):
                                for ay in (0, 1):
                                    for ax in (0, 1):
                                        uc += _W[cz, az] * _W[cy, ay] * _W[cx, ax] * q[az, ay, ax, k, j, i]
                            around = [mean[kk, jj, ii]
                                      for kk in (k + cz - 1, k + cz) for jj in (j + cy - 1, j + cy)
                                      for ii in (i + cx - 1, i + cx)
                                      if 0 <= kk < nz and 0 <= jj < ny and 0 <= ii < nx]
                            d = uc - mean[k, j, i]
                            if d > 0:
                                alpha = min(alpha, (max(around) - mean[k, j, i]) / d)
                            elif d < 0:
                                alpha = min(alpha, (min(around) - mean[k, j, i]) / d)
                out[:, :, :, k, j, i] = mean[k, j, i] + alpha * (q[:, :, :, k, j, i] - mean[k, j, i])
    return out
