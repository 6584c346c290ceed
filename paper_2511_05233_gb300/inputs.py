"""Seeded synthetic inputs shared by the CUDA path and the CPU oracle.

This module holds random numbers and voxel structures only: it contains none of
the model's arithmetic (no constants of the Li-S model, no equilibrium, no
residual).  Both sides of every parity test receive the arrays made here.

Structure recipe (stands in for the Blender/Worley cathode of Sec. 2.1, which is
not available): a Gaussian random field -- white noise N(0,1) from
``numpy.random.default_rng(seed)``, smoothed periodically in Fourier space by a
Gaussian of standard deviation ``corr_len/sqrt(2)`` voxels, which gives a field
with Gaussian covariance of length ``corr_len`` -- is thresholded at the
``porosity`` quantile over the cathode region: cells below the threshold are
macro-pores (phase 0), the rest coarse-grained active structure (phase 1).  The
last ``n_sep`` x-layers are the homogeneous separator (phase 2), which Sec. 2.1
treats as homogeneous regardless of dimensionality.  x is the transport
direction: the current collector is the x = 0 face, the lithium anode the
x = nx face.

Connectivity clean-up (6-connected): structure clusters that do not touch the
current collector carry no electronic current and are turned into pore; pore
clusters that do not reach the separator are cut off from the anode and are
turned into structure.
"""
from __future__ import annotations

import numpy as np

PORE, STRUCT, SEP = 0, 1, 2


def separator_layers(nx: int) -> int:
    """Number of homogeneous separator layers at the anode end of an nx-cell grid."""
    return max(2, nx // 8)


def gaussian_random_field(shape, corr_len: float, seed: int) -> np.ndarray:
    """Periodic Gaussian random field with Gaussian covariance of length ``corr_len`` voxels.

    ``shape`` is (nz, ny, nx) (x fastest in memory).
    """
    rng = np.random.default_rng(seed)
    w = rng.standard_normal(shape)
    sigma = corr_len / np.sqrt(2.0)
    what = np.fft.fftn(w)
    for ax, n in enumerate(shape):
        f = np.fft.fftfreq(n)
        filt = np.exp(-0.5 * (2.0 * np.pi * f * sigma) ** 2)
        sh = [1] * len(shape)
        sh[ax] = n
        what = what * filt.reshape(sh)
    return np.real(np.fft.ifftn(what))


def _label6(mask: np.ndarray):
    from scipy import ndimage

    st = ndimage.generate_binary_structure(3, 1)  # 6-connectivity
    return ndimage.label(mask, structure=st)


def make_structure(n, porosity: float, corr_len: float, seed: int, n_sep: int | None = None,
                   clean: bool = True, single_cluster: bool = False) -> np.ndarray:
    """Phase map uint8[nz, ny, nx] (x fastest) for a cubic (int n) or (nx, ny, nz) grid.

    Phases: 0 pore, 1 structure, 2 separator.  single_cluster: keep only the largest structure
    cluster touching the current collector (x = 0); smaller ones that touch it too become pore.
    """
    if np.isscalar(n):
        nx = ny = nz = int(n)
    else:
        nx, ny, nz = (int(v) for v in n)
    if n_sep is None:
        n_sep = separator_layers(nx)
    ncat = nx - n_sep
    if ncat < 1:
        raise ValueError("grid too short for a cathode")
    field = gaussian_random_field((nz, ny, nx), corr_len, seed)
    cat = field[:, :, :ncat]
    thr = np.quantile(cat, porosity)
    phase = np.full((nz, ny, nx), SEP, dtype=np.uint8)
    phase[:, :, :ncat] = np.where(cat < thr, PORE, STRUCT).astype(np.uint8)
    if clean:
        phase = clean_connectivity(phase, single_cluster)
    return phase


def clean_connectivity(phase: np.ndarray, single_cluster: bool = False) -> np.ndarray:
    """Flip floating structure clusters to pore and isolated pore clusters to structure; with
    single_cluster, also every structure cluster but the largest of those touching x = 0."""
    phase = phase.copy()
    lab, nlab = _label6(phase == STRUCT)
    if nlab:
        touching = np.unique(lab[:, :, 0])
        touching = touching[touching > 0]
        if single_cluster and touching.size > 1:
            sizes = np.bincount(lab.ravel(), minlength=nlab + 1)
            touching = touching[[int(np.argmax(sizes[touching]))]]
        keep = np.zeros(nlab + 1, dtype=bool)
        keep[touching] = True
        keep[0] = False
        floating = (lab > 0) & ~keep[lab]
        phase[floating] = PORE
    # pore clusters must reach the separator (or the anode face when there is none)
    liquid = (phase == PORE) | (phase == SEP)
    lab, nlab = _label6(liquid)
    if nlab:
        sep_labels = np.unique(lab[phase == SEP]) if np.any(phase == SEP) else np.unique(lab[:, :, -1])
        keep = np.zeros(nlab + 1, dtype=bool)
        keep[sep_labels] = True
        keep[0] = False
        isolated = (lab > 0) & ~keep[lab] & (phase == PORE)
        phase[isolated] = STRUCT
    return phase


def homogeneous_slab(nx: int, ny: int = 1, nz: int = 1, n_sep: int | None = None) -> np.ndarray:
    """Cathode made of structure cells only (the homogenised 1D model extruded in y and z)."""
    if n_sep is None:
        n_sep = separator_layers(nx)
    phase = np.full((nz, ny, nx), SEP, dtype=np.uint8)
    phase[:, :, : nx - n_sep] = STRUCT
    return phase


def uniform_noise(n: int, seed: int) -> np.ndarray:
    """U(-1, 1) draws, float64[n]; states are perturbed as value * (1 + 0.01 * noise)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=n)


def normal_noise(n: int, seed: int) -> np.ndarray:
    """N(0, 1) draws, float64[n] (direction vectors for Jacobian-vector products)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(n)


def batch_requests(n: int, seed: int):
    """Seeded mixed-size discharge requests: side, porosity, corr_len, C-rate, order."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        out.append(dict(side=int(rng.integers(24, 97)),
                        porosity=float(rng.uniform(0.4, 0.8)),
                        corr_len=float(rng.uniform(2.0, 8.0)),
                        f_C=float(np.exp(rng.uniform(np.log(0.1), np.log(2.0)))),
                        order=int(rng.integers(0, 2))))
    return out
