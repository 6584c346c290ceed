"""Shared set-up for the GPU parity tests: build/load libdgls, seeded cases, oracle references."""
import numpy as np

from oracle import chemistry as ch, init, lis, newton
from paper_2511_05233_gb300 import inputs

_BUILT = False


def ensure_built():
    global _BUILT
    import os

    from paper_2511_05233_gb300 import build

    if not _BUILT and not os.path.exists(build.LIB):
        build.build()
    _BUILT = True


def structure_with_collector(n, porosity, corr, seed):
    """The first structure from seed, seed + 1, ... that keeps a structure voxel on the current
    collector after the connectivity clean-up (small grids can lose all of it)."""
    for s in range(seed, seed + 100):
        phase = inputs.make_structure(n, porosity, corr, s)
        if np.any(phase[:, :, 0] == inputs.STRUCT):
            return phase
    raise RuntimeError("no structure touching x = 0")


def assert_state_close(model, grid, got, ref, rtol):
    """Max error per field relative to the magnitude of its kind of unknown: concentrations
    against the largest concentration, volume fractions against the largest volume fraction,
    potentials against the largest potential.  Newton stops on the row-scaled norm ||S R||, so a
    species present at 1e-12 mol/m^3 (S^2-) is only resolved to rtol times the concentration
    scale, not to rtol of itself."""
    lay = lis.layout(model, grid)

    def kind(f):
        return "pot" if f in ("PhiL", "PhiS") else ("eps" if f.startswith("eps_") else "conc")
    scale = {}
    for f, off, ln, s in lay:
        k = kind(f)
        scale[k] = max(scale.get(k, 0.0), np.abs(ref[off:off + ln]).max())
    for f, off, ln, s in lay:
        err = np.abs(got[off:off + ln] - ref[off:off + ln]).max() / (scale[kind(f)] + 1e-300)
        assert err <= rtol, (f, err)


def make_case(chem_name, order, n, porosity=0.6, corr=2.0, seed=1, noise_seed=2, f_C=0.5, potential_noise=0.0):
    """A seeded structure and a perturbed state built from the oracle's equilibrium (never from
    the CUDA path): returns (oracle model, grid, phase, z^n, z)."""
    chem = ch.reduced3() if chem_name == "reduced3" else ch.tradeoff()
    phase = structure_with_collector(n, porosity, corr, seed)
    grid = lis.Grid(phase, 1e-6)
    model = lis.Model(chem, order=order, f_C=f_C, eps_struct=1.0 - porosity)
    z0 = init.uniform_state(model, grid, init.equilibrium_fields(model))
    N = z0.size
    z = init.perturb(model, grid, z0, inputs.uniform_noise(N, noise_seed))
    if potential_noise:
        u = inputs.uniform_noise(N, noise_seed + 100)
        for f, off, ln, st in lis.layout(model, grid):
            if f in ("PhiL", "PhiS"):
                z[off:off + ln] += potential_noise * u[off:off + ln]
    return model, grid, phase, z0, z


def gpu_context(model, phase, h=1e-6, **kw):
    from paper_2511_05233_gb300 import dgls

    chem = dgls.TRADEOFF if model.chem.name == "tradeoff" else dgls.REDUCED3
    p = dgls.default_params(chem, model.order, f_C=model.f_C, eps_struct=model.eps_struct, T=model.T,
                            smooth=1 if model.smooth else 0, penalty=model.penalty, **kw)
    return dgls.Context(phase, h, p)


def to_dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def to_host(t):
    return t.detach().cpu().numpy()


def jvp_magnitude(model, grid, z, zn, t, dt, v):
    """|J| |v| with J the oracle's coloured complex-step Jacobian: the size of the products that
    sum to J v, against which rounding differences are measured."""
    J = newton.assemble_jacobian(model, grid, z, zn, t, dt)
    Ja = abs(J)
    return Ja @ np.abs(v), J
