"""ctypes binding of libdgls.so (include/dgls.h): argument marshalling only.

Device buffers are torch CUDA tensors (float64, contiguous); every compute step runs in the
library's CUDA kernels.  There is no CPU fallback: ``lib()`` raises if the library is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

OK, ERR_ARG, ERR_OOM, ERR_CUDA, ERR_NOCONV, ERR_NONFINITE, ERR_TIMEOUT, ERR_ABORTED = 0, -1, -2, -3, -4, -5, -6, -7
STATUS = {0: "DG_OK", -1: "DG_ERR_ARG", -2: "DG_ERR_OOM", -3: "DG_ERR_CUDA", -4: "DG_ERR_NOCONV",
          -5: "DG_ERR_NONFINITE", -6: "DG_ERR_TIMEOUT", -7: "DG_ERR_ABORTED"}
REDUCED3, TRADEOFF = 0, 1
FP64, MIXED = 0, 1
NAIVE, H211B, FIXED = 0, 1, 2


class Structure(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("h", C.c_double),
                ("phase", C.POINTER(C.c_uint8))]


class Params(C.Structure):
    _fields_ = [("order", C.c_int32), ("chemistry", C.c_int32), ("T", C.c_double), ("f_C", C.c_double),
                ("j_el", C.c_double), ("eps_struct", C.c_double), ("penalty", C.c_double), ("smooth", C.c_int32),
                ("precision", C.c_int32), ("gmres_restart", C.c_int32), ("gmres_max_it", C.c_int32),
                ("newton_rtol", C.c_double), ("newton_atol", C.c_double), ("newton_max_it", C.c_int32),
                ("eta_max", C.c_double), ("eta_min", C.c_double), ("hbm_budget_bytes", C.c_int64),
                ("preconditioner", C.c_int32), ("mg_cycles", C.c_int32), ("precond_every", C.c_int32),
                ("newton_stall_rtol", C.c_double), ("reorth", C.c_int32), ("species_mg", C.c_int32),
                ("jvp_form", C.c_int32)]


class StepInfo(C.Structure):
    _fields_ = [("converged", C.c_int32), ("newton_iterations", C.c_int32), ("gmres_iterations", C.c_int32),
                ("residual_evals", C.c_int32), ("jvp_evals", C.c_int32), ("norm0", C.c_double), ("norm", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ControllerState(C.Structure):
    _fields_ = [("t", C.c_double), ("dt", C.c_double), ("err_prev", C.c_double), ("dt_prev", C.c_double),
                ("sct", C.c_int32), ("halvings", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class DischargeOpts(C.Structure):
    _fields_ = [("controller", C.c_int32), ("t0", C.c_double), ("dt0", C.c_double), ("dt_min", C.c_double),
                ("dt_max", C.c_double), ("tol", C.c_double), ("cutoff_V", C.c_double), ("t_end", C.c_double),
                ("max_steps", C.c_int32), ("max_halvings", C.c_int32), ("replay_dt", C.POINTER(C.c_double)),
                ("n_replay", C.c_int32), ("limiter", C.c_int32), ("resume", C.POINTER(ControllerState))]


class Curve(C.Structure):
    _fields_ = [("n_max", C.c_int32), ("n", C.c_int32), ("t", C.POINTER(C.c_double)), ("dt", C.POINTER(C.c_double)),
                ("U_cell", C.POINTER(C.c_double)), ("c_m", C.POINTER(C.c_double)),
                ("newton_its", C.POINTER(C.c_int32)), ("gmres_its", C.POINTER(C.c_int32)),
                ("status", C.c_int32), ("attempts", C.c_int32), ("failures", C.c_int32),
                ("checkpoint", C.POINTER(ControllerState))]


_LIB = None
_P = C.c_void_p


def lib_path():
    return _build.LIB


def lib():
    """Load libdgls.so (raises if it has not been built: there is no fallback)."""
    global _LIB
    if _LIB is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} not built; run paper_2511_05233_gb300.build.build()")
        L = C.CDLL(path)
        sig = {
            "dg_params_default": (C.c_int, [C.POINTER(Params), C.c_int32, C.c_int32]),
            "dg_setup": (C.c_int, [C.POINTER(Structure), C.POINTER(Params), _P, C.POINTER(_P)]),
            "dg_setup_in": (C.c_int, [C.POINTER(Structure), C.POINTER(Params), _P, _P, C.c_int64, C.POINTER(_P)]),
            "dg_workspace_estimate": (C.c_int, [C.POINTER(Structure), C.POINTER(Params), C.POINTER(C.c_int64)]),
            "dg_destroy": (C.c_int, [_P]),
            "dg_last_error": (C.c_char_p, [_P]),
            "dg_layout": (C.c_int, [_P, C.POINTER(C.c_int64), C.POINTER(C.c_int32), C.POINTER(C.c_int64),
                                    C.POINTER(C.c_int64)]),
            "dg_equilibrium_state": (C.c_int, [_P, _P]),
            "dg_relax": (C.c_int, [_P, _P, C.c_double, C.c_int32]),
            "dg_residual": (C.c_int, [_P, _P, _P, C.c_double, C.c_double, _P]),
            "dg_residual_noalloc": (C.c_int, [_P, _P, _P, C.c_double, C.c_double, _P]),
            "dg_jvp": (C.c_int, [_P, _P, C.c_double, C.c_double, _P, _P]),
            "dg_jvp_fused": (C.c_int, [_P, _P, C.c_double, C.c_double, C.c_int32, _P, _P]),
            "dg_block_jacobi": (C.c_int, [_P, _P, C.c_double, C.c_double, _P, _P]),
            "dg_row_scales": (C.c_int, [_P, C.c_double, _P]),
            "dg_step": (C.c_int, [_P, _P, _P, C.c_double, C.c_double, C.POINTER(StepInfo)]),
            "dg_step_host": (C.c_int, [_P, _P, _P, C.c_double, C.c_double, C.POINTER(StepInfo)]),
            "dg_cell_voltage": (C.c_int, [_P, _P, C.POINTER(C.c_double)]),
            "dg_ledger": (C.c_int, [_P, _P, C.POINTER(C.c_double)]),
            "dg_discharge": (C.c_int, [_P, _P, C.POINTER(DischargeOpts), C.POINTER(Curve)]),
            "dg_profile": (C.c_int, [_P, C.c_int32]),
            "dg_profile_read": (C.c_int, [_P, C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
            "dg_launch_count": (C.c_int64, [_P]),
            "dg_limit": (C.c_int, [_P, _P]),
            "dg_reorth_count": (C.c_int64, [_P]),
            "dg_workspace_bytes": (C.c_int64, [_P]),
            "dg_batch_create": (C.c_int, [C.POINTER(_P), C.c_int32, _P, C.POINTER(_P)]),
            "dg_batch_destroy": (C.c_int, [_P]),
            "dg_batch_last_error": (C.c_char_p, [_P]),
            "dg_batch_launch_count": (C.c_int64, [_P]),
            "dg_batch_jvp": (C.c_int, [_P, C.POINTER(_P), C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_int32,
                                       C.POINTER(_P), C.POINTER(_P)]),
            "dg_batch_residual": (C.c_int, [_P, C.POINTER(_P), C.POINTER(_P), C.POINTER(C.c_double),
                                            C.POINTER(C.c_double), C.POINTER(_P)]),
            "dg_batch_autotune": (C.c_int, [_P, C.POINTER(_P), C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_int32,
                                            C.POINTER(_P), C.POINTER(_P), C.POINTER(C.c_int32)]),
            "dg_batch_step": (C.c_int, [_P, C.POINTER(_P), C.POINTER(_P), C.POINTER(C.c_double), C.POINTER(C.c_double),
                                        C.POINTER(StepInfo), C.POINTER(C.c_int32)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


class DGError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def default_params(chemistry=TRADEOFF, order=0, **kw):
    p = Params()
    st = lib().dg_params_default(C.byref(p), chemistry, order)
    if st != OK:
        raise DGError(st, "dg_params_default")
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def _ptr(t):
    """Device pointer of a contiguous float64 torch CUDA tensor."""
    import torch

    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError("expected a contiguous float64 CUDA tensor")
    return C.c_void_p(t.data_ptr())


def _structure(phase, h):
    ph = np.ascontiguousarray(phase, dtype=np.uint8)
    if ph.ndim != 3:
        raise ValueError("phase must be (nz, ny, nx)")
    nz, ny, nx = ph.shape
    return ph, Structure(nx, ny, nz, float(h), ph.ctypes.data_as(C.POINTER(C.c_uint8)))


def workspace_estimate(phase, h, params):
    """dg_workspace_estimate: device bytes a context for this structure and parameters needs."""
    ph, s = _structure(phase, h)
    n = C.c_int64()
    st = lib().dg_workspace_estimate(C.byref(s), C.byref(params), C.byref(n))
    if st != OK:
        raise DGError(st, "dg_workspace_estimate")
    return int(n.value)


class Context:
    """One discretised cell (structure + parameters) with its device workspaces (its own cudaMalloc
    allocations, or carved from `workspace`, a CUDA uint8 tensor the caller keeps and may reuse)."""

    def __init__(self, phase, h, params, stream=None, workspace=None):
        import torch

        self._lib = lib()
        ph, s = _structure(phase, h)
        self._phase = ph
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self.workspace = workspace
        h_ = C.c_void_p()
        if workspace is not None:
            if not (workspace.is_cuda and workspace.dtype == torch.uint8 and workspace.is_contiguous()):
                raise TypeError("workspace must be a contiguous uint8 CUDA tensor")
            st = self._lib.dg_setup_in(C.byref(s), C.byref(params), C.c_void_p(stream.cuda_stream),
                                       C.c_void_p(workspace.data_ptr()), workspace.numel(), C.byref(h_))
        else:
            st = self._lib.dg_setup(C.byref(s), C.byref(params), C.c_void_p(stream.cuda_stream), C.byref(h_))
        if st != OK:
            raise DGError(st, "dg_setup (no structure voxel at x = 0, bad arguments or out of memory)")
        self._h = h_
        self.params = params
        n = C.c_int64()
        nf = C.c_int32()
        off = (C.c_int64 * 10)()
        ln = (C.c_int64 * 10)()
        self._check(self._lib.dg_layout(self._h, C.byref(n), C.byref(nf), off, ln))
        self.n_dof = n.value
        self.n_fields = nf.value
        self.offsets = list(off)[: nf.value]
        self.lengths = list(ln)[: nf.value]

    def _check(self, st):
        if st != OK:
            raise DGError(st, self._lib.dg_last_error(self._h).decode())
        return st

    def close(self):
        if getattr(self, "_h", None):
            self._lib.dg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- device-buffer calls
    def new_state(self):
        import torch

        return torch.empty(self.n_dof, dtype=torch.float64, device="cuda")

    def equilibrium_state(self, z):
        self._check(self._lib.dg_equilibrium_state(self._h, _ptr(z)))
        return z

    def relax(self, z, dt=0.1, n_steps=40):
        self._check(self._lib.dg_relax(self._h, _ptr(z), dt, n_steps))
        return z

    def residual(self, z, zold, t, dt, out):
        self._check(self._lib.dg_residual(self._h, _ptr(z), _ptr(zold), t, dt, _ptr(out)))
        return out

    def residual_noalloc(self, z, zold, t, dt, out):
        """dg_residual_noalloc: DG0 residual with static scratch (no allocation, no workspace use)."""
        self._check(self._lib.dg_residual_noalloc(self._h, _ptr(z), _ptr(zold), t, dt, _ptr(out)))
        return out

    def jvp(self, z, t, dt, v, out):
        self._check(self._lib.dg_jvp(self._h, _ptr(z), t, dt, _ptr(v), _ptr(out)))
        return out

    def jvp_fused(self, z, t, dt, v, out):
        """dg_jvp_fused: the one-launch matrix-free product; FP64 for float64 v/out, FP32 (mixed
        contexts) for float32 v/out."""
        import torch

        if v.dtype == torch.float32:
            prec = MIXED
            ok = out.dtype == torch.float32 and v.is_cuda and out.is_cuda and v.is_contiguous() and out.is_contiguous()
            if not ok:
                raise TypeError("expected contiguous float32 CUDA tensors for v and out")
            vp, op = C.c_void_p(v.data_ptr()), C.c_void_p(out.data_ptr())
        else:
            prec = FP64
            vp, op = _ptr(v), _ptr(out)
        self._check(self._lib.dg_jvp_fused(self._h, _ptr(z), t, dt, prec, vp, op))
        return out

    def block_jacobi(self, z, t, dt, v, out):
        self._check(self._lib.dg_block_jacobi(self._h, _ptr(z), t, dt, _ptr(v), _ptr(out)))
        return out

    def row_scales(self, dt, out):
        self._check(self._lib.dg_row_scales(self._h, dt, _ptr(out)))
        return out

    def step(self, zn, z, t, dt, check=True):
        info = StepInfo()
        st = self._lib.dg_step(self._h, _ptr(zn), _ptr(z), t, dt, C.byref(info))
        if check and st != OK:
            self._check(st)
        return st, info

    def step_host(self, zn_host, z_host, t, dt, check=True):
        zn_host = np.ascontiguousarray(zn_host, dtype=np.float64)
        if z_host.dtype != np.float64 or not z_host.flags.c_contiguous:
            raise TypeError("z_host must be a contiguous float64 array")
        info = StepInfo()
        st = self._lib.dg_step_host(self._h, zn_host.ctypes.data_as(C.c_void_p), z_host.ctypes.data_as(C.c_void_p),
                                    t, dt, C.byref(info))
        if check and st != OK:
            self._check(st)
        return st, info

    def cell_voltage(self, z):
        u = C.c_double()
        self._check(self._lib.dg_cell_voltage(self._h, _ptr(z), C.byref(u)))
        return u.value

    def ledger(self, z):
        out = (C.c_double * 5)()
        self._check(self._lib.dg_ledger(self._h, _ptr(z), out))
        return list(out)

    def discharge(self, z, controller=NAIVE, dt0=1e-3, dt_min=1e-6, dt_max=10.0, tol=1e-5, cutoff_V=1.9,
                  t_end=0.0, max_steps=100000, max_halvings=30, replay_dt=None, t0=0.0, limiter=False,
                  resume=None):
        """Run dg_discharge; res["checkpoint"] is the controller state at return (a dict), which
        resume= takes to continue the run from the returned state."""
        n_max = max_steps if replay_dt is None else len(replay_dt)
        rs = None
        if resume is not None:
            rs = ControllerState(**resume)
        arr = {k: np.zeros(n_max) for k in ("t", "dt", "U_cell", "c_m")}
        nit = np.zeros(n_max, dtype=np.int32)
        git = np.zeros(n_max, dtype=np.int32)
        rp = None
        if replay_dt is not None:
            rp = np.ascontiguousarray(replay_dt, dtype=np.float64)
        o = DischargeOpts(controller, t0, dt0, dt_min, dt_max, tol, cutoff_V, t_end, max_steps, max_halvings,
                          rp.ctypes.data_as(C.POINTER(C.c_double)) if rp is not None else None,
                          len(rp) if rp is not None else 0, 1 if limiter else 0,
                          C.pointer(rs) if rs is not None else None)
        ck = ControllerState()
        cv = Curve(n_max, 0, *[arr[k].ctypes.data_as(C.POINTER(C.c_double)) for k in ("t", "dt", "U_cell", "c_m")],
                   nit.ctypes.data_as(C.POINTER(C.c_int32)), git.ctypes.data_as(C.POINTER(C.c_int32)), 0, 0, 0,
                   C.pointer(ck))
        st = self._lib.dg_discharge(self._h, _ptr(z), C.byref(o), C.byref(cv))
        n = cv.n
        res = {k: v[:n].copy() for k, v in arr.items()}
        res.update(newton_its=nit[:n].copy(), gmres_its=git[:n].copy(), status=STATUS.get(st, st),
                   attempts=cv.attempts, failures=cv.failures, checkpoint=ck.as_dict())
        if st not in (OK, ERR_ABORTED, ERR_NOCONV):
            self._check(st)
        return res

    PROFILE_CATEGORIES = ("residual", "jvp", "precond_build", "precond_apply", "krylov")

    def profile(self, enable=True):
        self._check(self._lib.dg_profile(self._h, 1 if enable else 0))

    def profile_read(self):
        ms = (C.c_double * 5)()
        calls = (C.c_int64 * 5)()
        self._check(self._lib.dg_profile_read(self._h, ms, calls))
        return {k: (ms[i], calls[i]) for i, k in enumerate(self.PROFILE_CATEGORIES)}

    def launch_count(self):
        return int(self._lib.dg_launch_count(self._h))

    def limit(self, z):
        """Vertex-based slope limiter of the liquid species of a DG1 state, in place (asynchronous)."""
        self._check(self._lib.dg_limit(self._h, _ptr(z)))

    def reorth_count(self):
        return int(self._lib.dg_reorth_count(self._h))

    def workspace_bytes(self):
        return int(self._lib.dg_workspace_bytes(self._h))


def _dev_ptr(t, dtypes=("float64",)):
    import torch

    if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous() or str(t.dtype)[6:] not in dtypes:
        raise TypeError("expected contiguous CUDA tensors of " + "/".join(dtypes))
    return t.data_ptr()


class Batch:
    """dg_batch: several contexts (uneven grids, DG0 and DG1, one chemistry) evaluated together --
    one launch per kind of kernel over all instances -- and stepped concurrently."""

    def __init__(self, contexts, stream=None):
        import torch

        self._lib = lib()
        self.contexts = list(contexts)          # keeps the contexts alive as long as the batch
        n = len(self.contexts)
        arr = (_P * n)(*[c._h.value for c in self.contexts])
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = _P()
        st = self._lib.dg_batch_create(arr, n, _P(stream.cuda_stream), C.byref(h))
        if st != OK:
            raise DGError(st, "dg_batch_create (contexts of different chemistries, or out of memory)")
        self._h = h
        self.n = n

    def _check(self, st):
        if st != OK:
            raise DGError(st, self._lib.dg_batch_last_error(self._h).decode())

    def _ptrs(self, tensors, dtypes=("float64",)):
        if len(tensors) != self.n:
            raise ValueError("one tensor per instance")
        return (_P * self.n)(*[_dev_ptr(t, dtypes) for t in tensors])

    def _dbl(self, xs):
        xs = list(xs)
        if len(xs) != self.n:
            raise ValueError("one value per instance")
        return (C.c_double * self.n)(*[float(x) for x in xs])

    @staticmethod
    def _prec(vs):
        import torch

        return MIXED if vs[0].dtype == torch.float32 else FP64

    def jvp(self, zs, ts, dts, vs, outs):
        prec = self._prec(vs)
        dt = ("float32",) if prec == MIXED else ("float64",)
        self._check(self._lib.dg_batch_jvp(self._h, self._ptrs(zs), self._dbl(ts), self._dbl(dts), prec,
                                           self._ptrs(vs, dt), self._ptrs(outs, dt)))
        return outs

    def residual(self, zs, zns, ts, dts, rs):
        self._check(self._lib.dg_batch_residual(self._h, self._ptrs(zs), self._ptrs(zns), self._dbl(ts),
                                                self._dbl(dts), self._ptrs(rs)))
        return rs

    def autotune(self, zs, ts, dts, vs, outs):
        """Choose the schedules by timed trials; returns (DG1 block order, DG0 block size)."""
        prec = self._prec(vs)
        dt = ("float32",) if prec == MIXED else ("float64",)
        ch = (C.c_int32 * 2)()
        self._check(self._lib.dg_batch_autotune(self._h, self._ptrs(zs), self._dbl(ts), self._dbl(dts), prec,
                                                self._ptrs(vs, dt), self._ptrs(outs, dt), ch))
        return int(ch[0]), int(ch[1])

    def step(self, zns, zs, ts, dts):
        """One implicit step of every instance; returns (statuses, step infos)."""
        infos = (StepInfo * self.n)()
        sts = (C.c_int32 * self.n)()
        self._check(self._lib.dg_batch_step(self._h, self._ptrs(zns), self._ptrs(zs), self._dbl(ts), self._dbl(dts),
                                            infos, sts))
        return [int(x) for x in sts], [infos[k] for k in range(self.n)]

    def launch_count(self):
        return int(self._lib.dg_batch_launch_count(self._h))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.dg_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
