"""Torch-facing wrappers over the C ABI (device memory and streams only).

``Band`` and ``Hierarchy`` own the C handles; vectors are CUDA tensors in the
library's band order (float64 or float32).  Nothing here computes: every
step of the method runs in libcpm.so.
"""
from __future__ import annotations

import numpy as np
import torch

from . import capi

_KINDS = {"circle": capi.CPM_CIRCLE, "sphere": capi.CPM_SPHERE, "torus": capi.CPM_TORUS,
          "ellipsoid": capi.CPM_ELLIPSOID, "dziuk": capi.CPM_DZIUK}
_SMOOTHERS = {"jacobi": capi.CPM_SMOOTH_JACOBI, "rm": capi.CPM_SMOOTH_RM, "rbgs": capi.CPM_SMOOTH_RBGS}


def make_surface(kind: str, *params: float) -> capi.cpm_surface:
    s = capi.cpm_surface()
    s.kind = _KINDS[kind]
    for i, p in enumerate(params):
        s.param[i] = float(p)
    if kind in ("circle", "sphere") and not params:
        s.param[0] = 1.0
    return s


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _ptr(t: torch.Tensor, dtype, n: int) -> int:
    if not t.is_cuda or t.dtype != dtype or not t.is_contiguous() or t.numel() != n:
        raise ValueError(f"expected a contiguous CUDA {dtype} tensor of {n} elements")
    return t.data_ptr()


class Band:
    """Band B and ghost ring of one surface at spacing dx (cpm_build_band)."""

    def __init__(self, kind: str, params=(), dx: float = 1 / 64, lo: float = -2.0,
                 lambda2: float = 0.0, stream=None):
        self.kind = kind
        self.params = tuple(params)
        self.dim = 2 if kind == "circle" else 3
        self.dx = dx
        self.lo = lo
        g = capi.cpm_grid()
        g.lo, g.dx, g.n, g.lambda2 = lo, dx, 0, lambda2
        self.handle = capi.cpm_build_band(make_surface(kind, *self.params), g, _stream(stream))
        self.nb, self.ng = capi.cpm_band_info(self.handle)

    def export(self):
        """(ijk, cp, stencil_base) of B+ (B first, then G) as numpy arrays."""
        n = self.nb + self.ng
        ijk = np.empty((n, self.dim), np.int32)
        cp = np.empty((n, self.dim), np.float64)
        base = np.empty((n, self.dim), np.int32)
        capi.cpm_band_export(self.handle, ijk.ctypes.data, cp.ctypes.data, base.ctypes.data)
        return ijk, cp, base

    def counts(self, stream=None):
        """(|B|, nnz(L), nnz(E_3), nnz(M)) as Table 4.1 counts them (cpm_band_counts)."""
        return tuple(capi.cpm_band_counts(self.handle, _stream(stream)))

    def close(self):
        if getattr(self, "handle", None):
            capi.cpm_band_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Hierarchy:
    """Multigrid hierarchy on a band (cpm_build_hierarchy) and its operators."""

    def __init__(self, band: Band, coarsest_dx: float = 0.0, nu1: int = 3, nu2: int = 3,
                 omega: float = 0.8, smoother: str = "jacobi", c: float = 1.0,
                 c_device: torch.Tensor | None = None, residual: str = "extended",
                 coarse_sweeps: int = 0, coarse_f64_max: int = 0, coarse_dense_max: int = 0,
                 op_form: str = "mbr", transfer_deg: int = 1, cycle: int = 1,
                 a_device: torch.Tensor | None = None, relative: bool = False,
                 ext_variant: int | None = None, coarse_gmres: int = 0, outer_f64: bool = False,
                 stream=None):
        o = capi.cpm_mg_opts()
        o.coarsest_dx, o.nu1, o.nu2, o.omega = coarsest_dx, nu1, nu2, omega
        o.smoother, o.transfer_deg, o.c = _SMOOTHERS[smoother], transfer_deg, c
        o.cycle = cycle
        o.residual_mode = {"extended": capi.CPM_RESID_EXTENDED, "plain": capi.CPM_RESID_PLAIN}[residual]
        o.coarse_sweeps = coarse_sweeps
        o.coarse_f64_max, o.coarse_dense_max = coarse_f64_max, coarse_dense_max
        o.op_form = {"mbr": capi.CPM_OP_MBR, "paper": capi.CPM_OP_PAPER,
                     "vardiff": capi.CPM_OP_VARDIFF}[op_form]
        o.a_device = _ptr(a_device, torch.float64, band.nb) if a_device is not None else None
        o.relative = int(relative)
        o.ext_variant = 0 if ext_variant is None else int(ext_variant) + 1
        o.coarse_gmres = coarse_gmres
        o.outer_f64 = int(outer_f64)
        o.c_device = _ptr(c_device, torch.float64, band.nb) if c_device is not None else None
        self.band = band
        self.handle = capi.cpm_build_hierarchy(band.handle, o, _stream(stream))
        self.n_levels, self.nb = capi.cpm_hier_info(self.handle, 0)

    def ext_tuning(self, level: int = 0):
        """(FP32 extension variant chosen for the level, ms of each candidate)."""
        return capi.cpm_hier_ext_tuning(self.handle, level)

    def level_size(self, level: int) -> int:
        return capi.cpm_hier_info(self.handle, level)[1]

    def apply(self, u: torch.Tensor, level: int = 0, out: torch.Tensor | None = None, stream=None):
        n = self.level_size(level)
        prec = capi.CPM_F64 if u.dtype == torch.float64 else capi.CPM_F32
        out = torch.empty_like(u) if out is None else out
        capi.cpm_apply(self.handle, level, prec, _ptr(u, u.dtype, n), _ptr(out, u.dtype, n), _stream(stream))
        return out

    def extend(self, u: torch.Tensor, level: int = 0, with_ghost: bool = False,
               out: torch.Tensor | None = None, stream=None):
        """w = E u on B (and the ghost ring when with_ghost)."""
        n = self.level_size(level)
        nw = n + (self.ghost_size(level) if with_ghost else 0)
        prec = capi.CPM_F64 if u.dtype == torch.float64 else capi.CPM_F32
        out = torch.empty(nw, dtype=u.dtype, device=u.device) if out is None else out
        capi.cpm_extend(self.handle, level, prec, _ptr(u, u.dtype, n), _ptr(out, u.dtype, nw),
                        with_ghost, _stream(stream))
        return out

    def ghost_size(self, level: int) -> int:
        if level == 0:
            return self.band.ng
        raise ValueError("ghost sizes of coarse levels are not exported")

    def smooth(self, f: torch.Tensor, u: torch.Tensor, sweeps: int = 1, level: int = 0, stream=None):
        n = self.level_size(level)
        prec = capi.CPM_F64 if u.dtype == torch.float64 else capi.CPM_F32
        capi.cpm_smooth(self.handle, level, prec, _ptr(f, u.dtype, n), _ptr(u, u.dtype, n), sweeps,
                        _stream(stream))
        return u

    def vcycle(self, f: torch.Tensor, u: torch.Tensor, stream=None):
        prec = capi.CPM_F64 if u.dtype == torch.float64 else capi.CPM_F32
        capi.cpm_vcycle(self.handle, prec, _ptr(f, u.dtype, self.nb), _ptr(u, u.dtype, self.nb),
                        _stream(stream))
        return u

    def residual(self, f: torch.Tensor, u: torch.Tensor, out: torch.Tensor | None = None, stream=None):
        """r = f - A u on the finest level (FP64)."""
        out = torch.empty_like(f) if out is None else out
        capi.cpm_residual(self.handle, _ptr(f, torch.float64, self.nb), _ptr(u, torch.float64, self.nb),
                          _ptr(out, torch.float64, self.nb), _stream(stream))
        return out

    def set_smoother(self, smoother: "Smoother | None"):
        """Use a learned smoother for the first finest-level pre-sweep of FP32 V-cycles."""
        self._smoother = smoother
        capi.cpm_hier_set_smoother(self.handle, smoother.handle if smoother else None)

    def smoother_correction(self, r: torch.Tensor, out: torch.Tensor | None = None, stream=None):
        out = torch.empty_like(r) if out is None else out
        capi.cpm_mlp_correction(self.handle, _ptr(r, torch.float32, self.nb),
                                _ptr(out, torch.float32, self.nb), _stream(stream))
        return out

    def smoother_loss_grad(self, r: torch.Tensor, stream=None):
        grad = np.empty(capi.CPM_MLP_NPARAMS, np.float32)
        loss = capi.cpm_mlp_loss_grad(self.handle, _ptr(r, torch.float32, self.nb), grad.ctypes.data,
                                      _stream(stream))
        return loss, grad

    def smoother_train_step(self, r: torch.Tensor, lr: float = 1e-3, want_loss: bool = True,
                            stream=None):
        return capi.cpm_mlp_train_step(self.handle, _ptr(r, torch.float32, self.nb), lr,
                                       _stream(stream), want_loss)

    def solve(self, f: torch.Tensor, u: torch.Tensor | None = None, tol: float = 1e-10,
              max_iter: int = 100, mode: str = "f64", use_graph: bool = True, stream=None,
              raise_on_fail: bool = True, inner_cycles: int = 1, zero_init: bool | None = None,
              learned: bool = False, fmg: bool = False):
        zero = u is None if zero_init is None else bool(zero_init)
        if u is None:
            u = torch.empty_like(f)
        o = capi.cpm_solve_opts()
        o.tol, o.max_iter = tol, max_iter
        o.mode = capi.CPM_SOLVE_MIXED if mode == "mixed" else capi.CPM_SOLVE_F64
        o.use_graph, o.zero_init = int(use_graph), int(zero)
        o.inner_cycles = inner_cycles
        o.learned = int(learned)
        o.fmg = int(fmg)
        st, rep = capi.cpm_solve(self.handle, _ptr(f, torch.float64, self.nb),
                                 _ptr(u, torch.float64, self.nb), o, _stream(stream), raise_on_fail)
        n = min(rep.iters + 1, capi.CPM_MAX_HISTORY)
        return u, {"status": st, "iters": rep.iters, "converged": bool(rep.converged),
                   "rel_residual": rep.rel_residual, "history": list(rep.history[:n]),
                   "seconds": rep.seconds, "learned_iters": rep.learned_iters,
                   "fallback": bool(rep.fallback), "jacobi_factor": rep.jacobi_factor,
                   "learned_factor": rep.learned_factor, "learned_worst": rep.learned_worst,
                   "f64_checks": rep.f64_checks, "pair_floor": rep.pair_floor}

    def residual_norms(self, f: torch.Tensor, u: torch.Tensor, stream=None):
        return capi.cpm_residual_norms(self.handle, _ptr(f, torch.float64, self.nb),
                                       _ptr(u, torch.float64, self.nb), _stream(stream))

    def close(self):
        if getattr(self, "handle", None):
            capi.cpm_hier_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _report(st, rep) -> dict:
    n = min(rep.iters + 1, capi.CPM_MAX_HISTORY)
    return {"status": st, "iters": rep.iters, "converged": bool(rep.converged),
            "rel_residual": rep.rel_residual, "history": list(rep.history[:n]),
            "seconds": rep.seconds, "f64_checks": rep.f64_checks, "pair_floor": rep.pair_floor}


class Batch:
    """Independent systems A_i u = f over several hierarchies (cpm_build_batch).

    System ``s = i * n_rhs + k`` uses ``hiers[i]``; every system has its own
    workspace.  The hierarchies must outlive the batch.
    """

    def __init__(self, hiers: list[Hierarchy], n_rhs: int = 1, tune_cache: str | None = None):
        self.hiers = list(hiers)
        self.n_rhs = n_rhs
        self.sizes = [h.nb for h in self.hiers for _ in range(n_rhs)]
        self.handle = capi.cpm_build_batch([h.handle for h in self.hiers], n_rhs, tune_cache)

    def solve(self, fs: list[torch.Tensor], us: list[torch.Tensor] | None = None, tol: float = 1e-10,
              max_iter: int = 100, mode: str = "mixed", inner_cycles: int = 1,
              zero_init: bool | None = None, stream=None, raise_on_fail: bool = True):
        if len(fs) != len(self.sizes):
            raise ValueError(f"expected {len(self.sizes)} right-hand sides")
        zero = us is None if zero_init is None else bool(zero_init)
        if us is None:
            us = [torch.empty_like(f) for f in fs]
        o = capi.cpm_solve_opts()
        o.tol, o.max_iter = tol, max_iter
        o.mode = capi.CPM_SOLVE_MIXED if mode == "mixed" else capi.CPM_SOLVE_F64
        o.use_graph, o.zero_init, o.inner_cycles, o.learned = 1, int(zero), inner_cycles, 0
        fp = [_ptr(f, torch.float64, n) for f, n in zip(fs, self.sizes)]
        up = [_ptr(u, torch.float64, n) for u, n in zip(us, self.sizes)]
        st, reps = capi.cpm_solve_batch(self.handle, fp, up, o, _stream(stream), raise_on_fail)
        return us, [_report(st, r) for r in reps]

    def info(self):
        """(concurrency chosen by the autotuner, ms of one iteration per K = 1, 2, 4, ...)."""
        return capi.cpm_batch_info(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            capi.cpm_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Smoother:
    """Learned smoother network (cpm_mlp): parameters live on the device."""

    def __init__(self, seed: int = 0, params: np.ndarray | None = None, handle: int | None = None):
        self.handle = handle if handle is not None else capi.cpm_mlp_create(seed)
        if params is not None:
            self.set_params(params)

    @classmethod
    def load(cls, path: str) -> "Smoother":
        """A network written by ``save`` (cpm_mlp_load)."""
        return cls(handle=capi.cpm_mlp_load(path))

    def train(self, fields, steps: int = 400, lr: float = 2e-3, lr_final: float = 0.0,
              reset: bool = False, stream=None) -> dict:
        """cpm_mlp_train on [(Hierarchy, FP64 residual field), ...]; the library
        scales each field, sets this network as the hierarchies' smoother and
        runs the Adam schedule."""
        o = capi.cpm_train_opts()
        o.steps, o.lr, o.lr_final, o.reset = steps, lr, lr_final, int(reset)
        hs = [h.handle for h, _ in fields]
        rs = [_ptr(r, torch.float64, h.nb) for h, r in fields]
        for h, _ in fields:
            h._smoother = self
        rep = capi.cpm_mlp_train(self.handle, hs, rs, o, _stream(stream))
        return {"steps": rep.steps, "fields": rep.n_fields, "loss_first": rep.loss_first,
                "loss_last": rep.loss_last, "seconds": rep.seconds}

    def get_params(self) -> np.ndarray:
        out = np.empty(capi.CPM_MLP_NPARAMS, np.float32)
        capi.cpm_mlp_get_params(self.handle, out.ctypes.data)
        return out

    def set_params(self, params: np.ndarray):
        p = np.ascontiguousarray(params, dtype=np.float32)
        assert p.size == capi.CPM_MLP_NPARAMS
        capi.cpm_mlp_set_params(self.handle, p.ctypes.data)

    def save(self, path: str):
        """Parameters and Adam state to a file (cpm_mlp_save)."""
        capi.cpm_mlp_save(self.handle, path)

    def close(self):
        if getattr(self, "handle", None):
            capi.cpm_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
