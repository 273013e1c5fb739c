"""ctypes binding of the C ABI in ``include/cpm.h`` (argument marshalling only).

Every function here has the name of the C entry point it calls and passes
plain pointers and sizes; all computation happens in ``libcpm.so``.  Device
vectors are passed as integer device addresses (``tensor.data_ptr()``) and
streams as ``cudaStream_t`` integers (``torch.cuda.current_stream().cuda_stream``).
A missing or unloadable library raises; there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

from . import _build

CPM_OK, CPM_ERR_ARG, CPM_ERR_OOM, CPM_ERR_CUDA, CPM_ERR_REACH = 0, 1, 2, 3, 4
CPM_ERR_DIVERGED, CPM_ERR_NOT_CONVERGED, CPM_ERR_TIMEOUT, CPM_ERR_CHECKED, CPM_ERR_SINGULAR = 5, 6, 7, 8, 9
CPM_CIRCLE, CPM_SPHERE, CPM_TORUS, CPM_ELLIPSOID, CPM_DZIUK = 0, 1, 2, 3, 4
CPM_SMOOTH_JACOBI, CPM_SMOOTH_RM, CPM_SMOOTH_RBGS = 0, 1, 2
CPM_F64, CPM_F32 = 0, 1
CPM_RESID_EXTENDED, CPM_RESID_PLAIN = 0, 1
CPM_SOLVE_F64, CPM_SOLVE_MIXED = 0, 1
CPM_OP_MBR, CPM_OP_PAPER, CPM_OP_VARDIFF = 0, 1, 2
CPM_MAX_HISTORY = 256
CPM_NOALLOC_MAX_POINTS = 1048576


class cpm_surface(C.Structure):
    _fields_ = [("kind", C.c_int32), ("pad_", C.c_int32), ("param", C.c_double * 8)]


class cpm_grid(C.Structure):
    _fields_ = [("lo", C.c_double), ("dx", C.c_double), ("n", C.c_int64), ("lambda2", C.c_double)]


class cpm_mg_opts(C.Structure):
    _fields_ = [("coarsest_dx", C.c_double), ("nu1", C.c_int32), ("nu2", C.c_int32),
                ("omega", C.c_double), ("smoother", C.c_int32), ("transfer_deg", C.c_int32),
                ("c", C.c_double), ("c_device", C.c_void_p), ("residual_mode", C.c_int32),
                ("coarse_sweeps", C.c_int32), ("coarse_f64_max", C.c_int32),
                ("coarse_dense_max", C.c_int32), ("op_form", C.c_int32), ("cycle", C.c_int32),
                ("a_device", C.c_void_p), ("relative", C.c_int32), ("coarse_gmres", C.c_int32),
                ("ext_variant", C.c_int32),
                ("outer_f64", C.c_int32)]


class cpm_solve_opts(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iter", C.c_int32), ("mode", C.c_int32),
                ("use_graph", C.c_int32), ("zero_init", C.c_int32), ("inner_cycles", C.c_int32),
                ("learned", C.c_int32), ("fmg", C.c_int32)]


class cpm_solve_report(C.Structure):
    _fields_ = [("iters", C.c_int32), ("converged", C.c_int32), ("rel_residual", C.c_double),
                ("history", C.c_double * CPM_MAX_HISTORY), ("seconds", C.c_double),
                ("learned_iters", C.c_int32), ("fallback", C.c_int32),
                ("jacobi_factor", C.c_double), ("learned_factor", C.c_double),
                ("learned_worst", C.c_double), ("f64_checks", C.c_int32), ("pair_floor", C.c_double)]


CPM_MLP_NPARAMS = 6337


class cpm_train_set(C.Structure):
    _fields_ = [("n_fields", C.c_int32), ("hier", C.POINTER(C.c_void_p)),
                ("r", C.POINTER(C.c_void_p))]


class cpm_train_opts(C.Structure):
    _fields_ = [("steps", C.c_int32), ("lr", C.c_float), ("lr_final", C.c_float),
                ("reset", C.c_int32)]


class cpm_train_report(C.Structure):
    _fields_ = [("steps", C.c_int32), ("n_fields", C.c_int32), ("loss_first", C.c_double),
                ("loss_last", C.c_double), ("seconds", C.c_double)]


class CpmError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {msg} (status {status})")
        self.status = status


_lib = None

# name -> (restype, argtypes)
_PROTOS = {
    "cpm_status_str": (C.c_char_p, [C.c_int]),
    "cpm_last_error": (C.c_char_p, []),
    "cpm_build_band": (C.c_int, [C.POINTER(cpm_surface), C.POINTER(cpm_grid), C.c_void_p,
                                 C.POINTER(C.c_void_p)]),
    "cpm_band_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "cpm_band_export": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "cpm_band_counts": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.c_void_p]),
    "cpm_band_destroy": (C.c_int, [C.c_void_p]),
    "cpm_build_hierarchy": (C.c_int, [C.c_void_p, C.POINTER(cpm_mg_opts), C.c_void_p,
                                      C.POINTER(C.c_void_p)]),
    "cpm_hier_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.c_int32, C.POINTER(C.c_int64)]),
    "cpm_hier_ext_tuning": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_double)]),
    "cpm_apply": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    "cpm_extend": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_int32,
                             C.c_void_p]),
    "cpm_kernel_launches": (C.c_int64, []),
    "cpm_smooth": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_int32,
                             C.c_void_p]),
    "cpm_vcycle": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    "cpm_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(cpm_solve_opts),
                            C.POINTER(cpm_solve_report), C.c_void_p]),
    "cpm_residual": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "cpm_residual_norms": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_double),
                                     C.POINTER(C.c_double), C.c_void_p]),
    "cpm_residual_norms_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                             C.c_void_p]),
    "cpm_hier_destroy": (C.c_int, [C.c_void_p]),
    "cpm_mlp_create": (C.c_int, [C.c_uint64, C.POINTER(C.c_void_p)]),
    "cpm_mlp_set_params": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32]),
    "cpm_mlp_get_params": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32]),
    "cpm_mlp_destroy": (C.c_int, [C.c_void_p]),
    "cpm_hier_set_smoother": (C.c_int, [C.c_void_p, C.c_void_p]),
    "cpm_mlp_correction": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "cpm_mlp_loss_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_double), C.c_void_p,
                                    C.c_void_p]),
    "cpm_mlp_train_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_float, C.POINTER(C.c_double),
                                     C.c_void_p]),
    "cpm_mlp_train": (C.c_int, [C.c_void_p, C.POINTER(cpm_train_set), C.POINTER(cpm_train_opts),
                                C.POINTER(cpm_train_report), C.c_void_p]),
    "cpm_mlp_save": (C.c_int, [C.c_void_p, C.c_char_p]),
    "cpm_mlp_load": (C.c_int, [C.c_char_p, C.POINTER(C.c_void_p)]),
    "cpm_build_batch": (C.c_int, [C.POINTER(C.c_void_p), C.c_int32, C.c_int32, C.c_char_p,
                                  C.POINTER(C.c_void_p)]),
    "cpm_solve_batch": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                  C.POINTER(cpm_solve_opts), C.c_void_p, C.c_void_p]),
    "cpm_batch_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_double)]),
    "cpm_batch_destroy": (C.c_int, [C.c_void_p]),
}


def exported_names():
    """Entry points declared in include/cpm.h and bound here."""
    return sorted(_PROTOS)


def lib(path: str | None = None):
    """Load libcpm.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1307_4354_gb300._build.build()")
    L = C.CDLL(path)
    for name, (res, args) in _PROTOS.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(status: int, where: str):
    if status != CPM_OK:
        L = lib()
        raise CpmError(status, where, (L.cpm_last_error() or b"").decode() or
                       L.cpm_status_str(status).decode())


def cpm_status_str(status: int) -> str:
    return lib().cpm_status_str(status).decode()


def cpm_last_error() -> str:
    return lib().cpm_last_error().decode()


def cpm_build_band(surface: cpm_surface, grid: cpm_grid, stream: int = 0) -> int:
    out = C.c_void_p()
    _check(lib().cpm_build_band(C.byref(surface), C.byref(grid), C.c_void_p(stream), C.byref(out)),
           "cpm_build_band")
    return out.value


def cpm_band_info(band: int):
    nb, ng = C.c_int64(), C.c_int64()
    _check(lib().cpm_band_info(C.c_void_p(band), C.byref(nb), C.byref(ng)), "cpm_band_info")
    return nb.value, ng.value


def cpm_band_export(band: int, ijk_ptr: int | None, cp_ptr: int | None, base_ptr: int | None):
    _check(lib().cpm_band_export(C.c_void_p(band), C.c_void_p(ijk_ptr), C.c_void_p(cp_ptr),
                                 C.c_void_p(base_ptr)), "cpm_band_export")


def cpm_band_counts(band: int, stream: int = 0):
    out = (C.c_int64 * 4)()
    _check(lib().cpm_band_counts(C.c_void_p(band), out, C.c_void_p(stream)), "cpm_band_counts")
    return list(out)


def cpm_band_destroy(band: int):
    _check(lib().cpm_band_destroy(C.c_void_p(band)), "cpm_band_destroy")


def cpm_build_hierarchy(band: int, opts: cpm_mg_opts, stream: int = 0) -> int:
    out = C.c_void_p()
    _check(lib().cpm_build_hierarchy(C.c_void_p(band), C.byref(opts), C.c_void_p(stream),
                                     C.byref(out)), "cpm_build_hierarchy")
    return out.value


def cpm_hier_info(h: int, level: int = 0):
    nl, nb = C.c_int32(), C.c_int64()
    _check(lib().cpm_hier_info(C.c_void_p(h), C.byref(nl), level, C.byref(nb)), "cpm_hier_info")
    return nl.value, nb.value


def cpm_hier_ext_tuning(h: int, level: int):
    v = C.c_int32()
    ms = (C.c_double * 3)()
    _check(lib().cpm_hier_ext_tuning(C.c_void_p(h), level, C.byref(v), ms), "cpm_hier_ext_tuning")
    return v.value, list(ms)


def cpm_apply(h: int, level: int, prec: int, u_ptr: int, Mu_ptr: int, stream: int = 0):
    _check(lib().cpm_apply(C.c_void_p(h), level, prec, C.c_void_p(u_ptr), C.c_void_p(Mu_ptr),
                           C.c_void_p(stream)), "cpm_apply")


def cpm_extend(h: int, level: int, prec: int, u_ptr: int, w_ptr: int, with_ghost: bool,
               stream: int = 0):
    _check(lib().cpm_extend(C.c_void_p(h), level, prec, C.c_void_p(u_ptr), C.c_void_p(w_ptr),
                            int(with_ghost), C.c_void_p(stream)), "cpm_extend")


def cpm_kernel_launches() -> int:
    return int(lib().cpm_kernel_launches())


def cpm_smooth(h: int, level: int, prec: int, f_ptr: int, u_ptr: int, sweeps: int, stream: int = 0):
    _check(lib().cpm_smooth(C.c_void_p(h), level, prec, C.c_void_p(f_ptr), C.c_void_p(u_ptr), sweeps,
                            C.c_void_p(stream)), "cpm_smooth")


def cpm_vcycle(h: int, prec: int, f_ptr: int, u_ptr: int, stream: int = 0):
    _check(lib().cpm_vcycle(C.c_void_p(h), prec, C.c_void_p(f_ptr), C.c_void_p(u_ptr),
                            C.c_void_p(stream)), "cpm_vcycle")


def cpm_solve(h: int, f_ptr: int, u_ptr: int, opts: cpm_solve_opts, stream: int = 0,
              raise_on_fail: bool = True) -> tuple[int, cpm_solve_report]:
    rep = cpm_solve_report()
    st = lib().cpm_solve(C.c_void_p(h), C.c_void_p(f_ptr), C.c_void_p(u_ptr), C.byref(opts),
                         C.byref(rep), C.c_void_p(stream))
    if raise_on_fail or st not in (CPM_OK, CPM_ERR_NOT_CONVERGED, CPM_ERR_DIVERGED):
        _check(st, "cpm_solve")
    return st, rep


def cpm_residual(h: int, f_ptr: int, u_ptr: int, r_ptr: int, stream: int = 0):
    _check(lib().cpm_residual(C.c_void_p(h), C.c_void_p(f_ptr), C.c_void_p(u_ptr), C.c_void_p(r_ptr),
                              C.c_void_p(stream)), "cpm_residual")


def cpm_residual_norms(h: int, f_ptr: int, u_ptr: int, stream: int = 0):
    rel, l2 = C.c_double(), C.c_double()
    _check(lib().cpm_residual_norms(C.c_void_p(h), C.c_void_p(f_ptr), C.c_void_p(u_ptr),
                                    C.byref(rel), C.byref(l2), C.c_void_p(stream)),
           "cpm_residual_norms")
    return rel.value, l2.value


def cpm_residual_norms_noalloc(h: int, f_ptr: int, u_ptr: int, norms_ptr: int, stream: int = 0):
    """Residual norms into a device buffer of 2 doubles; allocates nothing."""
    _check(lib().cpm_residual_norms_noalloc(C.c_void_p(h), C.c_void_p(f_ptr), C.c_void_p(u_ptr),
                                            C.c_void_p(norms_ptr), C.c_void_p(stream)),
           "cpm_residual_norms_noalloc")


def cpm_hier_destroy(h: int):
    _check(lib().cpm_hier_destroy(C.c_void_p(h)), "cpm_hier_destroy")


def cpm_mlp_create(seed: int = 0) -> int:
    out = C.c_void_p()
    _check(lib().cpm_mlp_create(seed, C.byref(out)), "cpm_mlp_create")
    return out.value


def cpm_mlp_set_params(m: int, params_ptr: int, n: int = CPM_MLP_NPARAMS):
    _check(lib().cpm_mlp_set_params(C.c_void_p(m), C.c_void_p(params_ptr), n), "cpm_mlp_set_params")


def cpm_mlp_get_params(m: int, params_ptr: int, n: int = CPM_MLP_NPARAMS):
    _check(lib().cpm_mlp_get_params(C.c_void_p(m), C.c_void_p(params_ptr), n), "cpm_mlp_get_params")


def cpm_mlp_destroy(m: int):
    _check(lib().cpm_mlp_destroy(C.c_void_p(m)), "cpm_mlp_destroy")


def cpm_hier_set_smoother(h: int, m: int | None):
    _check(lib().cpm_hier_set_smoother(C.c_void_p(h), C.c_void_p(m)), "cpm_hier_set_smoother")


def cpm_mlp_correction(h: int, r_ptr: int, du_ptr: int, stream: int = 0):
    _check(lib().cpm_mlp_correction(C.c_void_p(h), C.c_void_p(r_ptr), C.c_void_p(du_ptr),
                                    C.c_void_p(stream)), "cpm_mlp_correction")


def cpm_mlp_loss_grad(h: int, r_ptr: int, grad_ptr: int | None, stream: int = 0) -> float:
    loss = C.c_double()
    _check(lib().cpm_mlp_loss_grad(C.c_void_p(h), C.c_void_p(r_ptr), C.byref(loss),
                                   C.c_void_p(grad_ptr), C.c_void_p(stream)), "cpm_mlp_loss_grad")
    return loss.value


def cpm_mlp_train_step(h: int, r_ptr: int, lr: float, stream: int = 0, want_loss: bool = True):
    loss = C.c_double()
    _check(lib().cpm_mlp_train_step(C.c_void_p(h), C.c_void_p(r_ptr), C.c_float(lr),
                                    C.byref(loss) if want_loss else None, C.c_void_p(stream)),
           "cpm_mlp_train_step")
    return loss.value if want_loss else None


def cpm_mlp_train(m: int, hiers: list[int], r_ptrs: list[int], opts: cpm_train_opts,
                  stream: int = 0) -> cpm_train_report:
    n = len(hiers)
    if n != len(r_ptrs):
        raise ValueError("one hierarchy per field")
    ts = cpm_train_set()
    ts.n_fields = n
    ha = (C.c_void_p * n)(*hiers)
    ra = (C.c_void_p * n)(*r_ptrs)
    ts.hier = C.cast(ha, C.POINTER(C.c_void_p))
    ts.r = C.cast(ra, C.POINTER(C.c_void_p))
    rep = cpm_train_report()
    _check(lib().cpm_mlp_train(C.c_void_p(m), C.byref(ts), C.byref(opts), C.byref(rep),
                               C.c_void_p(stream)), "cpm_mlp_train")
    return rep


def cpm_mlp_save(m: int, path: str):
    _check(lib().cpm_mlp_save(C.c_void_p(m), path.encode()), "cpm_mlp_save")


def cpm_mlp_load(path: str) -> int:
    out = C.c_void_p()
    _check(lib().cpm_mlp_load(path.encode(), C.byref(out)), "cpm_mlp_load")
    return out.value


def cpm_build_batch(hiers: list[int], n_rhs: int, tune_cache: str | None = None) -> int:
    arr = (C.c_void_p * len(hiers))(*hiers)
    out = C.c_void_p()
    _check(lib().cpm_build_batch(arr, len(hiers), n_rhs,
                                 tune_cache.encode() if tune_cache else None, C.byref(out)),
           "cpm_build_batch")
    return out.value


def cpm_solve_batch(b: int, f_ptrs: list[int], u_ptrs: list[int], opts: cpm_solve_opts,
                    stream: int = 0, raise_on_fail: bool = True):
    n = len(f_ptrs)
    fa = (C.c_void_p * n)(*f_ptrs)
    ua = (C.c_void_p * n)(*u_ptrs)
    reps = (cpm_solve_report * n)()
    st = lib().cpm_solve_batch(C.c_void_p(b), fa, ua, C.byref(opts), reps, C.c_void_p(stream))
    if raise_on_fail or st not in (CPM_OK, CPM_ERR_NOT_CONVERGED, CPM_ERR_DIVERGED):
        _check(st, "cpm_solve_batch")
    return st, list(reps)


def cpm_batch_info(b: int):
    k = C.c_int32()
    ms = (C.c_double * 8)()
    _check(lib().cpm_batch_info(C.c_void_p(b), C.byref(k), ms), "cpm_batch_info")
    return k.value, list(ms)


def cpm_batch_destroy(b: int):
    _check(lib().cpm_batch_destroy(C.c_void_p(b)), "cpm_batch_destroy")
