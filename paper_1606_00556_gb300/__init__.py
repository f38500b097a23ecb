"""Python binding of libbosolve (the sm_103a CPR-FGMRES black-oil Jacobian
solver).  Argument marshalling only: every step of the solve runs in the
library's CUDA kernels.  Functions keep the C names of include/bosolve.h;
vectors are torch CUDA tensors (float64, length 3 nx ny nz, natural
interleaved order: unknown 3c+k = (p, Sw, Sg)[k] of cell c), matrix inputs
numpy arrays (host) or torch CUDA tensors (device).

There is no fallback: importing works without a GPU, but every call needs
the compiled library and raises if it is missing.
"""
from __future__ import annotations

import ctypes
import os
import sys

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libbosolve.so")

BO_OK = 0
BO_ERR_ARG = -1
BO_ERR_CUDA = -2
BO_ERR_OOM = -3
BO_ERR_PATTERN = -4
BO_ERR_NONFINITE = -5
BO_ERR_BREAKDOWN = -6
BO_ERR_NOT_CONVERGED = -7
BO_ERR_TIMEOUT = -8
BO_MEM_HOST = 0
BO_MEM_DEVICE = 1
BO_PREC_FP64 = 0
BO_PREC_FP32 = 1
BO_PREC_BF16 = 2
BO_STAGE_CPR = 0
BO_STAGE_ILU = 1
BO_STAGE_AMG = 2
BO_STAGE_CPR_DECOUPLED = 3
BO_STAGE_ARNOLDI_SPMV = 4
BO_DECOUPLE_QI = 0
BO_DECOUPLE_ABF = 1
BO_LAUNCH_STREAM = 0
BO_LAUNCH_GRAPH = 1
BO_LAUNCH_BATCH_GRAPH = 2

# every symbol include/bosolve.h declares
EXPORTS = (
    "bo_status_str", "bo_prec_opts_default", "bo_solve_opts_default", "bo_ctx_create", "bo_ctx_destroy",
    "bo_mat_create_bsr", "bo_mat_create_csr", "bo_mat_update_values", "bo_mat_spmv", "bo_mat_destroy",
    "bo_prec_setup", "bo_prec_update", "bo_prec_apply", "bo_prec_spmv_decoupled", "bo_prec_amg_levels",
    "bo_prec_destroy", "bo_solve", "bo_solve_bicgstab", "bo_solve_batched", "bo_prec_residual_history", "bo_newton_update",
    "bo_kernel_launches",
    "bo_mat_residual_noalloc",
    "bo_cnn_create", "bo_cnn_destroy", "bo_cnn_param_count", "bo_cnn_get_params", "bo_cnn_set_params",
    "bo_cnn_get_grads", "bo_cnn_forward", "bo_cnn_backward", "bo_cnn_adam_step",
    "bo_conv3d_forward", "bo_conv3d_backward_data", "bo_conv3d_backward_weights",
    "bo_prec_set_coarse_space", "bo_learned_coarse_space", "bo_learned_guess",
    "bo_dp_create", "bo_dp_update_values", "bo_dp_fracture_matrix", "bo_dp_solve", "bo_dp_solve_batched",
    "bo_dp_destroy",
    "bo_prec_set_launch_mode", "bo_prec_set_amg_tile", "bo_set_batch_streams", "bo_autotune_batched", "bo_update_batched",
    "bo_set_conv_engine", "bo_tc_status", "bo_set_amg_cooperative", "bo_set_amg_barrier_spins", "bo_set_gs_fused",
    "bo_newton_opts_default", "bo_model_create", "bo_model_destroy", "bo_model_assemble", "bo_newton_solve",
    "bo_wells_create", "bo_wells_update_values", "bo_wells_set_coupling", "bo_wells_spmv", "bo_solve_bordered",
    "bo_wells_destroy",
    "bo_ow_create", "bo_ow_update_values", "bo_ow_matrix", "bo_ow_spmv", "bo_ow_solve", "bo_ow_solve_bicgstab",
    "bo_ow_destroy",
)


class BoError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {_status_str(status)} ({status})")


class BoArgError(BoError, ValueError, TypeError):
    """An argument the binding rejects before the call (status BO_ERR_ARG):
    a wrong dtype, length, layout or device.  The C ABI takes plain pointers
    and cannot check what they point to, so the binding does."""

    def __init__(self, where):
        super().__init__(BO_ERR_ARG, where)


class bo_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
                ("ncontinua", ctypes.c_int32)]


class bo_prec_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("amg_nu1", ctypes.c_int32), ("amg_nu2", ctypes.c_int32),
                ("amg_overcorr", ctypes.c_double), ("amg_coarse_max", ctypes.c_int32),
                ("decoupling", ctypes.c_int32)]


class bo_solve_opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("restart", ctypes.c_int32), ("maxit", ctypes.c_int32),
                ("x0_is_zero", ctypes.c_int32), ("mem", ctypes.c_int32), ("profile", ctypes.c_int32)]


class bo_tune_result(ctypes.Structure):
    _fields_ = [("launch_mode", ctypes.c_int32), ("streams", ctypes.c_int32), ("best_ms", ctypes.c_double),
                ("from_cache", ctypes.c_int32), ("trial_ms", ctypes.c_double * 9),
                ("amg_cells", ctypes.c_int32), ("amg_threads", ctypes.c_int32), ("tile_ms", ctypes.c_double * 5)]


class bo_solve_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iters", ctypes.c_int32), ("restarts", ctypes.c_int32),
                ("true_rel_res", ctypes.c_double), ("est_rel_res", ctypes.c_double),
                ("solve_ms", ctypes.c_double), ("spmv_launches", ctypes.c_int32), ("spmv_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_FLUID_FIELDS = ("pref", "bw0", "cw", "muw", "bo0", "dbo", "rs0", "drs", "muo", "bg0", "dbg", "mug",
                 "rhow_sc", "rhoo_sc", "rhog_sc", "cr", "swc", "sorw", "sorg", "sgc", "nw", "now", "ng", "nog",
                 "gravity")


class bo_fluid(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in _FLUID_FIELDS]


BO_FORCING_FIXED, BO_FORCING_EW1, BO_FORCING_EW2, BO_FORCING_EW3 = 0, 1, 2, 3
BO_NEWTON_MAX_STEPS = 64


class bo_newton_opts(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("eps_rel", ctypes.c_double), ("forcing", ctypes.c_int32),
                ("theta_fixed", ctypes.c_double), ("theta_max", ctypes.c_double), ("theta_min", ctypes.c_double),
                ("gamma", ctypes.c_double), ("beta", ctypes.c_double), ("maxit", ctypes.c_int32),
                ("restart", ctypes.c_int32), ("lin_maxit", ctypes.c_int32)]


class bo_newton_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iters", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("lin_total", ctypes.c_int32), ("bnorm", ctypes.c_double * (BO_NEWTON_MAX_STEPS + 1)),
                ("theta", ctypes.c_double * BO_NEWTON_MAX_STEPS),
                ("lin_iters", ctypes.c_int32 * BO_NEWTON_MAX_STEPS),
                ("lin_rel_res", ctypes.c_double * BO_NEWTON_MAX_STEPS)]

    def as_dict(self):
        k = self.iters
        return {"status": self.status, "iters": k, "converged": bool(self.converged), "lin_total": self.lin_total,
                "norms": list(self.bnorm[:k + 1]), "thetas": list(self.theta[:k]),
                "linear_iters": list(self.lin_iters[:k]), "linear_rel_res": list(self.lin_rel_res[:k])}


_lib = None
_VP = ctypes.c_void_p


def build(force: bool = False) -> str:
    from .buildlib import build as _b
    return _b(force=force)


def lib():
    """The loaded libbosolve.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libbosolve.so not built ({LIB_PATH}); run paper_1606_00556_gb300.build()")
        L = ctypes.CDLL(LIB_PATH)
        L.bo_status_str.restype = ctypes.c_char_p
        L.bo_status_str.argtypes = [ctypes.c_int]
        L.bo_ctx_create.argtypes = [ctypes.c_int, _VP, ctypes.POINTER(_VP)]
        L.bo_ctx_destroy.argtypes = [_VP]
        for f in (L.bo_mat_create_bsr, L.bo_mat_create_csr):
            f.argtypes = [_VP, ctypes.POINTER(bo_grid), ctypes.c_int32, ctypes.c_int64, _VP, _VP, _VP, ctypes.c_int,
                          ctypes.POINTER(_VP)]
        L.bo_mat_update_values.argtypes = [_VP, _VP, ctypes.c_int]
        L.bo_mat_spmv.argtypes = [_VP, ctypes.c_double, _VP, ctypes.c_double, _VP, ctypes.c_int]
        L.bo_mat_destroy.argtypes = [_VP]
        L.bo_prec_setup.argtypes = [_VP, ctypes.POINTER(bo_prec_opts), ctypes.POINTER(_VP)]
        L.bo_prec_update.argtypes = [_VP]
        L.bo_prec_apply.argtypes = [_VP, ctypes.c_int, _VP, _VP]
        L.bo_prec_spmv_decoupled.argtypes = [_VP, _VP, _VP]
        L.bo_prec_amg_levels.argtypes = [_VP, ctypes.POINTER(ctypes.c_int32), ctypes.c_int]
        L.bo_prec_destroy.argtypes = [_VP]
        L.bo_solve.argtypes = [_VP, _VP, _VP, ctypes.POINTER(bo_solve_opts), ctypes.POINTER(bo_solve_info)]
        L.bo_solve_bicgstab.argtypes = [_VP, _VP, _VP, ctypes.POINTER(bo_solve_opts), ctypes.POINTER(bo_solve_info)]
        L.bo_solve_batched.argtypes = [ctypes.POINTER(_VP), ctypes.c_int, ctypes.POINTER(_VP), ctypes.POINTER(_VP),
                                       ctypes.POINTER(bo_solve_opts), ctypes.POINTER(bo_solve_info)]
        L.bo_prec_residual_history.argtypes = [_VP, ctypes.POINTER(ctypes.c_double), ctypes.c_int]
        L.bo_newton_update.argtypes = [_VP, _VP, _VP, ctypes.c_int64]
        L.bo_mat_residual_noalloc.argtypes = [_VP, _VP, _VP, _VP, _VP]
        L.bo_kernel_launches.restype = ctypes.c_int64
        L.bo_kernel_launches.argtypes = []
        L.bo_prec_opts_default.argtypes = [ctypes.POINTER(bo_prec_opts)]
        L.bo_solve_opts_default.argtypes = [ctypes.POINTER(bo_solve_opts)]
        _i = ctypes.c_int
        L.bo_cnn_create.argtypes = [_VP, _i, _i, _i, _i, ctypes.c_uint64, ctypes.POINTER(_VP)]
        L.bo_cnn_destroy.argtypes = [_VP]
        L.bo_cnn_param_count.restype = ctypes.c_int64
        L.bo_cnn_param_count.argtypes = [_VP]
        for f in (L.bo_cnn_get_params, L.bo_cnn_set_params, L.bo_cnn_get_grads):
            f.argtypes = [_VP, _VP, ctypes.c_int64]
        L.bo_cnn_forward.argtypes = [_VP, _VP, _i, _VP]
        L.bo_cnn_backward.argtypes = [_VP, _VP, _VP, _VP, _i, _i, ctypes.POINTER(ctypes.c_double)]
        L.bo_cnn_adam_step.argtypes = [_VP, ctypes.c_float]
        L.bo_conv3d_forward.argtypes = [_VP, _i, _i, _i, _i, _i, _i, _VP, _VP, _VP, _VP, _i, _VP, _VP]
        L.bo_conv3d_backward_data.argtypes = [_VP, _i, _i, _i, _i, _i, _i, _VP, _VP, _VP]
        L.bo_conv3d_backward_weights.argtypes = [_VP, _i, _i, _i, _i, _i, _i, _VP, _VP, _VP, _VP]
        L.bo_prec_set_coarse_space.argtypes = [_VP, _VP, _i, _i, _i]
        L.bo_learned_coarse_space.argtypes = [_VP, _VP, ctypes.c_double, _i, _i, _i]
        L.bo_dp_create.argtypes = [_VP, ctypes.POINTER(bo_grid), ctypes.c_int32, ctypes.c_int64, _VP, _VP, _VP, _i,
                                   ctypes.POINTER(_VP)]
        L.bo_dp_update_values.argtypes = [_VP, _VP, _i]
        L.bo_dp_fracture_matrix.restype = _VP
        L.bo_dp_fracture_matrix.argtypes = [_VP]
        L.bo_dp_solve.argtypes = [_VP, _VP, _VP, _VP, ctypes.POINTER(bo_solve_opts), ctypes.POINTER(bo_solve_info)]
        L.bo_dp_destroy.argtypes = [_VP]
        L.bo_dp_solve_batched.argtypes = [ctypes.POINTER(_VP), ctypes.POINTER(_VP), ctypes.c_int,
                                          ctypes.POINTER(_VP), ctypes.POINTER(_VP), ctypes.POINTER(bo_solve_opts),
                                          ctypes.POINTER(bo_solve_info)]
        L.bo_prec_set_launch_mode.argtypes = [_VP, _i]
        L.bo_prec_set_amg_tile.argtypes = [_VP, _i, _i]
        L.bo_set_batch_streams.argtypes = [_i]
        L.bo_set_conv_engine.argtypes = [_i]
        L.bo_set_amg_cooperative.argtypes = [_i]
        L.bo_set_amg_barrier_spins.argtypes = [ctypes.c_uint32]
        L.bo_set_gs_fused.argtypes = [_i]
        L.bo_tc_status.argtypes = []
        L.bo_update_batched.argtypes = [ctypes.POINTER(_VP), _i, ctypes.POINTER(_VP), _i]
        L.bo_autotune_batched.argtypes = [ctypes.POINTER(_VP), _i, ctypes.POINTER(_VP), ctypes.POINTER(_VP),
                                          ctypes.POINTER(bo_solve_opts), ctypes.c_char_p, ctypes.POINTER(bo_tune_result)]
        L.bo_learned_guess.argtypes = [_VP, _VP, _VP, ctypes.POINTER(ctypes.c_double), _i, _VP,
                                       ctypes.POINTER(ctypes.c_int)]
        L.bo_newton_opts_default.argtypes = [ctypes.POINTER(bo_newton_opts)]
        L.bo_model_create.argtypes = [_VP, ctypes.POINTER(bo_grid), ctypes.POINTER(bo_fluid), _VP, _VP, _VP, _VP, _VP,
                                      ctypes.c_int32, _VP, _VP, _VP, _VP, _VP, ctypes.POINTER(_VP)]
        L.bo_model_destroy.argtypes = [_VP]
        L.bo_model_assemble.argtypes = [_VP, _VP, _VP, ctypes.c_double, _VP, _VP, ctypes.POINTER(ctypes.c_double)]
        L.bo_newton_solve.argtypes = [_VP, _VP, _VP, _VP, ctypes.c_double, ctypes.POINTER(bo_newton_opts),
                                      ctypes.POINTER(bo_newton_info)]
        L.bo_wells_create.argtypes = [_VP, ctypes.c_int32, ctypes.c_int32, _VP, _VP, ctypes.POINTER(_VP)]
        L.bo_wells_update_values.argtypes = [_VP, _VP, _VP, _VP, _i]
        L.bo_wells_set_coupling.argtypes = [_VP, _i]
        L.bo_wells_spmv.argtypes = [_VP, ctypes.c_double, _VP, ctypes.c_double, _VP]
        L.bo_solve_bordered.argtypes = [_VP, _VP, _VP, _VP, ctypes.POINTER(bo_solve_opts),
                                        ctypes.POINTER(bo_solve_info)]
        L.bo_wells_destroy.argtypes = [_VP]
        L.bo_ow_create.argtypes = [_VP, ctypes.POINTER(bo_grid), ctypes.c_int32, ctypes.c_int64, _VP, _VP, _VP, _i,
                                   ctypes.POINTER(_VP)]
        L.bo_ow_update_values.argtypes = [_VP, _VP, _i]
        L.bo_ow_matrix.restype = _VP
        L.bo_ow_matrix.argtypes = [_VP]
        L.bo_ow_spmv.argtypes = [_VP, ctypes.c_double, _VP, ctypes.c_double, _VP]
        for f in (L.bo_ow_solve, L.bo_ow_solve_bicgstab):
            f.argtypes = [_VP, _VP, _VP, _VP, ctypes.POINTER(bo_solve_opts), ctypes.POINTER(bo_solve_info)]
        L.bo_ow_destroy.argtypes = [_VP]
        _lib = L
    return _lib


def _status_str(s):
    try:
        return lib().bo_status_str(s).decode()
    except Exception:
        return "status"


def _check(rc, where):
    if rc != BO_OK:
        raise BoError(rc, where)


def _ptr(a):
    """(pointer, mem kind) of a torch tensor or numpy array."""
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise BoArgError("tensor must be contiguous")
        return _VP(a.data_ptr()), (BO_MEM_DEVICE if a.is_cuda else BO_MEM_HOST)
    a = np.ascontiguousarray(a)
    return _VP(a.ctypes.data), BO_MEM_HOST


def _f64(a):
    if hasattr(a, "data_ptr"):
        import torch
        if a.dtype != torch.float64:
            raise BoArgError("vectors must be float64")
        return a
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a, what):
    """A host int32 copy of an index array, or the torch tensor itself if it
    is already int32."""
    if hasattr(a, "data_ptr"):
        import torch
        if a.dtype != torch.int32:
            raise BoArgError(f"{what} must be int32, not {a.dtype}")
        return a
    return np.ascontiguousarray(a, dtype=np.int32)


def _count(a):
    return int(a.numel()) if hasattr(a, "numel") else int(np.size(a))


def _need(a, n, what):
    if _count(a) != n:
        raise BoArgError(f"{what} must have {n} entries, not {_count(a)}")


def _on_device(t, ctx, what):
    if ctx is not None and t.is_cuda and t.get_device() != ctx.device:
        raise BoArgError(f"{what} is on cuda:{t.get_device()}, the context on cuda:{ctx.device}")


def _vec(t, n, what, ctx=None, host=False, out=False):
    """(pointer, mem kind, object to keep alive) of a float64 vector of
    exactly n entries: a contiguous torch tensor on the context's device, or
    where `host` is allowed a CPU tensor or a numpy array.  A numpy input is
    converted to a contiguous float64 copy; a numpy output (`out`) is written
    in place, so it must already be one."""
    if hasattr(t, "data_ptr"):
        import torch
        if t.dtype != torch.float64:
            raise BoArgError(f"{what} must be float64, not {t.dtype}")
        if not t.is_contiguous():
            raise BoArgError(f"{what} must be contiguous")
        if not t.is_cuda and not host:
            raise BoArgError(f"{what} must be a CUDA tensor")
        _on_device(t, ctx, what)
        _need(t, n, what)
        return _VP(t.data_ptr()), (BO_MEM_DEVICE if t.is_cuda else BO_MEM_HOST), t
    if not host:
        raise BoArgError(f"{what} must be a CUDA tensor")
    if out:
        if not (isinstance(t, np.ndarray) and t.dtype == np.float64 and t.flags.c_contiguous and t.flags.writeable):
            raise BoArgError(f"{what} must be a writeable C-contiguous float64 array (it is written in place)")
        a = t
    else:
        a = np.ascontiguousarray(t, dtype=np.float64)
    _need(a, n, what)
    return _VP(a.ctypes.data), BO_MEM_HOST, a


def _dvec(t, n, what, ctx=None):
    """Device pointer of a contiguous float64 CUDA vector of n entries."""
    return _vec(t, n, what, ctx)[0]


_CUDA_STREAM_LEGACY = 1  # cudaStreamLegacy: the legacy default stream


def _alive():
    return not sys.is_finalizing()


class Context:
    """bo_ctx: a device and the CUDA stream every call is ordered on.

    By default the context uses torch's current stream on `device`, so the
    library's work is ordered with the torch operations that produce its
    inputs and consume its outputs."""

    def __init__(self, device: int = 0, stream=None):
        h = _VP()
        if stream is None:
            import torch
            stream = torch.cuda.current_stream(device)
        handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        s = _VP(handle if handle else _CUDA_STREAM_LEGACY)
        _check(lib().bo_ctx_create(device, s, ctypes.byref(h)), "bo_ctx_create")
        self.h = h
        self.device = device
        self.stream = stream

    def close(self):
        if self.h and _alive():
            lib().bo_ctx_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def grid(nx, ny, nz, dx=100.0, dy=100.0, dz=20.0) -> bo_grid:
    return bo_grid(nx, ny, nz, dx, dy, dz, 1)


class Matrix:
    """bo_mat: one Jacobian on a structured grid."""

    def __init__(self, ctx: Context, g: bo_grid, h, keep, nval=None):
        self.ctx, self.grid, self.h, self._keep = ctx, g, h, keep
        self.n = 3 * g.nx * g.ny * g.nz
        self.nval = nval  # values bo_mat_update_values reads (None: not updatable here)

    @classmethod
    def from_bsr(cls, ctx, g: bo_grid, rowptr, col, val):
        """bo_mat_create_bsr; arrays on host (numpy) or device (torch)."""
        rowptr, col, val = _i32(rowptr, "rowptr"), _i32(col, "col"), _f64(val)
        rp, m1 = _ptr(rowptr)
        cp, m2 = _ptr(col)
        vp, m3 = _ptr(val)
        if len({m1, m2, m3}) != 1:
            raise BoArgError("rowptr, col and val must all be host or all device")
        h = _VP()
        nb = g.nx * g.ny * g.nz
        nnzb = _count(col)
        _need(rowptr, nb + 1, "rowptr")
        _need(val, 9 * nnzb, "val")
        _check(lib().bo_mat_create_bsr(ctx.h, ctypes.byref(g), nb, nnzb, rp, cp, vp, m1, ctypes.byref(h)),
               "bo_mat_create_bsr")
        return cls(ctx, g, h, (rowptr, col, val), 9 * nnzb)

    @classmethod
    def from_csr(cls, ctx, g: bo_grid, rowptr, col, val):
        """bo_mat_create_csr (scalar CSR, interleaved unknowns)."""
        rowptr, col, val = _i32(rowptr, "rowptr"), _i32(col, "col"), _f64(val)
        rp, m1 = _ptr(rowptr)
        cp, m2 = _ptr(col)
        vp, m3 = _ptr(val)
        if len({m1, m2, m3}) != 1:
            raise BoArgError("rowptr, col and val must all be host or all device")
        h = _VP()
        nrows = 3 * g.nx * g.ny * g.nz
        nnz = _count(col)
        _need(rowptr, nrows + 1, "rowptr")
        _need(val, nnz, "val")
        _check(lib().bo_mat_create_csr(ctx.h, ctypes.byref(g), nrows, nnz, rp, cp, vp, m1, ctypes.byref(h)),
               "bo_mat_create_csr")
        return cls(ctx, g, h, (rowptr, col, val), nnz)

    def update_values(self, val):
        """bo_mat_update_values."""
        val = _f64(val)
        if self.nval is not None:
            _need(val, self.nval, "val")
        vp, mem = _ptr(val)
        if mem == BO_MEM_DEVICE:
            _on_device(val, self.ctx, "val")
        _check(lib().bo_mat_update_values(self.h, vp, mem), "bo_mat_update_values")

    def spmv(self, x, y, alpha=1.0, beta=0.0, precision=BO_PREC_FP64):
        """bo_mat_spmv: y = alpha A x + beta y (device tensors)."""
        _check(lib().bo_mat_spmv(self.h, alpha, _dvec(x, self.n, "x", self.ctx), beta, _dvec(y, self.n, "y", self.ctx),
                                 precision), "bo_mat_spmv")
        return y

    def close(self):
        if self.h and _alive():
            lib().bo_mat_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class DualPorosity:
    """bo_dp: a dual-porosity system (2N block rows; fracture nodes first).
    `fracture_matrix` is the condensed fracture system to build the
    Preconditioner on; `solve` solves the full system."""

    def __init__(self, ctx: Context, nx, ny, nz, rowptr, col, val, dx=100.0, dy=100.0, dz=20.0):
        g = bo_grid(nx, ny, nz, dx, dy, dz, 2)
        rowptr, col, val = _i32(rowptr, "rowptr"), _i32(col, "col"), _f64(val)
        rp, m1 = _ptr(rowptr)
        cp, m2 = _ptr(col)
        vp, m3 = _ptr(val)
        if len({m1, m2, m3}) != 1:
            raise BoArgError("rowptr, col and val must all be host or all device")
        h = _VP()
        N = nx * ny * nz
        nnzb = _count(col)
        _need(rowptr, 2 * N + 1, "rowptr")
        _need(val, 9 * nnzb, "val")
        _check(lib().bo_dp_create(ctx.h, ctypes.byref(g), 2 * N, nnzb, rp, cp, vp, m1, ctypes.byref(h)),
               "bo_dp_create")
        self.h, self.ctx, self.N, self.nval = h, ctx, N, 9 * nnzb
        self._keep = (rowptr, col, val)
        # a borrowed handle: the bo_dp owns the condensed matrix
        self.fracture_matrix = Matrix(ctx, bo_grid(nx, ny, nz, dx, dy, dz, 1), _VP(lib().bo_dp_fracture_matrix(h)), ())
        self.fracture_matrix.close = lambda: None

    def update_values(self, val):
        val = _f64(val)
        _need(val, self.nval, "val")
        vp, mem = _ptr(val)
        if mem == BO_MEM_DEVICE:
            _on_device(val, self.ctx, "val")
        _check(lib().bo_dp_update_values(self.h, vp, mem), "bo_dp_update_values")

    def solve(self, P: "Preconditioner", b, x, tol=1e-8, restart=30, maxit=500, x0_is_zero=True,
              raise_on_error=True):
        o = bo_solve_opts(tol, restart, maxit, int(x0_is_zero), BO_MEM_DEVICE, 0)
        info = bo_solve_info()
        n = 6 * self.N
        rc = lib().bo_dp_solve(self.h, P.h, _dvec(b, n, "b", self.ctx), _dvec(x, n, "x", self.ctx), ctypes.byref(o),
                               ctypes.byref(info))
        if raise_on_error and rc != BO_OK:
            raise BoError(rc, "bo_dp_solve")
        return info.as_dict()

    def close(self):
        if self.h and _alive():
            lib().bo_dp_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class OilWater:
    """bo_ow: a two-phase oil-water system (2x2 blocks, see
    include/bosolve.h).  `matrix` is the padded three-unknown matrix to set
    the preconditioner up on; vectors hold 2N doubles."""

    def __init__(self, ctx: "Context", nx, ny, nz, rowptr, col, val, dx=100.0, dy=100.0, dz=20.0):
        rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
        col = np.ascontiguousarray(col, dtype=np.int32)
        val = _f64(val)
        N = nx * ny * nz
        nnzb = col.size
        _need(val, 4 * nnzb, "val")
        vp, mem = _ptr(val)
        if mem == BO_MEM_DEVICE:
            raise BoArgError("pass the pattern and first values as host arrays")
        h = _VP()
        g = bo_grid(nx, ny, nz, dx, dy, dz, 1)
        _check(lib().bo_ow_create(ctx.h, ctypes.byref(g), N, nnzb, _VP(rowptr.ctypes.data), _VP(col.ctypes.data), vp,
                                  BO_MEM_HOST, ctypes.byref(h)), "bo_ow_create")
        self.h, self.ctx, self.N, self.nval = h, ctx, N, 4 * nnzb
        self.n = 2 * N
        self.matrix = Matrix(ctx, g, _VP(lib().bo_ow_matrix(h)), ())
        self.matrix.close = lambda: None

    def update_values(self, val):
        val = _f64(val)
        _need(val, self.nval, "val")
        vp, mem = _ptr(val)
        if mem == BO_MEM_DEVICE:
            _on_device(val, self.ctx, "val")
        _check(lib().bo_ow_update_values(self.h, vp, mem), "bo_ow_update_values")

    def spmv(self, x, y, alpha=1.0, beta=0.0):
        _check(lib().bo_ow_spmv(self.h, float(alpha), _dvec(x, self.n, "x", self.ctx), float(beta),
                                _dvec(y, self.n, "y", self.ctx)), "bo_ow_spmv")
        return y

    def solve(self, P: "Preconditioner", b, x, tol=1e-8, restart=30, maxit=500, x0_is_zero=True,
              raise_on_error=True, bicgstab=False):
        o = bo_solve_opts(tol, restart, maxit, int(x0_is_zero), BO_MEM_DEVICE, 0)
        info = bo_solve_info()
        f = lib().bo_ow_solve_bicgstab if bicgstab else lib().bo_ow_solve
        rc = f(self.h, P.h, _dvec(b, self.n, "b", self.ctx), _dvec(x, self.n, "x", self.ctx), ctypes.byref(o),
               ctypes.byref(info))
        if raise_on_error and rc != BO_OK:
            raise BoError(rc, "bo_ow_solve")
        return info.as_dict()

    def close(self):
        if self.h and _alive():
            lib().bo_ow_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Wells:
    """bo_wells: the border of rate-controlled wells on a matrix (see
    include/bosolve.h).  perf_cell, perf_well: one entry per perforation,
    grouped by well; values (apw, awp of 3 per perforation, aww per well)
    through update_values."""

    def __init__(self, mat: "Matrix", nwells, perf_cell, perf_well, apw=None, awp=None, aww=None):
        pc = np.ascontiguousarray(perf_cell, dtype=np.int32)
        pw = np.ascontiguousarray(perf_well, dtype=np.int32)
        if pc.size != pw.size:
            raise BoArgError("perf_cell and perf_well differ in length")
        h = _VP()
        _check(lib().bo_wells_create(mat.h, int(nwells), int(pc.size), _VP(pc.ctypes.data), _VP(pw.ctypes.data),
                                     ctypes.byref(h)), "bo_wells_create")
        self.h, self.mat, self.W, self.P = h, mat, int(nwells), int(pc.size)
        self.n = mat.n + self.W
        if aww is not None:
            self.update_values(apw, awp, aww)

    def update_values(self, apw, awp, aww):
        apw, awp, aww = _f64(apw), _f64(awp), _f64(aww)
        _need(apw, 3 * self.P, "apw")
        _need(awp, 3 * self.P, "awp")
        _need(aww, self.W, "aww")
        (pa, ma), (pb, mb), (pc, mc) = _ptr(apw), _ptr(awp), _ptr(aww)
        if not (ma == mb == mc):
            raise BoArgError("apw, awp and aww must all be host or all device arrays")
        _check(lib().bo_wells_update_values(self.h, pa, pb, pc, ma), "bo_wells_update_values")

    def set_coupling(self, mode: int):
        _check(lib().bo_wells_set_coupling(self.h, int(mode)), "bo_wells_set_coupling")

    def spmv(self, x, y, alpha=1.0, beta=0.0):
        """y = alpha A_b x + beta y (device vectors of 3N + W doubles)."""
        ctx = self.mat.ctx
        _check(lib().bo_wells_spmv(self.h, float(alpha), _dvec(x, self.n, "x", ctx), float(beta),
                                   _dvec(y, self.n, "y", ctx)), "bo_wells_spmv")
        return y

    def solve(self, P: "Preconditioner", b, x, tol=1e-8, restart=30, maxit=500, x0_is_zero=True,
              raise_on_error=True):
        """bo_solve_bordered on device vectors of 3N + W doubles."""
        ctx = self.mat.ctx
        o = bo_solve_opts(tol, restart, maxit, int(x0_is_zero), BO_MEM_DEVICE, 0)
        info = bo_solve_info()
        rc = lib().bo_solve_bordered(P.h, self.h, _dvec(b, self.n, "b", ctx), _dvec(x, self.n, "x", ctx),
                                     ctypes.byref(o), ctypes.byref(info))
        if raise_on_error and rc != BO_OK:
            raise BoError(rc, "bo_solve_bordered")
        d = info.as_dict()
        d["rc"] = rc
        return d

    def close(self):
        if self.h and _alive():
            lib().bo_wells_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Preconditioner:
    """bo_prec: CPR-FPF (decoupling + red-black block ILU(0) + AMG)."""

    def __init__(self, mat: Matrix, precision=BO_PREC_FP64, nu1=2, nu2=2, overcorr=1.3, coarse_max=128,
                 decoupling=0):
        o = bo_prec_opts(precision, nu1, nu2, overcorr, coarse_max, decoupling)
        h = _VP()
        _check(lib().bo_prec_setup(mat.h, ctypes.byref(o), ctypes.byref(h)), "bo_prec_setup")
        self.mat, self.h, self.opts = mat, h, o

    def update(self):
        """bo_prec_update (after Matrix.update_values)."""
        _check(lib().bo_prec_update(self.h), "bo_prec_update")

    def _d(self, t, what):
        return _dvec(t, self.mat.n, what, self.mat.ctx)

    def apply(self, stage, r, z):
        """bo_prec_apply: z = stage(r)."""
        _check(lib().bo_prec_apply(self.h, stage, self._d(r, "r"), self._d(z, "z")), "bo_prec_apply")
        return z

    def spmv_decoupled(self, x, y):
        """bo_prec_spmv_decoupled: y = D_QI^{-1} A x."""
        _check(lib().bo_prec_spmv_decoupled(self.h, self._d(x, "x"), self._d(y, "y")), "bo_prec_spmv_decoupled")
        return y

    def amg_levels(self):
        """bo_prec_amg_levels: [(nx, ny, nz), ...]."""
        buf = (ctypes.c_int32 * (3 * 24))()
        n = lib().bo_prec_amg_levels(self.h, buf, 24)
        if n < 0:
            raise BoError(n, "bo_prec_amg_levels")
        return [tuple(buf[3 * i:3 * i + 3]) for i in range(n)]

    def solve(self, b, x, tol=1e-8, restart=30, maxit=500, x0_is_zero=True, profile=False, raise_on_error=True):
        """bo_solve: FGMRES(restart) + CPR to ||b - A x|| <= tol ||b||.
        b, x: torch CUDA tensors (device) or numpy arrays (host).  Returns
        the bo_solve_info fields as a dict."""
        bp, m1, _kb = _vec(b, self.mat.n, "b", self.mat.ctx, host=True)
        xp, m2, _kx = _vec(x, self.mat.n, "x", self.mat.ctx, host=True, out=True)
        if m1 != m2:
            raise BoArgError("b and x must both be host or both device")
        o = bo_solve_opts(tol, restart, maxit, int(x0_is_zero), m1, int(profile))
        info = bo_solve_info()
        rc = lib().bo_solve(self.h, bp, xp, ctypes.byref(o), ctypes.byref(info))
        if raise_on_error and rc not in (BO_OK, BO_ERR_NOT_CONVERGED):
            raise BoError(rc, "bo_solve")
        d = info.as_dict()
        d["status"] = rc
        return d

    def solve_bicgstab(self, b, x, tol=1e-8, maxit=500, x0_is_zero=True, raise_on_error=True):
        """bo_solve_bicgstab: BiCGSTAB + CPR to ||b - A x|| <= tol ||b||
        (same arguments and result as solve)."""
        bp, m1, _kb = _vec(b, self.mat.n, "b", self.mat.ctx, host=True)
        xp, m2, _kx = _vec(x, self.mat.n, "x", self.mat.ctx, host=True, out=True)
        if m1 != m2:
            raise BoArgError("b and x must both be host or both device")
        o = bo_solve_opts(tol, 30, maxit, int(x0_is_zero), m1, 0)
        info = bo_solve_info()
        rc = lib().bo_solve_bicgstab(self.h, bp, xp, ctypes.byref(o), ctypes.byref(info))
        if raise_on_error and rc not in (BO_OK, BO_ERR_NOT_CONVERGED):
            raise BoError(rc, "bo_solve_bicgstab")
        d = info.as_dict()
        d["status"] = rc
        return d

    def set_launch_mode(self, mode):
        """BO_LAUNCH_STREAM, BO_LAUNCH_GRAPH (per-column CUDA graphs) or BO_LAUNCH_BATCH_GRAPH
        (one graph per column for a whole bo_solve_batched batch, in lockstep)."""
        _check(lib().bo_prec_set_launch_mode(self.h, int(mode)), "bo_prec_set_launch_mode")

    def set_amg_tile(self, cells, threads):
        """bo_prec_set_amg_tile: level-0 cells per thread and threads per block of the
        per-kernel AMG form."""
        _check(lib().bo_prec_set_amg_tile(self.h, int(cells), int(threads)), "bo_prec_set_amg_tile")

    def set_coarse_space(self, dp, tile=(16, 16, 8)):
        """Learned coarse space from a predicted pressure update dp (device
        float64, one value per cell, natural order); None removes it."""
        ptr = _dvec(dp, self.mat.n // 3, "dp", self.mat.ctx) if dp is not None else None
        _check(lib().bo_prec_set_coarse_space(self.h, ptr, *[int(t) for t in tile]), "bo_prec_set_coarse_space")

    def learned_coarse_space(self, pred, scale, tile=(16, 16, 8)):
        """Learned coarse space from the network prediction pred [V, 4]
        (device float32; channel 0 times scale is the pressure update)."""
        V = self.mat.n // 3
        ptr = _dev(pred, "float32", "pred", 4 * V) if pred is not None else None
        _check(lib().bo_learned_coarse_space(self.h, ptr, float(scale), *[int(t) for t in tile]),
               "bo_learned_coarse_space")

    def learned_guess(self, b, pred, scale, ncomp, x0) -> bool:
        """x0 from the network prediction pred [V, 4] (scaled per component);
        falls back to zero unless it lowers the residual.  Returns whether the
        guess was kept."""
        sc = (ctypes.c_double * 3)(*[float(v) for v in scale])
        used = ctypes.c_int(0)
        V = self.mat.n // 3
        _check(lib().bo_learned_guess(self.h, self._d(b, "b"), _dev(pred, "float32", "pred", 4 * V), sc, int(ncomp),
                                      self._d(x0, "x0"), ctypes.byref(used)), "bo_learned_guess")
        return bool(used.value)

    def residual_history(self, cap=4096):
        buf = (ctypes.c_double * cap)()
        n = lib().bo_prec_residual_history(self.h, buf, cap)
        return np.array(buf[:max(n, 0)])

    def close(self):
        if self.h and _alive():
            lib().bo_prec_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def bo_mat_residual_noalloc(mat: Matrix, b, x, r, norms):
    """r = b - A x, norms[0:2] = (||r||, ||b||) on the device, with no device
    allocation during the call (see include/bosolve.h)."""
    d = lambda t, w: _dvec(t, mat.n, w, mat.ctx)
    _check(lib().bo_mat_residual_noalloc(mat.h, d(b, "b"), d(x, "x"), d(r, "r"), _dvec(norms, 2, "norms", mat.ctx)),
           "bo_mat_residual_noalloc")
    return r, norms


def bo_solve_batched(precs, bs, xs, tol=1e-8, restart=30, maxit=500, x0_is_zero=True):
    """bo_solve_batched: solve every (precs[r], bs[r]) into xs[r] at once
    (device tensors).  Returns (status, [info dict per system])."""
    n = len(precs)
    if not (len(bs) == len(xs) == n) or n == 0:
        raise ValueError("one b and one x per preconditioner")
    P = (_VP * n)(*[p.h for p in precs])
    B = (_VP * n)(*[p._d(t, f"b[{i}]") for i, (p, t) in enumerate(zip(precs, bs))])
    X = (_VP * n)(*[p._d(t, f"x[{i}]") for i, (p, t) in enumerate(zip(precs, xs))])
    o = bo_solve_opts(tol, restart, maxit, int(x0_is_zero), BO_MEM_DEVICE, 0)
    infos = (bo_solve_info * n)()
    rc = lib().bo_solve_batched(P, n, B, X, ctypes.byref(o), infos)
    out = []
    for i in infos:
        d = i.as_dict()
        out.append(d)
    return rc, out


def bo_dp_solve_batched(dps, precs, bs, xs, tol=1e-8, restart=30, maxit=500, x0_is_zero=True):
    """bo_dp_solve_batched: the dual-porosity systems dps[r] with
    preconditioners precs[r] (on their fracture matrices), device vectors
    bs[r], xs[r] of 6 N_r doubles.  Returns (status, list of info dicts)."""
    n = len(dps)
    if not (len(precs) == len(bs) == len(xs) == n) or n < 1:
        raise BoArgError("bo_dp_solve_batched: lists of different lengths")
    D = (_VP * n)(*[d.h for d in dps])
    P = (_VP * n)(*[p.h for p in precs])
    B = (_VP * n)(*[_dvec(b, 2 * d.N * 3, "b", d.ctx) for b, d in zip(bs, dps)])
    X = (_VP * n)(*[_dvec(x, 2 * d.N * 3, "x", d.ctx) for x, d in zip(xs, dps)])
    o = bo_solve_opts(tol, restart, maxit, int(x0_is_zero), BO_MEM_DEVICE, 0)
    infos = (bo_solve_info * n)()
    rc = lib().bo_dp_solve_batched(D, P, n, B, X, ctypes.byref(o), infos)
    if rc not in (BO_OK, BO_ERR_NOT_CONVERGED):
        raise BoError(rc, "bo_dp_solve_batched")
    return rc, [i.as_dict() for i in infos]


def bo_update_batched(precs, vals=None):
    """bo_update_batched: new values (device tensors, or None to keep) for
    every preconditioner's matrix, then refresh them all, one sync in all."""
    n = len(precs)
    P = (_VP * n)(*[p.h for p in precs])
    if vals is None:
        V = None
    else:
        if len(vals) != n:
            raise BoArgError("one value array (or None) per preconditioner")
        for i, (p, v) in enumerate(zip(precs, vals)):
            if v is not None and p.mat.nval is not None:
                _need(v, p.mat.nval, f"vals[{i}]")
        V = (_VP * n)(*[_VP(_dev(v, "float64", "val").value) if v is not None else None for v in vals])
    _check(lib().bo_update_batched(P, n, V, BO_MEM_DEVICE), "bo_update_batched")


def bo_set_amg_cooperative(on: int):
    """2 (default): level 0 as two cooperative launches per V-cycle around
    one cluster launch for the coarser levels; 1: the cooperative launches
    cover every multi-block level; 0: one kernel per sweep."""
    _check(lib().bo_set_amg_cooperative(int(on)), "bo_set_amg_cooperative")


def bo_set_gs_fused(on: int):
    """1 (default): CGS2 in three passes (first update fused with the second
    coefficient pass); 0: four separate passes."""
    _check(lib().bo_set_gs_fused(int(on)), "bo_set_gs_fused")


def bo_set_amg_barrier_spins(spins: int):
    """Polls of an AMG grid barrier before it gives up (0: the default)."""
    _check(lib().bo_set_amg_barrier_spins(int(spins)), "bo_set_amg_barrier_spins")


def bo_set_conv_engine(engine: int):
    """0: mma.sync, 1: tcgen05 for the 32 -> 32 convolutions."""
    _check(lib().bo_set_conv_engine(int(engine)), "bo_set_conv_engine")


def bo_tc_status() -> int:
    return int(lib().bo_tc_status())


def bo_set_batch_streams(n: int):
    _check(lib().bo_set_batch_streams(int(n)), "bo_set_batch_streams")


def bo_autotune_batched(precs, bs, xs, cache_path=None, tol=1e-8, restart=30, maxit=500):
    """bo_autotune_batched: pick (launch mode, stream-pool width) for this
    batch by timing, or from the JSON cache; returns a dict of the result."""
    n = len(precs)
    if not (len(bs) == len(xs) == n) or n == 0:
        raise BoArgError("one b and one x per preconditioner")
    P = (_VP * n)(*[p.h for p in precs])
    B = (_VP * n)(*[p._d(t, f"b[{i}]") for i, (p, t) in enumerate(zip(precs, bs))])
    X = (_VP * n)(*[p._d(t, f"x[{i}]") for i, (p, t) in enumerate(zip(precs, xs))])
    o = bo_solve_opts(tol, restart, maxit, 1, BO_MEM_DEVICE, 0)
    res = bo_tune_result()
    path = cache_path.encode() if cache_path else None
    _check(lib().bo_autotune_batched(P, n, B, X, ctypes.byref(o), path, ctypes.byref(res)), "bo_autotune_batched")
    return {"launch_mode": res.launch_mode, "streams": res.streams, "best_ms": res.best_ms,
            "from_cache": bool(res.from_cache), "trial_ms": list(res.trial_ms),
            "amg_cells": res.amg_cells, "amg_threads": res.amg_threads, "tile_ms": list(res.tile_ms)}


def bo_kernel_launches() -> int:
    """Kernels the library has launched in this process so far."""
    return int(lib().bo_kernel_launches())


def bo_newton_update(ctx: Context, state, dx):
    """state += dx on the device (paper Alg. 1 update)."""
    n = _count(state)
    _check(lib().bo_newton_update(ctx.h, _dvec(state, n, "state", ctx), _dvec(dx, n, "dx", ctx), n),
           "bo_newton_update")


# ---------------------------------------------------------------- learned update
def _dev(t, dtype_name, what, n=None):
    """Device pointer of a contiguous CUDA tensor of the given dtype (and,
    if n is given, of exactly n entries)."""
    if t is None:
        return None
    if not hasattr(t, "data_ptr") or not t.is_cuda or not t.is_contiguous():
        raise BoArgError(f"{what} must be a contiguous CUDA tensor")
    if str(t.dtype) != "torch." + dtype_name:
        raise BoArgError(f"{what} must be {dtype_name}")
    if n is not None:
        _need(t, n, what)
    return _VP(t.data_ptr())


def _bits(t):
    """BF16 tensor -> the same storage as int16 bit patterns (no copy)."""
    import torch
    return t.view(torch.int16) if t.dtype == torch.bfloat16 else t


def fluid(**values) -> bo_fluid:
    """A bo_fluid from keyword values (every field of the struct required)."""
    missing = [k for k in _FLUID_FIELDS if k not in values]
    if missing:
        raise BoArgError(f"fluid: missing {missing}")
    return bo_fluid(**{k: float(values[k]) for k in _FLUID_FIELDS})


class Model:
    """bo_model: the black-oil residual and Jacobian on the device, and the
    inexact Newton method around the solver (paper Sec. 2.1, 2.3, 3.1)."""

    def __init__(self, ctx: Context, g: bo_grid, fl: bo_fluid, kx, ky, kz, phi0, depth, perf_cell=(),
                 perf_type=(), perf_bhp=(), perf_dref=(), perf_wi=()):
        N = g.nx * g.ny * g.nz
        arrs = []
        for nm, a in (("kx", kx), ("ky", ky), ("kz", kz), ("phi0", phi0), ("depth", depth)):
            a = np.ascontiguousarray(a, dtype=np.float64)
            if a.size != N:
                raise BoArgError(f"{nm}: {a.size} values for {N} cells")
            arrs.append(a)
        pc = np.ascontiguousarray(perf_cell, dtype=np.int32).ravel()
        pt = np.ascontiguousarray(perf_type, dtype=np.int32).ravel()
        pb, pd, pw = (np.ascontiguousarray(v, dtype=np.float64).ravel() for v in (perf_bhp, perf_dref, perf_wi))
        if not (pc.size == pt.size == pb.size == pd.size == pw.size):
            raise BoArgError("perforation arrays of different lengths")
        self._keep = (arrs, pc, pt, pb, pd, pw)
        h = _VP()
        vp = lambda a: _VP(a.ctypes.data) if a.size else None
        _check(lib().bo_model_create(ctx.h, ctypes.byref(g), ctypes.byref(fl), *[vp(a) for a in arrs],
                                     ctypes.c_int32(pc.size), vp(pc), vp(pt), vp(pb), vp(pd), vp(pw),
                                     ctypes.byref(h)), "bo_model_create")
        self.ctx, self.grid, self.h = ctx, g, h
        self.n = 3 * N
        self.nnzb = N + 2 * ((g.nx - 1) * g.ny * g.nz + g.nx * (g.ny - 1) * g.nz + g.nx * g.ny * (g.nz - 1))

    def assemble(self, x, xn, dt, b=None, val=None):
        """bo_model_assemble: b = -R(x) and the Jacobian values (BSR order of
        the 7-point pattern) into the given device tensors; returns ||b||."""
        nb = ctypes.c_double(0.0)
        bp = _dvec(b, self.n, "b", self.ctx) if b is not None else None
        vp = _dvec(val, 9 * self.nnzb, "val", self.ctx) if val is not None else None
        _check(lib().bo_model_assemble(self.h, _dvec(x, self.n, "x", self.ctx), _dvec(xn, self.n, "xn", self.ctx),
                                       float(dt), bp, vp, ctypes.byref(nb)), "bo_model_assemble")
        return nb.value

    def newton(self, P, x, xn, dt, raise_on_error=True, **opts):
        """bo_newton_solve on x (device, in place); opts: the fields of
        bo_newton_opts (forcing 'ew1' | 'ew2' | 'ew3' or a float theta).
        Returns the info dict."""
        o = bo_newton_opts()
        lib().bo_newton_opts_default(ctypes.byref(o))
        forcing = opts.pop("forcing", "ew3")
        if isinstance(forcing, str):
            o.forcing = {"ew1": BO_FORCING_EW1, "ew2": BO_FORCING_EW2, "ew3": BO_FORCING_EW3}[forcing]
        else:
            o.forcing, o.theta_fixed = BO_FORCING_FIXED, float(forcing)
        for k, v in opts.items():
            if not hasattr(o, k):
                raise BoArgError(f"newton: unknown option {k}")
            setattr(o, k, v)
        info = bo_newton_info()
        rc = lib().bo_newton_solve(self.h, P.h, _dvec(x, self.n, "x", self.ctx), _dvec(xn, self.n, "xn", self.ctx),
                                   float(dt), ctypes.byref(o), ctypes.byref(info))
        if raise_on_error and rc not in (BO_OK, BO_ERR_NOT_CONVERGED):
            raise BoError(rc, "bo_newton_solve")
        d = info.as_dict()
        d["status"] = rc
        return d

    def close(self):
        if self.h and _alive():
            lib().bo_model_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class CNN:
    """bo_cnn: the 3D convolutional network of the learned Newton update
    (16 input channels, 32 hidden, 6 residual blocks; prediction [B, V, 4]
    FP32).  Inputs are torch.bfloat16 [B, nz, ny, nx, 16] (or flat)."""

    def __init__(self, ctx: Context, nx, ny, nz, max_batch=1, seed=0):
        h = _VP()
        _check(lib().bo_cnn_create(ctx.h, nx, ny, nz, max_batch, seed, ctypes.byref(h)), "bo_cnn_create")
        self.h, self.ctx = h, ctx
        self.dims = (nx, ny, nz)
        self.V = nx * ny * nz
        self.max_batch = max_batch

    @property
    def nparam(self) -> int:
        return int(lib().bo_cnn_param_count(self.h))

    def get_params(self) -> np.ndarray:
        out = np.zeros(self.nparam, np.float32)
        _check(lib().bo_cnn_get_params(self.h, _VP(out.ctypes.data), out.size), "bo_cnn_get_params")
        return out

    def set_params(self, p) -> None:
        p = np.ascontiguousarray(p, dtype=np.float32)
        _check(lib().bo_cnn_set_params(self.h, _VP(p.ctypes.data), p.size), "bo_cnn_set_params")

    def get_grads(self) -> np.ndarray:
        out = np.zeros(self.nparam, np.float32)
        _check(lib().bo_cnn_get_grads(self.h, _VP(out.ctypes.data), out.size), "bo_cnn_get_grads")
        return out

    def forward(self, x, pred):
        B = x.shape[0]
        _check(lib().bo_cnn_forward(self.h, _dev(_bits(x), "int16", "x", 16 * B * self.V), B,
                                    _dev(pred, "float32", "pred", 4 * B * self.V)), "bo_cnn_forward")
        return pred

    def backward(self, x, target, mask=None, nout=1, want_loss=True):
        B = x.shape[0]
        loss = ctypes.c_double(0.0)
        _check(lib().bo_cnn_backward(self.h, _dev(_bits(x), "int16", "x", 16 * B * self.V),
                                     _dev(target, "float32", "target", 4 * B * self.V),
                                     _dev(mask, "float32", "mask", B * self.V), nout, B,
                                     ctypes.byref(loss) if want_loss else None), "bo_cnn_backward")
        return loss.value if want_loss else None

    def adam_step(self, lr):
        _check(lib().bo_cnn_adam_step(self.h, ctypes.c_float(lr)), "bo_cnn_adam_step")

    def close(self):
        if self.h and _alive():
            lib().bo_cnn_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def bo_conv3d_forward(ctx: Context, dims, x, w, bias, residual=None, relu=False, y=None, yf=None):
    """One 3x3x3 convolution (see bo_conv3d_forward in include/bosolve.h).
    dims = (nx, ny, nz); x [B, V, cin] bf16, w [27, cout, cin] bf16, bias
    [cout] f32; y [B, V, cout] bf16 and/or yf f32."""
    nx, ny, nz = dims
    B = x.shape[0]
    cin, cout = w.shape[2], w.shape[1]
    BV = B * nx * ny * nz
    # with y given, yf holds output channels 0..3 only (the network's prediction)
    nyf = BV * (4 if y is not None else cout)
    _check(lib().bo_conv3d_forward(ctx.h, nx, ny, nz, B, cin, cout, _dev(_bits(x), "int16", "x", BV * cin),
                                   _dev(_bits(w), "int16", "w", 27 * cout * cin),
                                   _dev(bias, "float32", "bias", cout),
                                   _dev(_bits(residual), "int16", "residual", BV * cout) if residual is not None else None,
                                   int(relu), _dev(_bits(y), "int16", "y", BV * cout) if y is not None else None,
                                   _dev(yf, "float32", "yf", nyf)), "bo_conv3d_forward")


def bo_conv3d_backward_data(ctx: Context, dims, dy, w, dx):
    nx, ny, nz = dims
    B = dy.shape[0]
    cin, cout = w.shape[2], w.shape[1]
    BV = B * nx * ny * nz
    _check(lib().bo_conv3d_backward_data(ctx.h, nx, ny, nz, B, cin, cout, _dev(_bits(dy), "int16", "dy", BV * cout),
                                         _dev(_bits(w), "int16", "w", 27 * cout * cin),
                                         _dev(dx, "float32", "dx", BV * cin)), "bo_conv3d_backward_data")


def bo_conv3d_backward_weights(ctx: Context, dims, x, dy, dw, db):
    nx, ny, nz = dims
    B = x.shape[0]
    cout, cin = dw.shape[1], dw.shape[2]
    BV = B * nx * ny * nz
    _check(lib().bo_conv3d_backward_weights(ctx.h, nx, ny, nz, B, cin, cout, _dev(_bits(x), "int16", "x", BV * cin),
                                            _dev(dy, "float32", "dy", BV * cout),
                                            _dev(dw, "float32", "dw", 27 * cout * cin),
                                            _dev(db, "float32", "db", cout)), "bo_conv3d_backward_weights")
