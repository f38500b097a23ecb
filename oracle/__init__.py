"""FP64 CPU oracle of the CPR-FGMRES black-oil Jacobian solver.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline leg may import this package; the solver library never does, and it
shares no code with the GPU path.  ``oracle.cpp`` holds the arithmetic (plain
single-threaded double-precision loops); this module compiles it with g++ and
marshals numpy arrays.

Pinned by tests/test_oracle_pins.py against dense linear algebra, textbook
characterisations and closed forms; see the docstring of each function for
the paper passage it follows.  ``newton.py`` holds the inexact Newton method
(Alg. 1) on top of these solvers, pinned by tests/test_oracle_newton_pins.py.
tests/test_oracle_mutations.py compiles altered copies of oracle.cpp and
loads them through the BO_ORACLE_LIB variable to show that the pins fail on
each planted mistake.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# BO_ORACLE_LIB names a prebuilt oracle library to load instead (the pin
# tests' planted-mistake checks compile altered copies of oracle.cpp)
_LIB_PATH = os.environ.get("BO_ORACLE_LIB") or os.path.join(_HERE, "liboracle.so")
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I32 = ctypes.POINTER(ctypes.c_int32)
_I64 = ctypes.POINTER(ctypes.c_int64)

SMOOTHER_RBGS = 0
SMOOTHER_JACOBI = 1


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "oracle.cpp")
    if os.environ.get("BO_ORACLE_LIB"):
        return _LIB_PATH
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(src):
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-pthread", "-shared", "-fPIC", src, "-o", _LIB_PATH])
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        L.or_rel_residual.restype = ctypes.c_double
        L.or_amg_create.restype = ctypes.c_void_p
        L.or_amg_create.argtypes = [ctypes.c_int64, _I32, _I32, _D, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
        L.or_amg_nlevels.argtypes = [ctypes.c_void_p]
        L.or_amg_level_dims.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
        L.or_amg_level_matrix.restype = ctypes.c_int64
        L.or_amg_level_matrix.argtypes = [ctypes.c_void_p, ctypes.c_int, _I32, _I32, _D]
        L.or_amg_vcycle.argtypes = [ctypes.c_void_p, _D, _D]
        L.or_amg_destroy.argtypes = [ctypes.c_void_p]
        L.or_prec_ilu0_create.restype = ctypes.c_void_p
        L.or_prec_ilu0_create.argtypes = [ctypes.c_int64, ctypes.c_int, _I32, _I32, _D, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
        L.or_prec_cpr_create.restype = ctypes.c_void_p
        L.or_prec_cpr_create.argtypes = [ctypes.c_int64, _I32, _I32, _D, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_int)]
        L.or_prec_apply.argtypes = [ctypes.c_void_p, _D, _D]
        L.or_prec_cpr_set_coarse.argtypes = [ctypes.c_void_p, _D] + [ctypes.c_int] * 6
        L.or_prec_cpr_coarse_apply.argtypes = [ctypes.c_void_p, _D, _D]
        L.or_prec_destroy.argtypes = [ctypes.c_void_p]
        L.or_gmres.argtypes = [ctypes.c_int64, ctypes.c_int, _I32, _I32, _D, _D, _D, ctypes.c_int, ctypes.c_int,
                               ctypes.c_double, ctypes.c_void_p, _D]
        L.or_bicgstab.argtypes = [ctypes.c_int64, ctypes.c_int, _I32, _I32, _D, _D, _D, ctypes.c_int,
                                  ctypes.c_double, ctypes.c_void_p, _D]
        _lib = L
    return _lib


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _p(a, t):
    return a.ctypes.data_as(t)


class BsrMatrix:
    """A BSR matrix as plain numpy arrays (val shaped (nnzb, bs, bs))."""

    def __init__(self, rowptr, col, val):
        self.rowptr = _i(rowptr)
        self.col = _i(col)
        self.val = _d(val)
        self.nb = self.rowptr.size - 1
        self.bs = self.val.shape[-1]

    @property
    def n(self):
        return self.nb * self.bs

    def args(self):
        return (ctypes.c_int64(self.nb), ctypes.c_int(self.bs), _p(self.rowptr, _I32), _p(self.col, _I32),
                _p(self.val, _D))

    def to_dense(self) -> np.ndarray:
        bs = self.bs
        A = np.zeros((self.n, self.n))
        for i in range(self.nb):
            for e in range(self.rowptr[i], self.rowptr[i + 1]):
                j = self.col[e]
                A[i * bs:(i + 1) * bs, j * bs:(j + 1) * bs] += self.val[e]
        return A


def spmv(A: BsrMatrix, x) -> np.ndarray:
    """y = A x (paper Sec. 3.3, y = alpha A x + beta y with alpha=1, beta=0)."""
    x = _d(x)
    y = np.zeros(A.n)
    lib().or_bsr_spmv(*A.args(), _p(x, _D), _p(y, _D))
    return y


def spmv_threads(A: BsrMatrix, x, nthreads: int, y=None) -> np.ndarray:
    """y = A x over nthreads host threads (the CPU SpMV bandwidth baseline)."""
    x = _d(x)
    y = np.zeros(A.n) if y is None else y
    lib().or_bsr_spmv_threads(*A.args(), _p(x, _D), _p(y, _D), ctypes.c_int(int(nthreads)))
    return y


def qi_decouple(A: BsrMatrix):
    """(D_QI^{-1} A, g): g[i] = the weights of the decoupled pressure row of
    cell i, (1, -a_01/a_11, -a_02/a_22) of A_ii (paper Sec. 3.2, Quasi-IMPES),
    or row 0 of A_ii^{-1} where Quasi-IMPES leaves a non-positive pressure
    pivot.  Raises on a zero pivot."""
    out = np.zeros_like(A.val)
    w = np.zeros((A.nb, 3))
    rc = lib().or_qi_decouple(ctypes.c_int64(A.nb), _p(A.rowptr, _I32), _p(A.col, _I32), _p(A.val, _D),
                              _p(out, _D), _p(w, _D))
    if rc != 0:
        raise ArithmeticError("QI decoupling: zero saturation pivot")
    return BsrMatrix(A.rowptr, A.col, out), w


def abf_decouple(A: BsrMatrix) -> BsrMatrix:
    """ABF decoupling (paper Sec. 3.2, the Alternate Block Factorization it
    cites): D^{-1} A with D the block diagonal of A, every block of block
    row i multiplied on the left by A_ii^{-1} (any block size)."""
    val = np.empty_like(A.val)
    for i in range(A.nb):
        lo, hi = A.rowptr[i], A.rowptr[i + 1]
        d = [e for e in range(lo, hi) if A.col[e] == i]
        if len(d) != 1:
            raise ValueError(f"block row {i} has no single diagonal block")
        Dinv = np.linalg.inv(A.val[d[0]])
        for e in range(lo, hi):
            val[e] = Dinv @ A.val[e]
    return BsrMatrix(A.rowptr, A.col, val)


def abf_scale(A: BsrMatrix, v) -> np.ndarray:
    """D^{-1} v for the ABF operator D of A (block diagonal of A)."""
    v = np.asarray(v, np.float64).reshape(A.nb, A.bs)
    out = np.empty_like(v)
    for i in range(A.nb):
        for e in range(A.rowptr[i], A.rowptr[i + 1]):
            if A.col[e] == i:
                out[i] = np.linalg.solve(A.val[e], v[i])
    return out.ravel()


def pad_two_phase(A: BsrMatrix) -> BsrMatrix:
    """A 2x2 BSR matrix of the two-phase model (unknowns p_o, S_w) as 3x3
    blocks with a third unknown that only its own unit diagonal touches, so
    that the three-phase CPR applies; its solution is the 2x2 one with a zero
    third component."""
    val = np.zeros((A.val.shape[0], 3, 3))
    val[:, :2, :2] = A.val
    for i in range(A.nb):
        for e in range(A.rowptr[i], A.rowptr[i + 1]):
            if A.col[e] == i:
                val[e, 2, 2] = 1.0
    return BsrMatrix(A.rowptr, A.col, val)


def solve_two_phase(A: BsrMatrix, b, dims, tol=1e-13, m=30, maxit=5000):
    """x with ||b - A x|| <= tol ||b|| for a two-phase 2x2 system on an
    nx x ny x nz grid: GMRES(m) with the CPR of the padded matrix (block
    ILU(0) and AMG on the pressure block; natural-order ILU(0) alone stalls
    on the pressure part).  Returns (x (2N), info)."""
    P3 = pad_two_phase(A)
    b3 = np.zeros((A.nb, 3))
    b3[:, :2] = np.asarray(b, np.float64).reshape(A.nb, 2)
    x3, info = gmres(P3, b3.ravel(), m=m, maxit=maxit, tol=tol, prec=cpr_prec(P3, dims))
    return x3.reshape(A.nb, 3)[:, :2].ravel().copy(), info


def red_black_perm(nx, ny, nz) -> np.ndarray:
    perm = np.zeros(nx * ny * nz, np.int64)
    lib().or_red_black_perm(nx, ny, nz, _p(perm, _I64))
    return perm


def permute(A: BsrMatrix, perm) -> BsrMatrix:
    """P A P^T with perm[new] = old."""
    perm = np.ascontiguousarray(perm, np.int64)
    orow = np.zeros_like(A.rowptr)
    ocol = np.zeros_like(A.col)
    oval = np.zeros_like(A.val)
    lib().or_bsr_permute(*A.args(), _p(perm, _I64), _p(orow, _I32), _p(ocol, _I32), _p(oval, _D))
    return BsrMatrix(orow, ocol, oval)


def ilu0(A: BsrMatrix) -> BsrMatrix:
    """Block ILU(0) factors (L unit lower, U upper) on A's pattern, in A's
    ordering (paper Sec. 3.2: ILU(0) as the RAS local solver)."""
    lu = np.zeros_like(A.val)
    rc = lib().or_bsr_ilu0(*A.args(), _p(lu, _D))
    if rc != 0:
        raise ArithmeticError("ILU(0): singular pivot block")
    return BsrMatrix(A.rowptr, A.col, lu)


def ilu0_solve(LU: BsrMatrix, r) -> np.ndarray:
    r = _d(r)
    z = np.zeros(LU.n)
    lib().or_bsr_ilu0_solve(*LU.args(), _p(r, _D), _p(z, _D))
    return z


def dense_solve(A, b) -> np.ndarray:
    A = _d(A)
    b = _d(b)
    x = np.zeros(b.size)
    rc = lib().or_dense_solve(ctypes.c_int(b.size), _p(A, _D), _p(b, _D), _p(x, _D))
    if rc != 0:
        raise ArithmeticError("dense LU: zero pivot")
    return x


def rel_residual(A: BsrMatrix, b, x) -> float:
    """||b - A x|| / ||b|| with compensated sums (Alg. 1 criterion)."""
    b = _d(b)
    x = _d(x)
    return lib().or_rel_residual(*A.args(), _p(b, _D), _p(x, _D))


def pressure_block(A: BsrMatrix):
    """Scalar CSR (rowptr, col, val) of the (0, 0) entry of every block."""
    return A.rowptr.copy(), A.col.copy(), np.ascontiguousarray(A.val[:, 0, 0])


class AmgParams:
    def __init__(self, smoother=SMOOTHER_RBGS, nu1=2, nu2=2, omega=2.0 / 3.0, overcorr=1.3, coarse_max=128,
                 max_levels=20):
        self.smoother, self.nu1, self.nu2, self.omega = smoother, nu1, nu2, omega
        self.overcorr, self.coarse_max, self.max_levels = overcorr, coarse_max, max_levels

    def args(self):
        return (self.smoother, self.nu1, self.nu2, self.omega, self.overcorr, self.coarse_max, self.max_levels)


class Amg:
    """Aggregation AMG V-cycle on a scalar matrix on an nx x ny x nz grid
    (the AMG(A_pp) stage of paper Alg. 2)."""

    def __init__(self, rowptr, col, val, dims, params: AmgParams = None):
        self.params = params or AmgParams()
        self._keep = (_i(rowptr), _i(col), _d(val))
        st = ctypes.c_int(0)
        n = self._keep[0].size - 1
        self.h = lib().or_amg_create(n, _p(self._keep[0], _I32), _p(self._keep[1], _I32), _p(self._keep[2], _D),
                                     dims[0], dims[1], dims[2], *self.params.args(), ctypes.byref(st))
        if st.value != 0:
            raise ArithmeticError("AMG setup: singular coarsest matrix")

    @property
    def nlevels(self):
        return lib().or_amg_nlevels(self.h)

    def dims(self, l):
        d = (ctypes.c_int * 3)()
        lib().or_amg_level_dims(self.h, l, d)
        return tuple(d)

    def level_matrix(self, l):
        L = lib()
        nnz = L.or_amg_level_matrix(self.h, l, None, None, None)
        n = int(np.prod(self.dims(l)))
        rp = np.zeros(n + 1, np.int32)
        c = np.zeros(nnz, np.int32)
        v = np.zeros(nnz)
        L.or_amg_level_matrix(self.h, l, _p(rp, _I32), _p(c, _I32), _p(v, _D))
        return rp, c, v

    def vcycle(self, f) -> np.ndarray:
        f = _d(f)
        x = np.zeros(f.size)
        lib().or_amg_vcycle(self.h, _p(f, _D), _p(x, _D))
        return x

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.or_amg_destroy(self.h)
            self.h = None


class Prec:
    """A preconditioner handle: ILU(0) or CPR-FPF (paper Alg. 2)."""

    def __init__(self, h, keep):
        self.h, self._keep = h, keep

    def apply(self, r) -> np.ndarray:
        r = _d(r)
        z = np.zeros(r.size)
        lib().or_prec_apply(self.h, _p(r, _D), _p(z, _D))
        return z

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.or_prec_destroy(self.h)
            self.h = None


ORDER_NATURAL = 0
ORDER_RED_BLACK = 1
STAGE_CPR = 0
STAGE_ILU = 1
STAGE_AMG = 2
STAGE_CPR_DECOUPLED = 3


def ilu0_prec(A: BsrMatrix, ordering=ORDER_NATURAL, dims=(1, 1, 1)) -> Prec:
    st = ctypes.c_int(0)
    h = lib().or_prec_ilu0_create(*A.args(), ordering, dims[0], dims[1], dims[2], ctypes.byref(st))
    p = Prec(h, (A,))
    if st.value != 0:
        raise ArithmeticError("ILU(0): singular pivot block")
    return p


def cpr_prec(A: BsrMatrix, dims, ordering=ORDER_RED_BLACK, amg: AmgParams = None, stage=STAGE_CPR) -> Prec:
    """CPR-FPF of the undecoupled A (paper Alg. 2 on D_QI^{-1} A)."""
    amg = amg or AmgParams()
    st = ctypes.c_int(0)
    h = lib().or_prec_cpr_create(ctypes.c_int64(A.nb), _p(A.rowptr, _I32), _p(A.col, _I32), _p(A.val, _D),
                                 dims[0], dims[1], dims[2], ordering, *amg.args(), stage, ctypes.byref(st))
    p = Prec(h, (A,))
    if st.value != 0:
        raise ArithmeticError("CPR setup breakdown")
    return p


def cpr_set_coarse(prec: Prec, zc, dims, tile):
    """Learned coarse space of a CPR preconditioner (no counterpart in the
    paper): Z = tile restriction of the pressure field zc (natural order),
    E = Z^T A~_pp Z; every pressure correction gains Z E^{-1} Z^T f.
    zc None removes it."""
    if zc is None:
        lib().or_prec_cpr_set_coarse(prec.h, None, *dims, *tile)
        return
    zc = _d(zc)
    prec._keep = prec._keep + (zc,)
    if lib().or_prec_cpr_set_coarse(prec.h, _p(zc, _D), *dims, *tile) != 0:
        raise ArithmeticError("singular learned coarse matrix")


def cpr_coarse_apply(prec: Prec, fp):
    """The learned coarse correction alone: Z E^{-1} Z^T fp."""
    fp = _d(fp)
    ep = np.zeros_like(fp)
    lib().or_prec_cpr_coarse_apply(prec.h, _p(fp, _D), _p(ep, _D))
    return ep


def gmres(A: BsrMatrix, b, x0=None, m=30, maxit=1000, tol=1e-8, prec: Prec = None):
    """Restarted right-preconditioned GMRES(m) with MGS.  Returns
    (x, info) with info = dict(iters, relres, restarts, converged)."""
    b = _d(b)
    x = np.zeros(b.size) if x0 is None else _d(x0).copy()
    info = np.zeros(4)
    rc = lib().or_gmres(*A.args(), _p(b, _D), _p(x, _D), m, maxit, tol, prec.h if prec else None, _p(info, _D))
    return x, dict(iters=int(info[0]), relres=float(info[1]), restarts=int(info[2]), converged=(rc == 0))


def bicgstab(A: BsrMatrix, b, x0=None, maxit=1000, tol=1e-8, prec: Prec = None):
    """Right-preconditioned BiCGSTAB (two preconditioner applications and two
    products per iteration).  Returns (x, info) with info = dict(iters,
    relres, restarts, converged, breakdown)."""
    b = _d(b)
    x = np.zeros(b.size) if x0 is None else _d(x0).copy()
    info = np.zeros(4)
    rc = lib().or_bicgstab(*A.args(), _p(b, _D), _p(x, _D), maxit, tol, prec.h if prec else None, _p(info, _D))
    return x, dict(iters=int(info[0]), relres=float(info[1]), restarts=int(info[2]), converged=(rc == 0),
                   breakdown=(rc == -6))
