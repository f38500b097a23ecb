"""Seeded dual-porosity systems: every cell carries a fracture continuum
(the flowing network, wells) and a matrix continuum (storage) exchanging
fluid through a Warren-Root transfer term (paper Sec. 2.1's dual-porosity
model).  Node c < N is cell c's fracture node, node N + c its matrix node.

Recipe (the paper gives no dual-porosity data): matrix permeability
ln k_m = 4 + sigma g (g a Gaussian-filtered unit field, sigma ~ U[0.5, 2]),
fracture permeability k_f = 10 k_m, porosities phi_f = 0.04 and
phi_m = 0.14, shape factor 0.1 ft^-2.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field

import numpy as np

from . import Fluid, Grid, Well, default_fluid, lib
from .fields import TOP_DEPTH, _column, _depths, gaussian_field

PHI_F = 0.04
PHI_M = 0.14
SIGMA = 0.1  # ft^-2


@dataclass
class DualCase:
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    kx: np.ndarray      # fracture permeabilities (mD)
    ky: np.ndarray
    kz: np.ndarray
    km: np.ndarray      # matrix permeability (mD)
    phif: np.ndarray
    phim: np.ndarray
    depth: np.ndarray
    x: np.ndarray       # 6N: fracture nodes' (p, Sw, Sg), then the matrix nodes'
    xn: np.ndarray
    dt: float
    sigma: float = SIGMA
    wells: list = field(default_factory=list)
    fluid: Fluid = None
    rw: float = 0.25

    @property
    def N(self) -> int:
        return self.nx * self.ny * self.nz

    def grid(self) -> Grid:
        return Grid(self.nx, self.ny, self.nz, self.dx, self.dy, self.dz)


def dual_pattern(nx, ny, nz):
    """(rowptr int32[2N+1], col int32[nnzb]) of the dual-porosity system."""
    L = lib()
    g = Grid(nx, ny, nz, 1.0, 1.0, 1.0)
    L.bg_dual_nnzb.restype = ctypes.c_int64
    nnzb = L.bg_dual_nnzb(ctypes.byref(g))
    N = nx * ny * nz
    rowptr = np.zeros(2 * N + 1, np.int32)
    col = np.zeros(nnzb, np.int32)
    L.bg_dual_pattern(ctypes.byref(g), rowptr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                      col.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    return rowptr, col


def dual_case(seed: int, nx: int = 20, ny: int = 20, nz: int = 5, sigma_k: float = None,
              shape_factor: float = SIGMA) -> DualCase:
    """A five-spot-like dual-porosity realisation: injector (BHP 4000 psi) at
    column (0, 0), producer (BHP 2000 psi) at (nx-1, ny-1), both perforating
    the fracture nodes of every layer.  Fracture state: p = 3000 + 0.35
    (depth - top) + 100 h psi, water front of radius (nx + ny)/4 cells
    around the injector; matrix state: p_m = p_f - 30 u psi and
    Sw_m = 0.1 + 0.5 (Sw_f - 0.1) (the matrix lags the fractures), u, h
    smooth unit fields; Sg = 0.05 in both.  The first Newton system of a
    1-day step (x = x_n)."""
    rng = np.random.default_rng(seed)
    sig = rng.uniform(0.5, 2.0) if sigma_k is None else sigma_k
    shape = (nz, ny, nx)
    g = gaussian_field(shape, (max(1.0, nz / 8), max(1.0, ny / 8), max(1.0, nx / 8)), rng)
    km = np.exp(4.0 + sig * g).ravel()
    kf = 10.0 * km
    h = gaussian_field(shape, (max(1.0, nz / 4), max(1.0, ny / 4), max(1.0, nx / 4)), rng).ravel()
    u = np.abs(gaussian_field(shape, (1.0, 2.0, 2.0), rng)).ravel()
    N = nx * ny * nz
    depth = _depths(nx, ny, nz, 20.0)
    pf = 3000.0 + 0.35 * (depth - TOP_DEPTH) + 100.0 * h
    jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    d = np.hypot(ii, jj)
    swf = 0.1 + 0.75 * 0.5 * (1.0 - np.tanh((d - (nx + ny) / 4.0) / 3.0))
    swf = np.broadcast_to(swf[None], shape).ravel()
    x = np.empty(6 * N)
    x[0:3 * N:3] = pf
    x[1:3 * N:3] = swf
    x[2:3 * N:3] = 0.05
    x[3 * N::3] = pf - 30.0 * u
    x[3 * N + 1::3] = 0.1 + 0.5 * (swf - 0.1)
    x[3 * N + 2::3] = 0.05
    wells = [Well(0, 4000.0, _column(nx, ny, nz, 0, 0)), Well(1, 2000.0, _column(nx, ny, nz, nx - 1, ny - 1))]
    return DualCase(nx, ny, nz, 100.0, 100.0, 20.0, kf, kf.copy(), kf.copy(), km, np.full(N, PHI_F),
                    np.full(N, PHI_M), depth, x, x.copy(), 1.0, shape_factor, wells, default_fluid())


def assemble_dual(case: DualCase, jacobian: bool = True):
    """Residual R (6N) and BSR Jacobian (2N block rows) of a dual-porosity
    case: dict(rowptr, col, val (nnzb, 3, 3), R, b = -R)."""
    L = lib()
    g = case.grid()
    fl = case.fluid if case.fluid is not None else default_fluid()
    rowptr, col = dual_pattern(case.nx, case.ny, case.nz)
    R = np.zeros(6 * case.N)
    val = np.zeros((col.size, 3, 3)) if jacobian else None
    d = lambda a: np.ascontiguousarray(a, dtype=np.float64)  # noqa: E731
    i32 = lambda a: np.ascontiguousarray(a, dtype=np.int32)  # noqa: E731
    wt = i32([w.kind for w in case.wells] or [0])
    bhp = d([w.bhp for w in case.wells] or [0.0])
    dref = d([w.dref if w.dref else case.depth[int(np.min(w.cells))] for w in case.wells] or [0.0])
    pptr, cells, wis = [0], [], []
    for w in case.wells:
        for c in np.asarray(w.cells).ravel():
            cells.append(int(c))
            wis.append(L.bg_peaceman_wi(float(case.kx[c]), float(case.ky[c]), case.dx, case.dy, case.dz,
                                        case.rw, 0.0))
        pptr.append(len(cells))
    pptr, cells, wis = i32(pptr), i32(cells or [0]), d(wis or [0.0])
    arrs = [d(a) for a in (case.kx, case.ky, case.kz, case.km, case.phif, case.phim, case.depth, case.x, case.xn)]
    P = lambda a, t: a.ctypes.data_as(ctypes.POINTER(t))  # noqa: E731
    D, I = ctypes.c_double, ctypes.c_int32
    L.bg_assemble_dual.restype = ctypes.c_int
    rc = L.bg_assemble_dual(ctypes.byref(g), ctypes.byref(fl), *[P(a, D) for a in arrs[:9]],
                            D(case.dt), D(case.sigma), I(len(case.wells)), P(wt, I), P(bhp, D), P(dref, D),
                            P(pptr, I), P(cells, I), P(wis, D), P(rowptr, I), P(col, I), P(R, D),
                            P(val, D) if val is not None else ctypes.cast(None, ctypes.POINTER(D)))
    if rc != 0:
        raise ValueError("dual assembly failed: non-positive pore volume or FVF")
    return dict(rowptr=rowptr, col=col, val=val, R=R, b=-R)
