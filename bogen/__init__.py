"""Seeded synthetic inputs for the black-oil Jacobian solver.

This package builds the Newton systems A dx = b that both the GPU solver and
the CPU oracle consume: seeded permeability/porosity fields, reservoir states
and wells (``fields``), and the fully implicit black-oil residual and exact
Jacobian (``assembly.cpp``; paper Sec. 2.1 Eq. 3, Sec. 2.3 Eq. 4, Alg. 1).
It holds none of the linear solver's arithmetic.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# BO_BOGEN_LIB names a prebuilt library to load instead (the generator pins'
# planted-mistake checks compile altered copies of assembly.cpp)
_LIB_PATH = os.environ.get("BO_BOGEN_LIB") or os.path.join(_HERE, "libbogen.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile assembly.cpp into libbogen.so (plain g++, no arch flags)."""
    src = os.path.join(_HERE, "assembly.cpp")
    if os.environ.get("BO_BOGEN_LIB"):
        return _LIB_PATH
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(src):
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", src, "-o", _LIB_PATH])
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_LIB_PATH)
        _lib.bg_peaceman_wi.restype = ctypes.c_double
        _lib.bg_peaceman_wi.argtypes = [ctypes.c_double] * 7
        _lib.bg_cell_mass.restype = ctypes.c_double
        _lib.bg_cell_mass.argtypes = [ctypes.POINTER(Fluid), ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_double, ctypes.c_int]
        _lib.bg_nnzb.restype = ctypes.c_int64
        _lib.bg_assemble.restype = ctypes.c_int
        _lib.bg_well_border.restype = ctypes.c_int
    return _lib


class Fluid(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in (
        "pref", "bw0", "cw", "muw", "bo0", "dbo", "rs0", "drs", "muo", "bg0", "dbg", "mug",
        "rhow_sc", "rhoo_sc", "rhog_sc", "cr", "swc", "sorw", "sorg", "sgc",
        "nw", "now", "ng", "nog", "gravity")]


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double)]


class BC(ctypes.Structure):
    _fields_ = [("enabled", ctypes.c_int32), ("p_left", ctypes.c_double), ("p_right", ctypes.c_double)]


def default_fluid(**over) -> Fluid:
    """Fluid/rock constants used for every synthetic case (the paper gives
    none for synthetic data): linear FVF and Rs tables about 3000 psi, Corey
    exponent 2 curves with s_wc = 0.1, s_orw = s_org = 0.1, s_gc = 0."""
    v = dict(pref=3000.0, bw0=1.0, cw=3e-6, muw=0.5,
             bo0=1.25, dbo=6e-5, rs0=0.6, drs=1.5e-4, muo=1.0,
             bg0=0.9, dbg=1.5e-4, mug=0.02,
             rhow_sc=62.4, rhoo_sc=50.0, rhog_sc=0.06, cr=4e-6,
             swc=0.1, sorw=0.1, sorg=0.1, sgc=0.0,
             nw=2.0, now=2.0, ng=2.0, nog=2.0, gravity=1.0)
    v.update(over)
    return Fluid(**v)


def incompressible_fluid(**over) -> Fluid:
    """Test fluid: constant FVFs, Rs and porosity, no gravity."""
    v = dict(cw=0.0, dbo=0.0, drs=0.0, dbg=0.0, cr=0.0, gravity=0.0)
    v.update(over)
    return default_fluid(**v)


@dataclass
class Well:
    kind: int            # 0 water injector, 1 producer
    bhp: float           # psi at dref (for a rate-controlled well: the current value of its unknown p_h)
    cells: np.ndarray    # perforated cell indices (int32)
    dref: float = 0.0    # reference depth of bhp; default: the top perforation
    control: int = 0     # 0 fixed BHP; 1 water, 2 oil, 3 liquid rate (paper Sec. 2.3)
    rate: float = 0.0    # the controlled rate into the reservoir, stb/day (> 0 injects, < 0 produces)


CTRL_BHP, CTRL_WATER, CTRL_OIL, CTRL_LIQUID = 0, 1, 2, 3


@dataclass
class Case:
    """One Newton system's worth of synthetic input."""
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    kx: np.ndarray
    ky: np.ndarray
    kz: np.ndarray
    phi0: np.ndarray
    depth: np.ndarray
    x: np.ndarray        # state (p, Sw, Sg) interleaved, 3N
    xn: np.ndarray       # previous time level
    dt: float
    wells: list = field(default_factory=list)
    fluid: Fluid = None
    bc: BC = None
    rw: float = 0.25

    @property
    def N(self) -> int:
        return self.nx * self.ny * self.nz

    def grid(self) -> Grid:
        return Grid(self.nx, self.ny, self.nz, self.dx, self.dy, self.dz)


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _ptr(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def well_index(case: Case, c: int) -> float:
    L = lib()
    return L.bg_peaceman_wi(float(case.kx[c]), float(case.ky[c]), case.dx, case.dy, case.dz, case.rw, 0.0)


def pattern(nx, ny, nz):
    """7-point BSR pattern (rowptr int32[N+1], col int32[nnzb])."""
    L = lib()
    g = Grid(nx, ny, nz, 1.0, 1.0, 1.0)
    nnzb = L.bg_nnzb(ctypes.byref(g))
    rowptr = np.zeros(nx * ny * nz + 1, np.int32)
    col = np.zeros(nnzb, np.int32)
    L.bg_pattern(ctypes.byref(g), _ptr(rowptr, ctypes.c_int32), _ptr(col, ctypes.c_int32))
    return rowptr, col


def rate_wells(case: Case):
    """The case's rate-controlled wells, in well order (the order of the
    bordered system's well unknowns)."""
    return [w for w in case.wells if w.control != CTRL_BHP]


def _bhps(case: Case, ph):
    """Every well's BHP, the rate-controlled ones taken from ph (if given)."""
    out, v = [], 0
    for w in case.wells:
        if w.control != CTRL_BHP and ph is not None:
            out.append(float(ph[v]))
            v += 1
        else:
            out.append(float(w.bhp))
    return out


def assemble(case: Case, jacobian: bool = True, x=None, ph=None):
    """Residual R (3N) and BSR Jacobian of ``case``.

    Returns dict(rowptr, col, val (nnzb,3,3), R, b=-R).  Raises on a bad state.
    With rate-controlled wells (Well.control != 0) their bottom-hole
    pressures are unknowns too: ph (one per such well, in well order;
    default: their Well.bhp) gives their values, and the result also holds
    `border` = dict(perf_cell, perf_well (the well unknown of each
    perforation), apw (P,3), awp (P,3), aww (W,), Rw (W,), bw = -Rw) of the
    bordered Newton system (paper Sec. 2.3 and Sec. 3.2), and the full
    right-hand side b_full = (b, bw).
    """
    L = lib()
    g = case.grid()
    fl = case.fluid if case.fluid is not None else default_fluid()
    rowptr, col = pattern(case.nx, case.ny, case.nz)
    nnzb = col.size
    R = np.zeros(3 * case.N)
    val = np.zeros((nnzb, 3, 3)) if jacobian else None
    xs = _d(case.x if x is None else x)
    wt = _i([w.kind for w in case.wells]) if case.wells else np.zeros(1, np.int32)
    bhp = _d(_bhps(case, ph)) if case.wells else np.zeros(1)
    dref = _d([w.dref if w.dref else case.depth[int(np.min(w.cells))] for w in case.wells]) if case.wells else np.zeros(1)
    pptr = [0]
    cells, wis = [], []
    for w in case.wells:
        for c in np.asarray(w.cells).ravel():
            cells.append(int(c))
            wis.append(well_index(case, int(c)))
        pptr.append(len(cells))
    pptr = _i(pptr)
    cells = _i(cells if cells else [0])
    wis = _d(wis if wis else [0.0])
    kx, ky, kz, phi0, depth, xn = map(_d, (case.kx, case.ky, case.kz, case.phi0, case.depth, case.xn))
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int32)
    rc = L.bg_assemble(ctypes.byref(g), ctypes.byref(fl),
                       _ptr(kx, ctypes.c_double), _ptr(ky, ctypes.c_double), _ptr(kz, ctypes.c_double),
                       _ptr(phi0, ctypes.c_double), _ptr(depth, ctypes.c_double),
                       _ptr(xs, ctypes.c_double), _ptr(xn, ctypes.c_double), ctypes.c_double(case.dt),
                       ctypes.c_int32(len(case.wells)), _ptr(wt, ctypes.c_int32), _ptr(bhp, ctypes.c_double),
                       _ptr(dref, ctypes.c_double), _ptr(pptr, ctypes.c_int32), _ptr(cells, ctypes.c_int32),
                       _ptr(wis, ctypes.c_double),
                       ctypes.byref(case.bc) if case.bc is not None else None,
                       _ptr(rowptr, ctypes.c_int32), _ptr(col, ctypes.c_int32),
                       _ptr(R, ctypes.c_double),
                       _ptr(val, ctypes.c_double) if val is not None else ctypes.cast(None, dp))
    if rc != 0:
        raise ValueError("assembly failed: non-positive pore volume or FVF")
    out = dict(rowptr=rowptr, col=col, val=val, R=R, b=-R)
    rw = rate_wells(case)
    if rw:
        W = len(rw)
        P = sum(np.asarray(w.cells).size for w in rw)
        ctrl = _i([w.control for w in case.wells])
        rate = _d([w.rate for w in case.wells])
        Rw, aww = np.zeros(W), np.zeros(W)
        apw, awp = np.zeros((P, 3)), np.zeros((P, 3))
        nv = L.bg_well_border(ctypes.byref(fl), _ptr(phi0, ctypes.c_double), _ptr(depth, ctypes.c_double),
                              _ptr(xs, ctypes.c_double), ctypes.c_int32(len(case.wells)), _ptr(wt, ctypes.c_int32),
                              _ptr(ctrl, ctypes.c_int32), _ptr(rate, ctypes.c_double), _ptr(bhp, ctypes.c_double),
                              _ptr(dref, ctypes.c_double), _ptr(pptr, ctypes.c_int32), _ptr(cells, ctypes.c_int32),
                              _ptr(wis, ctypes.c_double), _ptr(Rw, ctypes.c_double), _ptr(apw, ctypes.c_double),
                              _ptr(awp, ctypes.c_double), _ptr(aww, ctypes.c_double))
        if nv != W:
            raise ValueError("invalid well control (an injector under an oil-rate control)")
        pc = np.concatenate([np.asarray(w.cells, np.int32).ravel() for w in rw])
        pw = np.concatenate([np.full(np.asarray(w.cells).size, v, np.int32) for v, w in enumerate(rw)])
        out["border"] = dict(perf_cell=pc, perf_well=pw, apw=apw, awp=awp, aww=aww, Rw=Rw, bw=-Rw)
        out["b_full"] = np.concatenate([-R, -Rw])
    return out


def with_rate_controls(case: Case, fraction: float = 0.8, producer_control: int = CTRL_LIQUID):
    """A copy of ``case`` whose wells are rate-controlled: injectors under a
    water rate, producers under `producer_control`, each target `fraction`
    of the well's current rate at its BHP (so the bordered residual of the
    case's state is nonzero in the well rows)."""
    import copy
    c = copy.deepcopy(case)
    for w in c.wells:
        w.control = CTRL_WATER if w.kind == 0 else producer_control
        w.rate = 0.0
    a = assemble(c, jacobian=False)
    for w, r in zip(rate_wells(c), a["border"]["Rw"]):
        w.rate = fraction * float(r)
    return c


def model_inputs(case: Case) -> dict:
    """The case's rock, wells and fluid as plain arrays, for a consumer that
    assembles the same residual itself: kx, ky, kz, phi0, depth per cell; one
    entry per perforation of perf_cell, perf_type (0 injector, 1 producer),
    perf_bhp, perf_dref (the well's reference depth: its top perforation
    unless given) and perf_wi (the Peaceman index the assembly uses); fluid
    as a dict of the Fluid fields."""
    fl = case.fluid if case.fluid is not None else default_fluid()
    pc, pt, pb, pd, pw = [], [], [], [], []
    for w in case.wells:
        cells = np.asarray(w.cells).ravel()
        dref = w.dref if w.dref else case.depth[int(np.min(cells))]
        for c in cells:
            pc.append(int(c))
            pt.append(int(w.kind))
            pb.append(float(w.bhp))
            pd.append(float(dref))
            pw.append(well_index(case, int(c)))
    return dict(kx=_d(case.kx), ky=_d(case.ky), kz=_d(case.kz), phi0=_d(case.phi0), depth=_d(case.depth),
                perf_cell=np.asarray(pc, np.int32), perf_type=np.asarray(pt, np.int32), perf_bhp=_d(pb),
                perf_dref=_d(pd), perf_wi=_d(pw), fluid={k: getattr(fl, k) for k, _ in fl._fields_})


def cell_mass(fluid: Fluid, phi0, p, sw, sg, comp) -> float:
    return lib().bg_cell_mass(ctypes.byref(fluid), phi0, p, sw, sg, comp)


def relperm(fluid: Fluid, sw: float, sg: float):
    out = np.zeros(3)
    lib().bg_relperm(ctypes.byref(fluid), ctypes.c_double(sw), ctypes.c_double(sg), _ptr(out, ctypes.c_double))
    return out


from .fields import tiny_case, waterflood_case, gaussian_field, uniform_case, ensemble_specs, ensemble_case  # noqa: E402,F401,E501
from . import learned  # noqa: E402,F401
from . import dual  # noqa: E402,F401


# ------------------------------------------------------------ two-phase oil-water
def oil_water_fluid(**over) -> Fluid:
    """Fluid of the two-phase oil-water model (paper Sec. 2.2): dead oil
    (Rs = 0, no gas phase) with a compressibility of 1e-5 / psi (B_o =
    1.25 (1 - 1e-5 (p - 3000)); the three-phase table's B_o grows with p,
    which only dissolved gas makes physical: without it the oil would expand
    under compression and the pressure equation lose its definiteness), and
    the paper's SPE10 relative permeabilities k_rw = ((s_w - s_wc)/(1 - s_wc -
    s_or))^2, k_ro = ((1 - s_or - s_w)/(1 - s_wc - s_or))^2 with s_wc = s_or =
    0.2; other constants as default_fluid."""
    v = dict(rs0=0.0, drs=0.0, dbo=-1.25e-5, swc=0.2, sorw=0.2, sorg=0.2, sgc=0.0, nw=2.0, now=2.0)
    v.update(over)
    return default_fluid(**v)


def oil_water_case(nx: int = 128, ny: int = 128, nz: int = 64, seed: int = 42, **kw) -> Case:
    """A two-phase oil-water case on the waterflood generator's grid, rock
    and wells: the same permeability field and five-spot wells, the water
    front's saturations mapped from [0.1, 0.85] onto [s_wc, 1 - s_or] =
    [0.2, 0.8], no gas (Sg = 0 in the state vectors)."""
    from .fields import waterflood_case
    c = waterflood_case(nx, ny, nz, seed=seed, **kw)
    for v in (c.x, c.xn):
        sw = v[1::3]
        v[1::3] = 0.2 + (sw - 0.1) * (0.6 / 0.75)
        v[2::3] = 0.0
    c.fluid = oil_water_fluid()
    return c


def tiny_oil_water_case(seed: int = 0, nx: int = 20, ny: int = 20, nz: int = 5) -> Case:
    """The tiny case's grid, rock and wells with the two-phase fluid: state
    (3000 psi, Sw 0.3) times U[0.95, 1.05] per unknown, previous state
    uniform, Sg = 0."""
    from .fields import tiny_case
    c = tiny_case(seed, nx, ny, nz)
    rng = np.random.default_rng(seed + 1000)
    N = c.N
    c.xn = np.tile([3000.0, 0.3, 0.0], N)
    c.x = c.xn * np.concatenate([rng.uniform(0.95, 1.05, (N, 2)), np.ones((N, 1))], axis=1).ravel()
    c.fluid = oil_water_fluid()
    return c


def assemble_ow(case: Case, jacobian: bool = True, x=None):
    """Residual and 2x2 BSR Jacobian of the two-phase oil-water model (paper
    Sec. 2.2): unknowns (p_o, S_w) and equations (oil, water) per cell.

    The model is the three-phase one without gas: with Sg = 0 and Rs = 0 the
    gas phase has no mass, flux or well rate, Stone II reduces to k_row
    (k_ro(S_w, 0) = k_row(S_w)), and the oil and water equations are exactly
    Sec. 2.2's.  So the residual is the three-phase residual's (oil, water)
    rows at Sg = 0 and the Jacobian the (oil, water) x (p, S_w) part of each
    block.  x: the two-phase state (2N), default the case's.  Returns
    dict(rowptr, col, val (nnzb,2,2), R (2N), b = -R)."""
    N = case.N
    if x is None:
        x3 = np.asarray(case.x, np.float64)
    else:
        x2 = np.asarray(x, np.float64).reshape(N, 2)
        x3 = np.concatenate([x2, np.zeros((N, 1))], axis=1).ravel()
    a = assemble(case, jacobian=jacobian, x=x3)
    R = a["R"].reshape(N, 3)[:, :2].ravel().copy()
    val = a["val"][:, :2, :2].copy() if jacobian else None
    return dict(rowptr=a["rowptr"], col=a["col"], val=val, R=R, b=-R)


def state_ow(case: Case) -> np.ndarray:
    """The case's two-phase state (p_o, S_w) per cell."""
    return np.asarray(case.x, np.float64).reshape(-1, 3)[:, :2].ravel().copy()
