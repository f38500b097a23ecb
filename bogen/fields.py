"""Seeded synthetic reservoirs: permeability fields, states and wells.

Every array is indexed by cell c = i + nx (j + ny k) (numpy shape (nz, ny, nx)
flattened in C order).  Randomness comes only from numpy's PCG64
``default_rng(seed)``.  The workloads stand in for the paper's refined
SPE10/SPE1 models (Sec. 4), which are not available: log-normal permeability
with the stated correlation lengths, Corey curves, a five-spot pattern.
"""
from __future__ import annotations

import numpy as np

from . import Case, Well, default_fluid

TOP_DEPTH = 8000.0  # ft, depth of the top face of layer 0


def gaussian_field(shape_zyx, corr_zyx, rng) -> np.ndarray:
    """White noise filtered by a Gaussian of std ``corr`` cells per axis
    (periodic, via FFT), renormalised to zero mean and unit variance."""
    w = rng.standard_normal(shape_zyx)
    F = np.fft.fftn(w)
    k = np.meshgrid(*[np.fft.fftfreq(n) for n in shape_zyx], indexing="ij")
    H = np.exp(-2.0 * np.pi ** 2 * sum((s * kk) ** 2 for s, kk in zip(corr_zyx, k)))
    g = np.real(np.fft.ifftn(F * H))
    g -= g.mean()
    sd = g.std()
    return g / sd if sd > 0 else g


def _depths(nx, ny, nz, dz):
    k = np.arange(nz, dtype=np.float64)
    d = TOP_DEPTH + (k + 0.5) * dz
    return np.broadcast_to(d[:, None, None], (nz, ny, nx)).ravel().copy()


def _column(nx, ny, nz, i, j):
    return np.array([i + nx * (j + ny * k) for k in range(nz)], np.int32)


def tiny_case(seed: int = 0, nx: int = 20, ny: int = 20, nz: int = 5) -> Case:
    """One black-oil Newton system: 100x100x20 ft cells, ln k ~ N(4, 0.5^2)
    iid per cell (mD, isotropic), porosity 0.2; previous state uniform
    (3000 psi, Sw 0.2, Sg 0.05); current state that times U[0.95, 1.05] per
    unknown; a BHP water injector (3500 psi) at column (0, 0) and a BHP
    producer (2500 psi) at (nx-1, ny-1), perforated in every layer; dt 1 day."""
    rng = np.random.default_rng(seed)
    N = nx * ny * nz
    k = np.exp(rng.normal(4.0, 0.5, N))
    xn = np.tile([3000.0, 0.2, 0.05], N)
    x = xn * rng.uniform(0.95, 1.05, 3 * N)
    wells = [Well(0, 3500.0, _column(nx, ny, nz, 0, 0)),
             Well(1, 2500.0, _column(nx, ny, nz, nx - 1, ny - 1))]
    return Case(nx, ny, nz, 100.0, 100.0, 20.0, k, k.copy(), k.copy(), np.full(N, 0.2),
                _depths(nx, ny, nz, 20.0), x, xn, 1.0, wells, default_fluid())


def uniform_case(nx, ny, nz, k=100.0, p=3000.0, sw=0.2, sg=0.05, dx=100.0, dy=100.0, dz=20.0,
                 fluid=None, wells=None, dt=1.0) -> Case:
    """Homogeneous reservoir in a uniform state (used by the physics pins)."""
    N = nx * ny * nz
    kk = np.full(N, float(k))
    st = np.tile([p, sw, sg], N).astype(np.float64)
    return Case(nx, ny, nz, dx, dy, dz, kk, kk.copy(), kk.copy(), np.full(N, 0.2),
                _depths(nx, ny, nz, dz), st, st.copy(), dt, wells or [],
                fluid if fluid is not None else default_fluid())


def waterflood_case(nx: int = 128, ny: int = 128, nz: int = 64, seed: int = 42, day: int = 0,
                    sigma: float = 1.5, corr=(16.0, 16.0, 2.0), kvkh: float = 0.1,
                    front0: float = 40.0, front_speed: float = 2.0,
                    inj_bhp: float = 4000.0, prod_bhp: float = 2000.0) -> Case:
    """Five-spot waterflood, the first Newton system of day ``day``.

    ln k_h = 4 + sigma g, g a Gaussian-filtered unit-variance field with
    correlation std ``corr`` = (x, y, z) cells; k_v = kvkh k_h; porosity 0.2.
    Sw = 0.1 + 0.75 (1 - tanh((d - R_t)/4))/2 with d the horizontal distance
    (cells) to the nearest injector plus 3-cell-smoothed noise and the front
    radius R_t = front0 + front_speed * day; Sg = 0.05; p = 3000 psi plus
    the oil hydrostatic gradient below the top.  Injectors (BHP 4000 psi) at
    the four corner columns, producer (BHP 2000 psi) at the centre column,
    all layers.  The Newton iterate equals the previous time level (the
    first Newton system of a step), dt = 1 day.
    """
    rng = np.random.default_rng(seed)
    shape = (nz, ny, nx)
    g = gaussian_field(shape, (corr[2], corr[1], corr[0]), rng)
    kh = np.exp(4.0 + sigma * g).ravel()
    kv = kvkh * kh
    noise = gaussian_field(shape, (1.0, 3.0, 3.0), rng)
    inj = [(0, 0), (nx - 1, 0), (0, ny - 1), (nx - 1, ny - 1)]
    jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    d = np.min([np.hypot(ii - a, jj - b) for a, b in inj], axis=0)
    dd = d[None, :, :] + 3.0 * noise
    R = front0 + front_speed * day
    sw = 0.1 + 0.75 * 0.5 * (1.0 - np.tanh((dd - R) / 4.0))
    N = nx * ny * nz
    depth = _depths(nx, ny, nz, 20.0)
    p = 3000.0 + 0.35 * (depth - TOP_DEPTH)
    x = np.empty(3 * N)
    x[0::3] = p
    x[1::3] = sw.ravel()
    x[2::3] = 0.05
    wells = [Well(0, inj_bhp, _column(nx, ny, nz, a, b)) for a, b in inj]
    wells.append(Well(1, prod_bhp, _column(nx, ny, nz, nx // 2, ny // 2)))
    return Case(nx, ny, nz, 100.0, 100.0, 20.0, kh, kh.copy(), kv, np.full(N, 0.2),
                depth, x, x.copy(), 1.0, wells, default_fluid())


def ensemble_specs(n: int = 256, seed: int = 7, total_unknowns=(38e6, 42e6), max_draws: int = 10000):
    """Grid sizes and parameters of a batch of realisations of uneven size.

    nx, ny ~ log-uniform[32, 96] and nz ~ log-uniform[8, 24], rounded to
    integers (nx then rounded up to even: the solver's red-black layout pairs
    the cells of a grid row); the draw is repeated until the total number of
    unknowns 3 sum(nx ny nz) lies in `total_unknowns`.  Each realisation gets
    its own seed and a permeability sigma ~ U[0.5, 2.0].  Returns a list of
    dicts (dims, sigma, seed)."""
    rng = np.random.default_rng(seed)
    lo, hi = total_unknowns
    for _ in range(max_draws):
        nx = np.exp(rng.uniform(np.log(32), np.log(96), n)).round().astype(int)
        nx += nx % 2
        ny = np.exp(rng.uniform(np.log(32), np.log(96), n)).round().astype(int)
        nz = np.exp(rng.uniform(np.log(8), np.log(24), n)).round().astype(int)
        tot = 3 * int(np.sum(nx * ny * nz))
        if lo <= tot <= hi:
            sig = rng.uniform(0.5, 2.0, n)
            seeds = rng.integers(0, 2 ** 31 - 1, n)
            return [dict(dims=(int(a), int(b), int(c)), sigma=float(s), seed=int(q))
                    for a, b, c, s, q in zip(nx, ny, nz, sig, seeds)]
    raise RuntimeError("no draw within the unknown-count window")


def ensemble_case(spec) -> Case:
    """One realisation of the ensemble: the five-spot waterflood generator on
    the realisation's grid, with correlation lengths and front radius scaled
    to the grid (1/8 of the horizontal size, 1/8 of the layers)."""
    nx, ny, nz = spec["dims"]
    corr = (max(1.0, nx / 8), max(1.0, ny / 8), max(1.0, nz / 8))
    return waterflood_case(nx, ny, nz, seed=spec["seed"], day=0, sigma=spec["sigma"], corr=corr,
                           front0=0.3 * min(nx, ny), front_speed=0.0)
