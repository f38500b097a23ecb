"""Seeded inputs of the learned Newton update: reservoirs with one injector
and one producer, the network's input features and the scaling of its
targets.

The cases stand in for states a simulation would reach after a few days:
a smooth pressure field around the hydrostatic gradient and a water front
of random radius around the injector (the first Newton system of a step,
so x = x_n).  Randomness comes only from numpy's PCG64 default_rng(seed).
"""
from __future__ import annotations

import numpy as np

from . import Case, Well, default_fluid, well_index
from .fields import TOP_DEPTH, _column, _depths, gaussian_field

N_FEATURES = 6
N_CHANNELS = 16          # network input channels (features zero-padded)
TARGET_SCALE = (100.0, 0.01, 0.01)  # psi, -, -: targets are dx / TARGET_SCALE


def learned_case(seed: int, nx: int = 64, ny: int = 64, nz: int = 32) -> Case:
    """One realisation: ln k_h = 4 + sigma g with sigma ~ U[0.5, 2.0] and g a
    Gaussian-filtered field of correlation (nx/8, ny/8, nz/32) cells,
    k_v = 0.1 k_h; an injector (BHP ~ U[3500, 4500] psi) and a producer
    (BHP ~ U[1500, 2500] psi) at uniform-random columns at least
    min(16, nx/2, ny/2) cells apart, perforated in every layer;
    p = 3000 + 0.35 (depth - top) + 150 h psi (h a smooth unit field);
    Sw = 0.1 + 0.75 (1 - tanh((d - R)/3))/2 around the injector with
    R ~ U[0, min(nx, ny)/2] cells; Sg = 0.05; dt = 1 day."""
    rng = np.random.default_rng(seed)
    sigma = rng.uniform(0.5, 2.0)
    shape = (nz, ny, nx)
    g = gaussian_field(shape, (max(1.0, nz / 32), max(1.0, ny / 8), max(1.0, nx / 8)), rng)
    kh = np.exp(4.0 + sigma * g).ravel()
    kv = 0.1 * kh
    dmin = min(16.0, nx / 2, ny / 2)
    while True:
        wi = rng.integers(0, nx, 2)
        wj = rng.integers(0, ny, 2)
        if np.hypot(wi[0] - wi[1], wj[0] - wj[1]) >= dmin:
            break
    inj_bhp = rng.uniform(3500.0, 4500.0)
    prod_bhp = rng.uniform(1500.0, 2500.0)
    h = gaussian_field(shape, (max(1.0, nz / 8), max(1.0, ny / 4), max(1.0, nx / 4)), rng)
    depth = _depths(nx, ny, nz, 20.0)
    p = 3000.0 + 0.35 * (depth - TOP_DEPTH) + 150.0 * h.ravel()
    jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    d = np.hypot(ii - wi[0], jj - wj[0])
    R = rng.uniform(0.0, min(nx, ny) / 2)
    sw = 0.1 + 0.75 * 0.5 * (1.0 - np.tanh((d - R) / 3.0))
    sw = np.broadcast_to(sw[None], shape).ravel()
    N = nx * ny * nz
    x = np.empty(3 * N)
    x[0::3] = p
    x[1::3] = sw
    x[2::3] = 0.05
    wells = [Well(0, inj_bhp, _column(nx, ny, nz, int(wi[0]), int(wj[0]))),
             Well(1, prod_bhp, _column(nx, ny, nz, int(wi[1]), int(wj[1])))]
    return Case(nx, ny, nz, 100.0, 100.0, 20.0, kh, kh.copy(), kv, np.full(N, 0.2),
                depth, x, x.copy(), 1.0, wells, default_fluid())


def features(case: Case) -> np.ndarray:
    """Network input [V, 16] float32, voxel v = cell index: the 6 features
    (ln k_h - 4)/2, (p - 3000)/300, (Sw - 0.5)/0.4, 20 (Sg - 0.05),
    sign ln(1 + WI) at perforated cells (+ injector, - producer) and
    (BHP - p)/1000 at perforated cells; channels 6..15 zero."""
    N = case.N
    f = np.zeros((N, N_CHANNELS), np.float32)
    p = case.x[0::3]
    f[:, 0] = (np.log(case.kx) - 4.0) / 2.0
    f[:, 1] = (p - 3000.0) / 300.0
    f[:, 2] = (case.x[1::3] - 0.5) / 0.4
    f[:, 3] = 20.0 * (case.x[2::3] - 0.05)
    for w in case.wells:
        sgn = 1.0 if w.kind == 0 else -1.0
        for c in np.asarray(w.cells).ravel():
            f[c, 4] = sgn * np.log1p(well_index(case, int(c)))
            f[c, 5] = (w.bhp - p[c]) / 1000.0
    return f


def targets(dx: np.ndarray) -> np.ndarray:
    """Network target [V, 4] float32 from a Newton update dx (3N interleaved)."""
    N = dx.size // 3
    t = np.zeros((N, 4), np.float32)
    for k in range(3):
        t[:, k] = dx[k::3] / TARGET_SCALE[k]
    return t


def sample(seed: int, dims=(64, 64, 32)):
    """(features [V, 16] f32, assembled system dict) of realisation `seed`."""
    from . import assemble
    c = learned_case(seed, *dims)
    return features(c), assemble(c)


def _sample_star(args):
    return sample(*args)


def samples(seeds, dims=(64, 64, 32), processes: int = 0):
    """Yield (features, system) for each seed in order, built on a pool of
    `processes` spawned worker processes (0: in this process).  Streaming:
    at most a few samples are held at once."""
    if processes <= 1:
        for s in seeds:
            yield sample(int(s), dims)
        return
    import multiprocessing as mp
    seeds = [int(s) for s in seeds]
    step = 2 * processes  # bounded look-ahead: the pool runs at most this far ahead of the consumer
    with mp.get_context("spawn").Pool(processes) as pool:
        for i in range(0, len(seeds), step):
            for out in pool.imap(_sample_star, [(s, tuple(dims)) for s in seeds[i:i + step]], chunksize=1):
                yield out
