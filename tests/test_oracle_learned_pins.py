"""Pins of the oracle's learned coarse space (a Galerkin coarse space
spanned by the tile restrictions of a pressure field, added to every
pressure correction of CPR): Galerkin orthogonality, exactness on its own
span, the one-tile closed form and the composition with the AMG stage."""
import numpy as np
import scipy.sparse as sp

import bogen
import oracle
from oracle import BsrMatrix


def _system(seed, dims):
    c = bogen.tiny_case(seed, *dims)
    a = bogen.assemble(c)
    return BsrMatrix(a["rowptr"], a["col"], a["val"]), a["b"]


def _tile_index(dims, tile):
    nx, ny, nz = dims
    tx, ty, tz = tile
    ntx, nty = -(-nx // tx), -(-ny // ty)
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return (i // tx + ntx * (j // ty + nty * (k // tz))).ravel()


def _Z(zc, dims, tile):
    t = _tile_index(dims, tile)
    nt = t.max() + 1
    return sp.csr_matrix((zc, (np.arange(zc.size), t)), shape=(zc.size, nt)).toarray()


def _App(A):
    At, _ = oracle.qi_decouple(A)
    rp, c, v = oracle.pressure_block(At)
    return sp.csr_matrix((v, c, rp), shape=(A.nb, A.nb)).toarray()


DIMS = (10, 8, 6)
TILE = (4, 4, 3)  # ragged tiles at the +x and +y faces


def _setup(seed=0, zc=None):
    A, _ = _system(seed, DIMS)
    P = oracle.cpr_prec(A, DIMS, stage=oracle.STAGE_AMG)
    rng = np.random.default_rng(seed + 10)
    if zc is None:
        zc = rng.uniform(0.5, 2.0, A.nb) * np.sign(rng.standard_normal(A.nb))
    oracle.cpr_set_coarse(P, zc, DIMS, TILE)
    return A, P, zc, rng


def test_galerkin_orthogonality():
    # the corrected residual is orthogonal to the coarse space: Z^T (f - A~ e) = 0
    A, P, zc, rng = _setup(0)
    f = rng.standard_normal(A.nb)
    e = oracle.cpr_coarse_apply(P, f)
    Z = _Z(zc, DIMS, TILE)
    r = Z.T @ (f - _App(A) @ e)
    assert np.abs(r).max() <= 1e-10 * np.abs(Z.T @ f).max()


def test_exact_on_its_span():
    # an error that lies in span(Z) is removed exactly: f = A~ Z c gives e = Z c
    A, P, zc, rng = _setup(1)
    Z = _Z(zc, DIMS, TILE)
    c = rng.standard_normal(Z.shape[1])
    e = oracle.cpr_coarse_apply(P, _App(A) @ (Z @ c))
    np.testing.assert_allclose(e, Z @ c, rtol=1e-9, atol=1e-12)


def test_single_tile_closed_form():
    # one tile and zc = 1: E = 1^T A~ 1 (the sum of all entries) and e = (1^T f / E) 1
    A, _ = _system(2, DIMS)
    P = oracle.cpr_prec(A, DIMS, stage=oracle.STAGE_AMG)
    oracle.cpr_set_coarse(P, np.ones(A.nb), DIMS, DIMS)
    f = np.random.default_rng(3).standard_normal(A.nb)
    e = oracle.cpr_coarse_apply(P, f)
    np.testing.assert_allclose(e, np.full(A.nb, f.sum() / _App(A).sum()), rtol=1e-12)


def test_zero_tiles_contribute_nothing():
    # tiles where zc vanishes stay out of the correction (and E stays invertible)
    A, _ = _system(3, DIMS)
    zc = np.ones(A.nb)
    zc[_tile_index(DIMS, TILE) == 0] = 0.0
    P = oracle.cpr_prec(A, DIMS, stage=oracle.STAGE_AMG)
    oracle.cpr_set_coarse(P, zc, DIMS, TILE)
    e = oracle.cpr_coarse_apply(P, np.random.default_rng(4).standard_normal(A.nb))
    assert np.all(e[zc == 0.0] == 0.0)


def test_amg_stage_adds_the_correction():
    # the pressure stage with a coarse space equals the V-cycle plus Z E^{-1} Z^T f
    A, _ = _system(4, DIMS)
    plain = oracle.cpr_prec(A, DIMS, stage=oracle.STAGE_AMG)
    withc = oracle.cpr_prec(A, DIMS, stage=oracle.STAGE_AMG)
    zc = np.random.default_rng(5).uniform(0.5, 2.0, A.nb)
    oracle.cpr_set_coarse(withc, zc, DIMS, TILE)
    v = np.random.default_rng(6).standard_normal(A.n)
    z0, z1 = plain.apply(v), withc.apply(v)
    corr = oracle.cpr_coarse_apply(withc, v[0::3])
    np.testing.assert_allclose(z1[0::3], z0[0::3] + corr, rtol=1e-11, atol=1e-13)
    assert np.all(z1[1::3] == 0.0) and np.all(z1[2::3] == 0.0)


def test_cpr_gmres_with_coarse_space_converges():
    A, b = _system(5, DIMS)
    P = oracle.cpr_prec(A, DIMS)
    x_ref = np.linalg.solve(A.to_dense(), b)
    oracle.cpr_set_coarse(P, x_ref[0::3], DIMS, TILE)
    x, info = oracle.gmres(A, b, tol=1e-10, prec=P)
    assert info["converged"]
    np.testing.assert_allclose(x, x_ref, rtol=1e-6, atol=1e-8 * np.abs(x_ref).max())
