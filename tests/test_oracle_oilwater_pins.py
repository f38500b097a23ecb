"""Pins of the two-phase oil-water inputs (paper Sec. 2.2) and of the
oracle's ABF decoupling (paper Sec. 3.2, Alternate Block Factorization),
against what fixes them independently of the code:

  * the 2x2 Jacobian is the exact derivative of the two-phase residual
    (central differences);
  * each component's residuals sum to its accumulation change minus the
    well rates (mass balance; the fluxes cancel pairwise);
  * a single producing cell's oil and water rates follow the paper's SPE10
    relative permeabilities in closed form;
  * ABF: D^{-1} A has identity diagonal blocks and (D^{-1} A) x = D^{-1} (A x)
    with D^{-1} applied block by block by a dense solve;
  * the block-size-2 GMRES + ILU(0) and the padded-CPR reference solutions
    equal a dense LU solution (brute force)."""
import numpy as np
import pytest

import bogen
import oracle
from bogen import Well


def test_two_phase_jacobian_matches_central_differences():
    c = bogen.tiny_oil_water_case(3, 4, 3, 3)
    a = bogen.assemble_ow(c)
    A = oracle.BsrMatrix(a["rowptr"], a["col"], a["val"]).to_dense()
    x = bogen.state_ow(c)
    n = x.size
    for u in range(n):
        h = 1e-6 * max(abs(x[u]), 1e-3)
        xp, xm = x.copy(), x.copy()
        xp[u] += h
        xm[u] -= h
        d = (bogen.assemble_ow(c, jacobian=False, x=xp)["R"] - bogen.assemble_ow(c, jacobian=False, x=xm)["R"]) / (2 * h)
        assert np.abs(d - A[:, u]).max() <= 1e-5 * max(np.abs(A[:, u]).max(), 1e-12)


def test_two_phase_mass_balance():
    c = bogen.tiny_oil_water_case(1, 6, 5, 3)
    R = bogen.assemble_ow(c, jacobian=False)["R"].reshape(-1, 2)
    # the same state without wells: the residual sums are the accumulation change
    c0 = bogen.tiny_oil_water_case(1, 6, 5, 3)
    c0.wells = []
    R0 = bogen.assemble_ow(c0, jacobian=False)["R"].reshape(-1, 2)
    V = c.dx * c.dy * c.dz
    acc = np.zeros(2)
    for i in range(c.N):
        for comp in range(2):
            m = bogen.cell_mass(c.fluid, c.phi0[i], c.x[3 * i], c.x[3 * i + 1], 0.0, comp)
            mn = bogen.cell_mass(c.fluid, c.phi0[i], c.xn[3 * i], c.xn[3 * i + 1], 0.0, comp)
            acc[comp] += V / (5.615 * c.dt) * (m - mn)
    assert np.allclose(R0.sum(axis=0), acc, rtol=1e-10, atol=1e-9 * np.abs(acc).max())
    # with wells the sums drop by exactly the well rates (perforated rows only)
    assert np.abs(R - R0)[np.setdiff1d(np.arange(c.N), np.concatenate([w.cells for w in c.wells]))].max() == 0.0


@pytest.mark.parametrize("sw", [0.25, 0.5, 0.75])
def test_spe10_relative_permeabilities_in_producer_rates(sw):
    fl = bogen.oil_water_fluid()
    c = bogen.uniform_case(2, 1, 1, p=3000.0, sw=sw, sg=0.0, fluid=fl,
                           wells=[Well(1, 2500.0, np.array([0], np.int32))])
    R = bogen.assemble_ow(c, jacobian=False)["R"].reshape(-1, 2)
    wi = bogen.well_index(c, 0)
    krw = ((sw - 0.2) / 0.6) ** 2
    kro = ((0.8 - sw) / 0.6) ** 2
    q = wi * (2500.0 - 3000.0) * np.array([kro / (fl.muo * fl.bo0), krw / (fl.muw * fl.bw0)])
    # uniform state, no flow between the cells: the perforated cell's residual is -q
    assert np.allclose(R[0], -q, rtol=1e-12, atol=0)
    assert np.all(R[1] == 0.0)


@pytest.mark.parametrize("bs_case", ["three_phase", "two_phase"])
def test_abf_decoupling_identities(bs_case):
    if bs_case == "three_phase":
        c = bogen.tiny_case(2, 6, 4, 3)
        a = bogen.assemble(c)
    else:
        c = bogen.tiny_oil_water_case(2, 6, 4, 3)
        a = bogen.assemble_ow(c)
    A = oracle.BsrMatrix(a["rowptr"], a["col"], a["val"])
    B = oracle.abf_decouple(A)
    for i in range(A.nb):
        for e in range(A.rowptr[i], A.rowptr[i + 1]):
            if A.col[e] == i:
                assert np.abs(B.val[e] - np.eye(A.bs)).max() <= 1e-12
    rng = np.random.default_rng(0)
    x = rng.standard_normal(A.n)
    Ax = oracle.spmv(A, x)
    want = np.concatenate([np.linalg.solve(A.val[[e for e in range(A.rowptr[i], A.rowptr[i + 1]) if A.col[e] == i][0]],
                                           Ax[A.bs * i:A.bs * (i + 1)]) for i in range(A.nb)])
    got = oracle.spmv(B, x)
    assert np.abs(got - want).max() <= 1e-10 * np.abs(want).max()
    assert np.abs(oracle.abf_scale(A, Ax) - want).max() <= 1e-12 * np.abs(want).max()


def test_two_phase_reference_solutions_match_dense_lu():
    c = bogen.tiny_oil_water_case(0, 10, 8, 3)
    a = bogen.assemble_ow(c)
    A = oracle.BsrMatrix(a["rowptr"], a["col"], a["val"])
    xd = np.linalg.solve(A.to_dense(), a["b"])
    x, info = oracle.solve_two_phase(A, a["b"], (c.nx, c.ny, c.nz), tol=1e-13)
    assert info["converged"]
    assert np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd)
