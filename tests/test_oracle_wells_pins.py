"""Pins of the rate-controlled well border (paper Sec. 2.3 controls, the
bordered block form of Sec. 3.2) in the generator and of the oracle's
bordered solve, against what fixes the answer independently of that code:

  * the border is the exact derivative of the full residual (cells and well
    constraints) with respect to (cell unknowns, p_h): central differences;
  * the oracle's bordered BSR matrix, read back as a dense matrix, is that
    whole Jacobian (the well column in the cell rows, the well row in the
    well's own row, A_ww on its diagonal);
  * its GMRES + ILU(0) solution equals a dense LU solution (brute force);
  * Newton on the bordered system converges quadratically, and at the
    converged state each well's rate, measured as the change of the cell
    residuals when the well is removed (a path that never calls the border
    code), equals its target."""
import copy

import numpy as np
import pytest

import bogen
import oracle
from bogen import CTRL_LIQUID, CTRL_OIL, CTRL_WATER, Well
from oracle.bordered import bordered_bsr, bordered_matvec, bordered_solve, embed, extract
from oracle.newton import inexact_newton_wells


def _case(nx=4, ny=4, nz=3, seed=5, producer_control=CTRL_LIQUID):
    c = bogen.tiny_case(seed, nx, ny, nz)
    # a third well (a second producer, oil-rate controlled) in a middle column
    mid = np.array([nx // 2 + nx * (ny // 2 + ny * k) for k in range(nz)], np.int32)
    c.wells.append(Well(1, 2700.0, mid))
    c = bogen.with_rate_controls(c, fraction=0.8, producer_control=producer_control)
    c.wells[2].control = CTRL_OIL
    a = bogen.assemble(c, jacobian=False)
    c.wells[2].rate = 0.8 * (a["border"]["Rw"][2] + c.wells[2].rate)
    return c


def _full_residual(c, x, ph):
    a = bogen.assemble(c, jacobian=False, x=x, ph=ph)
    return np.concatenate([a["R"], a["border"]["Rw"]])


def _dense_bordered(a):
    """The bordered BSR matrix read back as a dense (3N + W) matrix."""
    N, W = a["rowptr"].size - 1, a["border"]["aww"].size
    B = bordered_bsr(oracle.BsrMatrix(a["rowptr"], a["col"], a["val"]), a["border"]).to_dense()
    keep = np.concatenate([np.arange(3 * N), 3 * N + 3 * np.arange(W)])
    return B[np.ix_(keep, keep)], B


def test_border_matches_central_differences():
    c = _case()
    a = bogen.assemble(c)
    bd = a["border"]
    N = c.N
    ph = np.array([w.bhp for w in bogen.rate_wells(c)])
    for v in range(ph.size):
        h = 1e-4
        pp, pm = ph.copy(), ph.copy()
        pp[v] += h
        pm[v] -= h
        d = (_full_residual(c, c.x, pp) - _full_residual(c, c.x, pm)) / (2 * h)
        # cell rows: -dQ/dp_h at this well's perforations, zero elsewhere
        col = np.zeros(3 * N)
        for e in np.nonzero(bd["perf_well"] == v)[0]:
            col[3 * bd["perf_cell"][e]:3 * bd["perf_cell"][e] + 3] = bd["apw"][e]
        assert np.abs(d[:3 * N] - col).max() <= 1e-6 * np.abs(col).max()
        # well rows: A_ww on the diagonal only
        want = np.zeros(ph.size)
        want[v] = bd["aww"][v]
        assert np.abs(d[3 * N:] - want).max() <= 1e-6 * abs(bd["aww"][v])
    for e in range(bd["perf_cell"].size):
        cell = bd["perf_cell"][e]
        for u in range(3):
            h = 1e-6 * max(abs(c.x[3 * cell + u]), 1e-3)
            xp, xm = c.x.copy(), c.x.copy()
            xp[3 * cell + u] += h
            xm[3 * cell + u] -= h
            dw = (_full_residual(c, xp, ph)[3 * N:] - _full_residual(c, xm, ph)[3 * N:]) / (2 * h)
            want = np.zeros(ph.size)
            want[bd["perf_well"][e]] = bd["awp"][e, u]
            assert np.abs(dw - want).max() <= 1e-5 * max(abs(bd["awp"][e, u]), 1e-3 * np.abs(bd["awp"]).max())


def test_bordered_matrix_is_the_jacobian_of_the_full_residual():
    c = _case(4, 3, 2)
    a = bogen.assemble(c)
    D, _ = _dense_bordered(a)
    N = c.N
    ph = np.array([w.bhp for w in bogen.rate_wells(c)])
    z = np.concatenate([c.x, ph])
    n = z.size
    J = np.zeros((n, n))
    for u in range(n):
        h = 1e-6 * max(abs(z[u]), 1e-3)
        zp, zm = z.copy(), z.copy()
        zp[u] += h
        zm[u] -= h
        J[:, u] = (_full_residual(c, zp[:3 * N], zp[3 * N:]) - _full_residual(c, zm[:3 * N], zm[3 * N:])) / (2 * h)
    for u in range(n):
        scale = max(np.abs(D[:, u]).max(), 1e-12)
        assert np.abs(J[:, u] - D[:, u]).max() <= 1e-5 * scale, u


def test_bordered_solve_matches_dense_lu():
    c = _case(6, 5, 3)
    a = bogen.assemble(c)
    A = oracle.BsrMatrix(a["rowptr"], a["col"], a["val"])
    x, info = bordered_solve(A, a["border"], a["b_full"], tol=1e-13)
    assert info["converged"]
    D, _ = _dense_bordered(a)
    xd = np.linalg.solve(D, a["b_full"])
    assert np.linalg.norm(x - xd) <= 1e-10 * np.linalg.norm(xd)
    # the matrix-free product agrees with the dense matrix
    y = bordered_matvec(A, a["border"], xd)
    assert np.linalg.norm(y - D @ xd) <= 1e-13 * np.linalg.norm(D @ xd)
    # embed / extract are inverse on the (3N + W) layout
    N, W = c.N, a["border"]["aww"].size
    assert np.array_equal(extract(embed(xd, N, W), N, W), xd)


def _well_rates(c, x, ph):
    """Each rate-controlled well's component rates (oil, water, gas) summed
    over its perforations, as the change of the cell residuals when that
    well alone is removed (R = ... - Q)."""
    rates = []
    wells_ph = copy.deepcopy(c)
    v = 0
    for w in wells_ph.wells:
        if w.control:
            w.bhp = float(ph[v])
            v += 1
        w.control = 0
    R_all = bogen.assemble(wells_ph, jacobian=False, x=x)["R"]
    for i, w in enumerate(wells_ph.wells):
        if not c.wells[i].control:
            continue
        other = copy.deepcopy(wells_ph)
        other.wells.pop(i)
        R_wo = bogen.assemble(other, jacobian=False, x=x)["R"]
        q = (R_wo - R_all).reshape(-1, 3)[np.asarray(w.cells)].sum(axis=0)
        rates.append(q)
    return np.array(rates)


@pytest.mark.parametrize("producer_control", [CTRL_LIQUID, CTRL_OIL])
def test_newton_meets_the_rate_targets(producer_control):
    c = _case(8, 6, 3, seed=2, producer_control=producer_control)
    b0 = np.linalg.norm(bogen.assemble(c)["b_full"])
    x, info = inexact_newton_wells(c, eps=1e-10 * b0, forcing=1e-12, maxit=20)
    assert info["converged"]
    nb = info["norms"]
    # quadratic: once below 1e-2 of the start, each norm is at most a
    # modest multiple of the square of the previous (relative to the start)
    rel = [v / nb[0] for v in nb]
    for r0, r1 in zip(rel, rel[1:]):
        if r0 < 1e-2:
            assert r1 <= 1e3 * r0 * r0 + 1e-12
    N = c.N
    q = _well_rates(c, x[:3 * N], x[3 * N:])
    for (qo, qw, qg), w in zip(q, bogen.rate_wells(c)):
        got = {CTRL_WATER: qw, CTRL_OIL: qo, CTRL_LIQUID: qo + qw}[w.control]
        assert got == pytest.approx(w.rate, rel=1e-7, abs=1e-6)
