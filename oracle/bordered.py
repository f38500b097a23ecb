"""The bordered Newton system of rate-controlled wells, on the CPU in FP64.

TEST INFRASTRUCTURE ONLY (part of the oracle): only the tests, the smoke
check and the benchmark's CPU baseline may call it.

A well under a fixed rate (paper Sec. 2.3) has its bottom-hole pressure p_h
as an unknown and one constraint equation, so the Newton system takes the
block form of Sec. 3.2 with the well rows and columns last:

    [ A     A_pw ] [dx  ]   [b  ]
    [ A_wp  A_ww ] [dp_h] = [b_w]

A_pw holds, in the rows of each perforated cell, the derivative of that
cell's three equations with respect to its well's p_h; A_wp the derivative
of each well's constraint with respect to the unknowns of its perforated
cells; A_ww (diagonal: a constraint involves only its own well's p_h) the
derivative with respect to p_h.  The border arrives per perforation e:
perf_cell[e], perf_well[e], apw[e, 0:3] (the column entries of rows 3c..3c+2),
awp[e, 0:3] (the row entries of columns 3c..3c+2), and aww[w].

Here the system is solved as written, the way the paper's solver treats it:
the well unknowns become extra block rows of the BSR matrix (a well's block
row holds p_h in its first slot and two identity slots with zero right-hand
side, which stay zero), and restarted GMRES with natural-order block ILU(0)
of the whole bordered matrix solves it.  Nothing of the device solver's
elimination of the wells is used.
"""
from __future__ import annotations

import numpy as np

from . import BsrMatrix, gmres, ilu0_prec, spmv


def bordered_bsr(A: BsrMatrix, border) -> BsrMatrix:
    """The bordered matrix as a BSR matrix of N + W block rows (3x3 blocks):
    block row N + w is well w, its unknown p_h in slot 0."""
    N = A.nb
    pc = np.asarray(border["perf_cell"], np.int64)
    pw = np.asarray(border["perf_well"], np.int64)
    apw = np.asarray(border["apw"], np.float64).reshape(-1, 3)
    awp = np.asarray(border["awp"], np.float64).reshape(-1, 3)
    aww = np.asarray(border["aww"], np.float64).ravel()
    W = aww.size
    well_of_cell = {}
    for e in range(pc.size):
        well_of_cell.setdefault(int(pc[e]), []).append(e)
    rows_col, rows_val = [], []
    # cell rows: the reservoir blocks, then (perforated cells) the well column
    for i in range(N):
        cols = list(A.col[A.rowptr[i]:A.rowptr[i + 1]])
        vals = [A.val[e] for e in range(A.rowptr[i], A.rowptr[i + 1])]
        for e in well_of_cell.get(i, []):
            blk = np.zeros((3, 3))
            blk[:, 0] = apw[e]                # d(cell equations)/d p_h
            cols.append(N + int(pw[e]))
            vals.append(blk)
        rows_col.append(cols)
        rows_val.append(vals)
    # well rows: the perforated cells' columns, then the diagonal block
    for w in range(W):
        cols, vals = [], []
        for e in sorted(np.nonzero(pw == w)[0], key=lambda e: pc[e]):
            blk = np.zeros((3, 3))
            blk[0, :] = awp[e]                # d(constraint)/d(cell unknowns)
            cols.append(int(pc[e]))
            vals.append(blk)
        cols.append(N + w)
        vals.append(np.diag([aww[w], 1.0, 1.0]))
        rows_col.append(cols)
        rows_val.append(vals)
    rowptr = np.zeros(N + W + 1, np.int64)
    for i, c in enumerate(rows_col):
        rowptr[i + 1] = rowptr[i] + len(c)
    col = np.concatenate([np.asarray(c, np.int64) for c in rows_col])
    val = np.concatenate([np.asarray(v).reshape(-1, 3, 3) for v in rows_val])
    return BsrMatrix(rowptr.astype(np.int32), col.astype(np.int32), val)


def embed(v, N, W):
    """(3N + W) vector -> the bordered BSR's 3(N + W) layout (p_h in slot 0)."""
    v = np.asarray(v, np.float64)
    out = np.zeros(3 * (N + W))
    out[:3 * N] = v[:3 * N]
    out[3 * N::3] = v[3 * N:]
    return out


def extract(u, N, W):
    """The bordered BSR's 3(N + W) layout -> (3N + W)."""
    u = np.asarray(u, np.float64)
    return np.concatenate([u[:3 * N], u[3 * N::3][:W]])


def bordered_matvec(A: BsrMatrix, border, x) -> np.ndarray:
    """(A x + A_pw x_w, A_wp x + A_ww x_w) for x = (cells, wells): the BSR
    product of the cell rows, then one pass over the perforations."""
    N = A.nb
    aww = np.asarray(border["aww"], np.float64).ravel()
    W = aww.size
    x = np.asarray(x, np.float64)
    xw = x[3 * N:]
    y = np.concatenate([spmv(A, x[:3 * N]), aww * xw])
    for e in range(np.asarray(border["perf_cell"]).size):
        c, w = int(border["perf_cell"][e]), int(border["perf_well"][e])
        for r in range(3):
            y[3 * c + r] += border["apw"][e][r] * xw[w]
            y[3 * N + w] += border["awp"][e][r] * x[3 * c + r]
    return y


def bordered_solve(A: BsrMatrix, border, b_full, tol=1e-13, m=30, maxit=20000, x0=None, B=None):
    """x with ||b_full - A_b x|| <= tol ||b_full||: GMRES(m) with natural
    block ILU(0) of the bordered BSR matrix.  Returns (x (3N + W), info)."""
    N, W = A.nb, np.asarray(border["aww"]).size
    B = bordered_bsr(A, border) if B is None else B
    u, info = gmres(B, embed(b_full, N, W), x0=None if x0 is None else embed(x0, N, W), m=m, maxit=maxit, tol=tol,
                    prec=ilu0_prec(B))
    return extract(u, N, W), info
