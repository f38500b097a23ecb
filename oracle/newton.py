"""The inexact Newton method of the paper (Alg. 1) on the CPU, in FP64.

TEST INFRASTRUCTURE ONLY (part of the oracle): only the tests, the smoke
check and the benchmark's CPU baseline may call it.

Each Newton step assembles the residual b(x) = -R(x) and the Jacobian A(x),
solves A dx = b to the forcing tolerance ||b(x^l) - A dx|| <= theta_l
||b(x^l)|| (Alg. 1), and updates x^{l+1} = x^l + dx until ||b(x^l)|| < eps.
`newton` is the loop itself over any residual and linear solver;
`inexact_newton` runs it on a seeded black-oil case with the input
generator's assembly and the oracle's right-preconditioned GMRES(30) and
CPR.

The forcing terms are the three choices of Sec. 3.1 (Eisenstat and Walker,
SIAM J. Sci. Comput. 17, 1996), computed after each step from the new
residual b(x^{l+1}), the old norm ||b(x^l)|| and the linear residual
r^l = b(x^l) - A dx:

  "ew1"  theta = ||b(x^{l+1}) - r^l|| / ||b(x^l)||
  "ew2"  theta = | ||b(x^{l+1})|| - ||r^l|| | / ||b(x^l)||
  "ew3"  theta = gamma (||b(x^{l+1})|| / ||b(x^l)||)^beta

or a fixed theta (a float).  Sec. 3.1 prints the second choice without the
absolute value; the source it cites defines it with one, and a negative
difference would be no tolerance at all, so the absolute value is taken.
The paper leaves the first step's theta and any safeguard open: here
theta_0 = theta_max, and every theta is clipped to [theta_min, theta_max].
Saturation updates are not chopped: the method is applied as stated, on
states where Newton's step stays physical.
"""
from __future__ import annotations

import numpy as np

from . import BsrMatrix, cpr_prec, gmres, spmv


def forcing_term(kind, b_new, nb_old, r, gamma=0.9, beta=2.0):
    """theta_{l+1} of Sec. 3.1 from b(x^{l+1}), ||b(x^l)|| and r^l (before
    the safeguards)."""
    b_new = np.asarray(b_new, dtype=np.float64)
    r = np.asarray(r, dtype=np.float64)
    if kind == "ew1":
        return float(np.linalg.norm(b_new - r)) / nb_old
    if kind == "ew2":
        return abs(float(np.linalg.norm(b_new)) - float(np.linalg.norm(r))) / nb_old
    if kind == "ew3":
        return gamma * (float(np.linalg.norm(b_new)) / nb_old) ** beta
    raise ValueError(f"unknown forcing term {kind!r}")


def newton(x0, assemble, solve, matvec, eps, forcing="ew3", theta_max=0.1, theta_min=1e-10, gamma=0.9, beta=2.0,
           maxit=20):
    """Alg. 1 over any problem.  assemble(x) -> (b, A) with b = b(x) = -R(x);
    solve(A, b, theta) -> (dx, linear iterations) with ||b - A dx|| <= theta
    ||b||; matvec(A, dx) -> A dx.  Returns (x, info): the final state and
    dict(iters, norms (||b|| per iterate), thetas, linear_iters,
    linear_rel_res = ||b - A dx|| / ||b|| per step, converged)."""
    x = np.array(x0, dtype=np.float64)
    b, A = assemble(x)
    norms = [float(np.linalg.norm(b))]
    thetas, lin, lin_res = [], [], []
    theta = float(forcing) if not isinstance(forcing, str) else theta_max
    while norms[-1] >= eps and len(thetas) < maxit:
        dx, its = solve(A, b, theta)
        r = b - matvec(A, dx)
        x = x + dx
        b_new, A = assemble(x)
        nb_old, nb_new = norms[-1], float(np.linalg.norm(b_new))
        thetas.append(theta)
        lin.append(its)
        lin_res.append(float(np.linalg.norm(r)) / nb_old)
        norms.append(nb_new)
        if isinstance(forcing, str):
            theta = min(max(forcing_term(forcing, b_new, nb_old, r, gamma, beta), theta_min), theta_max)
        b = b_new
    return x, dict(iters=len(thetas), norms=norms, thetas=thetas, linear_iters=lin, linear_rel_res=lin_res,
                   converged=norms[-1] < eps)


def inexact_newton(case, eps, forcing="ew3", theta_max=0.1, theta_min=1e-10, gamma=0.9, beta=2.0, maxit=20,
                   restart=30):
    """Alg. 1 on a seeded black-oil case (a bogen case: grid, rock, wells,
    previous state and the initial state case.x): the generator's residual
    and Jacobian, the oracle's GMRES(restart) with CPR (red-black ILU(0) and
    AMG) for each linear system.  Returns newton's (x, info)."""
    import bogen
    dims = (case.nx, case.ny, case.nz)

    def assemble(x):
        a = bogen.assemble(case, x=x)
        return a["b"], BsrMatrix(a["rowptr"], a["col"], a["val"])

    def solve(A, b, theta):
        dx, info = gmres(A, b, m=restart, maxit=5000, tol=theta, prec=cpr_prec(A, dims))
        return dx, info["iters"]

    return newton(case.x, assemble, solve, spmv, eps, forcing=forcing, theta_max=theta_max, theta_min=theta_min,
                  gamma=gamma, beta=beta, maxit=maxit)


def inexact_newton_wells(case, eps, forcing="ew3", theta_max=0.1, theta_min=1e-10, gamma=0.9, beta=2.0, maxit=20,
                         restart=30):
    """Alg. 1 on a case with rate-controlled wells (paper Sec. 2.3): the
    Newton unknowns are the cell states and the controlled wells' bottom-hole
    pressures, x = (cells (3N), p_h (W)); each step assembles the bordered
    system of Sec. 3.2 with the generator and solves it with the oracle's
    bordered GMRES (natural block ILU(0) of the whole bordered matrix).
    Returns newton's (x, info)."""
    import bogen
    from .bordered import bordered_bsr, bordered_matvec, bordered_solve
    N = case.N
    ph0 = np.array([w.bhp for w in bogen.rate_wells(case)], dtype=np.float64)
    W = ph0.size

    class Bordered:
        def __init__(self, A, border):
            self.A, self.border = A, border

    def assemble(x):
        a = bogen.assemble(case, x=x[:3 * N], ph=x[3 * N:])
        return a["b_full"], Bordered(BsrMatrix(a["rowptr"], a["col"], a["val"]), a["border"])

    def solve(Ab, b, theta):
        dx, info = bordered_solve(Ab.A, Ab.border, b, tol=theta, m=restart, maxit=20000)
        return dx, info["iters"]

    def matvec(Ab, dx):
        return bordered_matvec(Ab.A, Ab.border, dx)

    x0 = np.concatenate([np.asarray(case.x, np.float64), ph0])
    assert x0.size == 3 * N + W
    return newton(x0, assemble, solve, matvec, eps, forcing=forcing, theta_max=theta_max, theta_min=theta_min,
                  gamma=gamma, beta=beta, maxit=maxit)
