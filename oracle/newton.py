"""The inexact Newton method of the paper (Alg. 1) on the CPU, in FP64.

TEST INFRASTRUCTURE ONLY (part of the oracle): only the tests, the smoke
check and the benchmark's CPU baseline may call it.

Each Newton step assembles the residual b(x) = -R(x) and the Jacobian A(x)
with the seeded input generator, solves A dx = b with the oracle's
right-preconditioned GMRES(30) and CPR to the forcing tolerance
||b(x^l) - A dx|| <= theta_l ||b(x^l)|| (Alg. 1), and updates x^{l+1} =
x^l + dx until ||b(x^l)|| < eps.  The forcing terms are the three choices of
Sec. 3.1 (Eisenstat and Walker's, SIAM J. Sci. Comput. 17, 1996), computed
after each step from the new residual b(x^{l+1}), the old one b(x^l) and the
linear residual r^l = b(x^l) - A dx:

  "ew1"  theta = ||b(x^{l+1}) - r^l|| / ||b(x^l)||
  "ew2"  theta = | ||b(x^{l+1})|| - ||r^l|| | / ||b(x^l)||
  "ew3"  theta = gamma (||b(x^{l+1})|| / ||b(x^l)||)^beta

or a fixed theta (a float).  The paper leaves the first step's theta and any
safeguard open: here theta_0 = theta_max, and every theta is clipped to
[theta_min, theta_max].  Saturation updates are not chopped: the method is
applied as stated, on states where Newton's step stays physical.
"""
from __future__ import annotations

import numpy as np

from . import BsrMatrix, cpr_prec, gmres, spmv


def inexact_newton(case, eps, forcing="ew3", theta_max=0.1, theta_min=1e-10, gamma=0.9, beta=2.0, maxit=20,
                   restart=30):
    """Returns (x, info): the final state and dict(iters, norms (||b|| per
    iterate), thetas, linear_iters and linear_rel_res = ||b - A dx|| / ||b||
    (per step), converged)."""
    import bogen
    dims = (case.nx, case.ny, case.nz)
    x = np.array(case.x, dtype=np.float64)
    asm = bogen.assemble(case, x=x)
    b = asm["b"]
    norms = [float(np.linalg.norm(b))]
    thetas, lin, lin_res = [], [], []
    theta = float(forcing) if not isinstance(forcing, str) else theta_max
    while norms[-1] >= eps and len(thetas) < maxit:
        A = BsrMatrix(asm["rowptr"], asm["col"], asm["val"])
        dx, info = gmres(A, b, m=restart, maxit=5000, tol=theta, prec=cpr_prec(A, dims))
        r = b - spmv(A, dx)
        x = x + dx
        asm = bogen.assemble(case, x=x)
        b_new = asm["b"]
        nb_old, nb_new = norms[-1], float(np.linalg.norm(b_new))
        thetas.append(theta)
        lin.append(info["iters"])
        lin_res.append(float(np.linalg.norm(r)) / norms[-1])
        norms.append(nb_new)
        if isinstance(forcing, str):
            if forcing == "ew1":
                theta = float(np.linalg.norm(b_new - r)) / nb_old
            elif forcing == "ew2":
                theta = abs(nb_new - float(np.linalg.norm(r))) / nb_old
            elif forcing == "ew3":
                theta = gamma * (nb_new / nb_old) ** beta
            else:
                raise ValueError(f"unknown forcing term {forcing!r}")
            theta = min(max(theta, theta_min), theta_max)
        b = b_new
    return x, dict(iters=len(thetas), norms=norms, thetas=thetas, linear_iters=lin, linear_rel_res=lin_res,
                   converged=norms[-1] < eps)
