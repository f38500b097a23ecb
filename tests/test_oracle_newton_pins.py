"""Pins of the oracle's inexact Newton method (Alg. 1 with the forcing terms
of Sec. 3.1) on a seeded black-oil step: Newton's quadratic convergence when
the linear systems are solved exactly, the Alg. 1 condition
||b(x^l) - A dx|| <= theta_l ||b(x^l)|| at every step, the same solution
reached with every forcing term, and fewer linear iterations in total with
the forcing terms than with exact solves (the purpose of the method)."""
import numpy as np
import pytest

import bogen
from oracle.newton import inexact_newton


@pytest.fixture(scope="module")
def case():
    return bogen.tiny_case(0, 10, 10, 4)


@pytest.fixture(scope="module")
def exact(case):
    b0 = float(np.linalg.norm(bogen.assemble(case)["b"]))
    x, info = inexact_newton(case, eps=1e-8 * b0, forcing=1e-12, maxit=30)
    return b0, x, info


def test_exact_newton_converges_quadratically(exact):
    b0, x, info = exact
    n = info["norms"]
    assert info["converged"] and n[-1] < 1e-8 * b0
    # ||b_{l+1}|| / ||b_l||^2 settles to a constant over the last steps
    c = [n[l + 1] / n[l] ** 2 for l in range(len(n) - 3, len(n) - 1)]
    assert all(0 < v < 1e-2 for v in c) and max(c) / min(c) < 10.0, (n, c)


@pytest.mark.parametrize("forcing", ["ew1", "ew2", "ew3", 1e-2])
def test_forcing_terms_reach_the_same_solution_with_fewer_linear_iterations(case, exact, forcing):
    b0, x_ex, info_ex = exact
    x, info = inexact_newton(case, eps=1e-8 * b0, forcing=forcing, maxit=30)
    assert info["converged"]
    # Alg. 1's condition at every step, theta within the safeguards
    for th, rr in zip(info["thetas"], info["linear_rel_res"]):
        assert 1e-10 <= th <= 0.1 and rr <= th * (1 + 1e-12)
    # the nonlinear solution is unique: both end within the nonlinear tolerance
    assert np.linalg.norm(x - x_ex) <= 1e-6 * np.linalg.norm(x_ex)
    assert sum(info["linear_iters"]) < sum(info_ex["linear_iters"])


def test_converged_state_is_physical(exact):
    _, x, _ = exact
    sw, sg = x[1::3], x[2::3]
    assert np.all(sg > 0) and np.all(sw > 0) and np.all(sw + sg < 1)
