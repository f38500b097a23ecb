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


# ---- the forcing terms by hand (Sec. 3.1), on one unknown:
# R(x) = x^2 - 4, b(x) = -R(x) = 4 - x^2, A(x) = R'(x) = 2x.  The linear
# "solver" returns dx = c b / A, so its residual r = b - A dx = (1 - c) b is
# known exactly, and one step gives every quantity of the formulas in closed
# form.  theta_max = 1 keeps the values unclipped.
def _scalar_step(x0, c, forcing):
    from oracle.newton import newton

    def assemble(x):
        return np.array([4.0 - x[0] ** 2]), 2.0 * x[0]

    def solve(A, b, theta):
        return c * b / A, 1

    def matvec(A, dx):
        return A * dx

    _, info = newton(np.array([x0]), assemble, solve, matvec, eps=0.0, forcing=forcing, theta_max=1.0,
                     theta_min=1e-12, maxit=2)
    return info


# x0 = 1, c = 0.9: dx = 1.35, x1 = 2.35, b0 = 3, b1 = -1.5225, r0 = 0.3
#   ew1 = |b1 - r0| / |b0| = 1.8225 / 3; ew2 = | |b1| - |r0| | / |b0| = 1.2225 / 3;
#   ew3 = 0.9 (1.5225 / 3)^2
# x0 = 3, c = 1.5: dx = -1.25, x1 = 1.75, b0 = -5, b1 = 0.9375, r0 = 2.5
#   ew1 = 1.5625 / 5; ew2 = |0.9375 - 2.5| / 5 (the absolute value: without
#   it the term would be -0.3125); ew3 = 0.9 (0.9375 / 5)^2
@pytest.mark.parametrize("x0,c,forcing,theta1", [
    (1.0, 0.9, "ew1", 0.6075), (1.0, 0.9, "ew2", 0.4075), (1.0, 0.9, "ew3", 0.231800625),
    (3.0, 1.5, "ew1", 0.3125), (3.0, 1.5, "ew2", 0.3125), (3.0, 1.5, "ew3", 0.031640625),
])
def test_forcing_terms_by_hand_on_one_unknown(x0, c, forcing, theta1):
    info = _scalar_step(x0, c, forcing)
    assert info["thetas"][0] == 1.0  # theta_0 = theta_max
    assert info["thetas"][1] == pytest.approx(theta1, rel=1e-12, abs=0)
    assert info["linear_rel_res"][0] == pytest.approx(abs(1.0 - c), rel=1e-12)


def test_forcing_term_safeguards():
    # a term above theta_max is clipped to it; theta_0 is theta_max
    from oracle.newton import newton

    def assemble(x):
        return np.array([4.0 - x[0] ** 2]), 2.0 * x[0]

    _, info = newton(np.array([1.0]), assemble, lambda A, b, t: (0.9 * b / A, 1), lambda A, d: A * d, eps=0.0,
                     forcing="ew1", theta_max=0.5, maxit=2)
    assert info["thetas"] == [0.5, 0.5]
