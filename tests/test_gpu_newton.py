"""The black-oil residual and Jacobian assembled on the GPU, and the inexact
Newton method (Alg. 1 with the forcing terms of Sec. 3.1) run on the device,
against the CPU references: the seeded generator's assembly (bogen, the same
equations in plain FP64 loops) and the oracle's Newton loop
(oracle.newton.inexact_newton, GMRES + CPR in FP64).

Tolerances (derived from the arithmetic):
  * Jacobian entries: each is a sum of at most eight FP64 contributions
    (accumulation, six faces, wells) added in a different order on the two
    sides, so |A_gpu - A_cpu| <= 1e-12 of the largest entry of the block row.
  * Residual: b = -R sums the same terms with cancellation between the
    accumulation, the fluxes and the wells; 1e-11 of max |b|.
  * Newton with near-exact linear solves (theta = 1e-10): both sides take
    the same steps to linear-solve accuracy, so the residual norms agree to
    1e-6 relative at every step and the final states to 1e-9.
  * Forcing terms: the linear solvers differ (FGMRES + red-black CPR against
    GMRES + CPR), so the inexact iterates differ; the nonlinear solution is
    unique, and both end within 1e-6 of it."""
import numpy as np
import pytest

import bogen
import oracle
from oracle.newton import inexact_newton

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def bo():
    import paper_1606_00556_gb300 as m
    m.build()
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    return m


@pytest.fixture(scope="module")
def ctx(bo):
    return bo.Context(0)


def _model(bo, ctx, case):
    """The device model of a generator case: the same rock, wells (with the
    generator's Peaceman indices and reference depths) and fluid."""
    m = bogen.model_inputs(case)
    g = bo.grid(case.nx, case.ny, case.nz, case.dx, case.dy, case.dz)
    return bo.Model(ctx, g, bo.fluid(**m["fluid"]), m["kx"], m["ky"], m["kz"], m["phi0"], m["depth"],
                    m["perf_cell"], m["perf_type"], m["perf_bhp"], m["perf_dref"], m["perf_wi"])


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _assemble(bo, M, case, x):
    b = torch.zeros(M.n, dtype=torch.float64, device="cuda")
    val = torch.zeros(9 * M.nnzb, dtype=torch.float64, device="cuda")
    nb = M.assemble(_dev(x), _dev(case.xn), case.dt, b, val)
    return b.cpu().numpy(), val.cpu().numpy().reshape(-1, 3, 3), nb


def _compare(case, x, b, val, nb):
    a = bogen.assemble(case, x=x)
    rp = a["rowptr"]
    assert np.all(np.abs(b - a["b"]) <= 1e-11 * np.abs(a["b"]).max())
    assert nb == pytest.approx(np.linalg.norm(a["b"]), rel=1e-12)
    # per block row: every entry within 1e-12 of the row's largest entry
    rowmax = np.maximum.reduceat(np.abs(a["val"]).reshape(a["val"].shape[0], -1).max(axis=1), rp[:-1])
    bound = 1e-12 * np.repeat(rowmax, np.diff(rp))[:, None, None]
    assert np.all(np.abs(val - a["val"]) <= bound), np.abs(val - a["val"]).max()


CASES = {
    "tiny0": lambda: bogen.tiny_case(0),
    "tiny1": lambda: bogen.tiny_case(1),
    "tiny2_10x10x4": lambda: bogen.tiny_case(2, 10, 10, 4),
    "waterflood_32x24x8": lambda: bogen.waterflood_case(32, 24, 8, seed=5, day=2, corr=(4, 4, 1)),
    "flooded_12x12x4": lambda: bogen.waterflood_case(12, 12, 4, seed=3, day=0, corr=(2, 2, 1), front0=4.0),
}


@pytest.mark.parametrize("name", list(CASES))
def test_assembly_matches_generator_elementwise(bo, ctx, name):
    case = CASES[name]()
    M = _model(bo, ctx, case)
    b, val, nb = _assemble(bo, M, case, case.x)
    _compare(case, case.x, b, val, nb)
    # and at a second state: the pressure and saturations moved by a seeded
    # perturbation (upwind directions change with the potentials)
    rng = np.random.default_rng(7)
    x2 = np.array(case.x, dtype=np.float64)
    x2[0::3] += rng.uniform(-30, 30, case.N)
    x2[1::3] = np.clip(x2[1::3] + rng.uniform(-0.02, 0.02, case.N), 0.11, 0.85)
    x2[2::3] = np.clip(x2[2::3] + rng.uniform(-0.01, 0.01, case.N), 1e-4, 0.2)
    b2, val2, nb2 = _assemble(bo, M, case, x2)
    _compare(case, x2, b2, val2, nb2)
    M.close()


def test_assembly_without_gravity_and_with_general_corey_exponents(bo, ctx):
    case = bogen.tiny_case(3, 8, 6, 4)
    case.fluid = bogen.default_fluid(gravity=0.0, nw=3.0, now=1.5, ng=2.5, nog=2.0)
    M = _model(bo, ctx, case)
    b, val, nb = _assemble(bo, M, case, case.x)
    _compare(case, case.x, b, val, nb)


def test_assembly_of_an_unphysical_state_is_breakdown(bo, ctx):
    case = bogen.tiny_case(0, 4, 4, 2)
    M = _model(bo, ctx, case)
    x = np.array(case.x, dtype=np.float64)
    x[0] = -1e5  # Bo < 0 in cell 0
    with pytest.raises(bo.BoError) as e:
        M.assemble(_dev(x), _dev(case.xn), case.dt)
    assert e.value.status == bo.BO_ERR_BREAKDOWN


def test_assembly_1m_cells_matches_generator(bo, ctx):
    # the benchmark's grid: 128 x 128 x 64, every Jacobian entry
    case = bogen.waterflood_case(128, 128, 64, seed=42, day=0)
    M = _model(bo, ctx, case)
    b, val, nb = _assemble(bo, M, case, case.x)
    _compare(case, case.x, b, val, nb)
    M.close()


def _newton_setup(bo, ctx, case):
    M = _model(bo, ctx, case)
    a = bogen.assemble(case)
    A = bo.Matrix.from_bsr(ctx, bo.grid(case.nx, case.ny, case.nz, case.dx, case.dy, case.dz), a["rowptr"],
                           a["col"], a["val"])
    P = bo.Preconditioner(A)
    return M, A, P, float(np.linalg.norm(a["b"]))


@pytest.fixture(scope="module")
def newton_case():
    return bogen.tiny_case(0, 10, 10, 4)


@pytest.fixture(scope="module")
def oracle_exact(newton_case):
    b0 = float(np.linalg.norm(bogen.assemble(newton_case)["b"]))
    x, info = inexact_newton(newton_case, eps=1e-8 * b0, forcing=1e-10, maxit=30)
    assert info["converged"]
    return b0, x, info


def test_newton_with_exact_solves_follows_the_oracle(bo, ctx, newton_case, oracle_exact):
    b0, xo, io = oracle_exact
    M, A, P, nb0 = _newton_setup(bo, ctx, newton_case)
    x = _dev(newton_case.x)
    info = M.newton(P, x, _dev(newton_case.xn), newton_case.dt, forcing=1e-10, eps=1e-8 * b0, maxit=30)
    assert info["status"] == bo.BO_OK and info["converged"]
    assert info["iters"] == io["iters"]
    assert info["norms"][0] == pytest.approx(nb0, rel=1e-12)
    for ng, no in zip(info["norms"][:-1], io["norms"][:-1]):
        assert ng == pytest.approx(no, rel=1e-6)
    assert info["norms"][-1] < 1e-8 * b0
    xg = x.cpu().numpy()
    assert np.linalg.norm(xg - xo) <= 1e-9 * np.linalg.norm(xo)
    for th, rr in zip(info["thetas"], info["linear_rel_res"]):
        assert th == 1e-10 and rr <= th * (1 + 1e-9)


@pytest.mark.parametrize("forcing", ["ew1", "ew2", "ew3", 1e-2])
def test_newton_forcing_terms_reach_the_oracle_solution(bo, ctx, newton_case, oracle_exact, forcing):
    b0, xo, io = oracle_exact
    M, A, P, _ = _newton_setup(bo, ctx, newton_case)
    x = _dev(newton_case.x)
    info = M.newton(P, x, _dev(newton_case.xn), newton_case.dt, forcing=forcing, eps=1e-8 * b0, maxit=30)
    assert info["status"] == bo.BO_OK and info["converged"]
    # Alg. 1's condition at every step, theta within the safeguards
    for th, rr in zip(info["thetas"], info["linear_rel_res"]):
        assert 1e-10 <= th <= 0.1 and rr <= th * (1 + 1e-9)
    assert info["thetas"][0] == (0.1 if isinstance(forcing, str) else forcing)
    # the forcing formulas, recomputed from the reported norms where they suffice
    nbs, ths, lrr = info["norms"], info["thetas"], info["linear_rel_res"]
    for l in range(len(ths) - 1):
        if forcing == "ew3":
            want = 0.9 * (nbs[l + 1] / nbs[l]) ** 2
        elif forcing == "ew2":
            want = abs(nbs[l + 1] - lrr[l] * nbs[l]) / nbs[l]
        else:
            continue
        assert ths[l + 1] == pytest.approx(min(max(want, 1e-10), 0.1), rel=1e-9)
    # the same nonlinear solution as the oracle's exact Newton method, with
    # fewer linear iterations than near-exact solves
    xg = x.cpu().numpy()
    assert np.linalg.norm(xg - xo) <= 1e-6 * np.linalg.norm(xo)
    assert info["lin_total"] < sum(io["linear_iters"])


def test_newton_step_at_1m_cells(bo, ctx):
    # one 1-day step of the benchmark's waterflood on the device: converges
    # with the third forcing term, and the final state's residual, assembled
    # by the generator on the CPU, is below the nonlinear tolerance
    case = bogen.waterflood_case(128, 128, 64, seed=42, day=0)
    M, A, P, nb0 = _newton_setup(bo, ctx, case)
    P.close()
    P = bo.Preconditioner(A, precision=bo.BO_PREC_FP32)
    x = _dev(case.x)
    info = M.newton(P, x, _dev(case.xn), case.dt, forcing="ew3", eps_rel=1e-6, maxit=12)
    assert info["status"] == bo.BO_OK and info["converged"], info
    xg = x.cpu().numpy()
    r = bogen.assemble(case, jacobian=False, x=xg)["b"]
    assert np.linalg.norm(r) < 1e-6 * nb0 * (1 + 1e-9)
    assert np.linalg.norm(r) == pytest.approx(info["norms"][-1], rel=1e-8)
