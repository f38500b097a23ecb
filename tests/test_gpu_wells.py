"""Rate-controlled wells on the GPU (bo_wells, bo_solve_bordered) against the
oracle's bordered system (paper Sec. 2.3 controls, Sec. 3.2 block form):
the bordered product element by element, bordered solves against the
oracle's GMRES + ILU(0) solution of the whole bordered matrix, the
Woodbury-corrected preconditioner's iteration counts, Newton with well
unknowns, the 1M-cell waterflood with every well rate-controlled, and the
argument errors.

Tolerances:
  * product: the cell rows come from the public FP64 SpMV (split products,
    below 2^-44 of sum |a||x| per row); the border terms are FP64 FMAs, so
    |y - y_ref| <= 1e-12 (|A_b| |x|) per row;
  * solves: the oracle solution at 1e-13 is the reference; a solve to 1e-8
    is within 1e-6 of it in relative 2-norm (the survey's parity bar), and
    its FP64 residual, recomputed by the oracle, is at most 1e-8."""
import numpy as np
import pytest

import bogen
import oracle
from bogen import CTRL_LIQUID, CTRL_OIL, Well
from oracle.bordered import bordered_bsr, bordered_matvec, bordered_solve
from oracle.newton import inexact_newton_wells

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


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _case(seed, nx=20, ny=20, nz=5, producer_control=CTRL_LIQUID, third=False):
    c = bogen.tiny_case(seed, nx, ny, nz)
    if third:
        mid = np.array([nx // 2 + nx * (ny // 2 + ny * k) for k in range(nz)], np.int32)
        c.wells.append(Well(1, 2700.0, mid))
    return bogen.with_rate_controls(c, fraction=0.8, producer_control=producer_control)


def _gpu(bo, ctx, case, a, precision):
    A = bo.Matrix.from_bsr(ctx, bo.grid(case.nx, case.ny, case.nz, case.dx, case.dy, case.dz), a["rowptr"],
                           a["col"], a["val"])
    bd = a["border"]
    wl = bo.Wells(A, bd["aww"].size, bd["perf_cell"], bd["perf_well"], bd["apw"].ravel(), bd["awp"].ravel(),
                  bd["aww"])
    P = bo.Preconditioner(A, precision=precision)
    return A, wl, P


def _abs_product(A, bd, x):
    """|A_b| |x| per row (the scale of a product's rounding)."""
    Aa = oracle.BsrMatrix(A.rowptr, A.col, np.abs(A.val))
    bda = dict(bd, apw=np.abs(bd["apw"]), awp=np.abs(bd["awp"]), aww=np.abs(bd["aww"]))
    return bordered_matvec(Aa, bda, np.abs(x))


@pytest.mark.parametrize("seed", [0, 1])
def test_bordered_product_matches_oracle(bo, ctx, seed):
    case = _case(seed, 16, 12, 6, third=True)
    a = bogen.assemble(case)
    A, wl, P = _gpu(bo, ctx, case, a, bo.BO_PREC_FP64)
    Ao = oracle.BsrMatrix(a["rowptr"], a["col"], a["val"])
    rng = np.random.default_rng(seed)
    n = 3 * case.N + a["border"]["aww"].size
    x = rng.standard_normal(n)
    x[3 * case.N:] *= 100.0
    y0 = rng.standard_normal(n)
    ref = 0.7 * bordered_matvec(Ao, a["border"], x) - 0.3 * y0
    y = _dev(y0)
    wl.spmv(_dev(x), y, alpha=0.7, beta=-0.3)
    bound = 1e-12 * (0.7 * _abs_product(Ao, a["border"], x) + 0.3 * np.abs(y0))
    assert np.all(np.abs(y.cpu().numpy() - ref) <= bound)


@pytest.fixture(scope="module")
def cases():
    out = {}
    for name, kw in {"s0_liquid": dict(seed=0), "s1_oil": dict(seed=1, producer_control=CTRL_OIL),
                     "s2_three_wells": dict(seed=2, third=True)}.items():
        case = _case(**kw)
        a = bogen.assemble(case)
        Ao = oracle.BsrMatrix(a["rowptr"], a["col"], a["val"])
        xo, info = bordered_solve(Ao, a["border"], a["b_full"], tol=1e-13)
        assert info["converged"]
        out[name] = (case, a, Ao, xo)
    return out


@pytest.mark.parametrize("name", ["s0_liquid", "s1_oil", "s2_three_wells"])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
def test_bordered_solve_matches_oracle(bo, ctx, cases, name, prec):
    case, a, Ao, xo = cases[name]
    precision = {"fp64": bo.BO_PREC_FP64, "fp32": bo.BO_PREC_FP32, "bf16": bo.BO_PREC_BF16}[prec]
    A, wl, P = _gpu(bo, ctx, case, a, precision)
    x = torch.zeros(xo.size, dtype=torch.float64, device="cuda")
    info = wl.solve(P, _dev(a["b_full"]), x, tol=1e-8, maxit=300)
    assert info["rc"] == bo.BO_OK and info["true_rel_res"] <= 1e-8
    xg = x.cpu().numpy()
    r = a["b_full"] - bordered_matvec(Ao, a["border"], xg)
    assert np.linalg.norm(r) <= 1e-8 * np.linalg.norm(a["b_full"]) * (1 + 1e-6)
    assert np.linalg.norm(xg - xo) <= 1e-6 * np.linalg.norm(xo)
    # the well unknowns themselves (a few psi of p_h change) to the same bar
    W = a["border"]["aww"].size
    assert np.abs(xg[-W:] - xo[-W:]).max() <= 1e-6 * np.linalg.norm(xo)


def test_woodbury_correction_keeps_the_iteration_count(bo, ctx, cases):
    case, a, Ao, xo = cases["s2_three_wells"]
    A, wl, P = _gpu(bo, ctx, case, a, bo.BO_PREC_FP32)
    b = _dev(a["b_full"])
    x = torch.zeros(xo.size, dtype=torch.float64, device="cuda")
    with_c = wl.solve(P, b, x, tol=1e-8, maxit=300)
    # the same reservoir matrix with the wells at fixed BHP (no border)
    x3 = torch.zeros(3 * case.N, dtype=torch.float64, device="cuda")
    plain = P.solve(_dev(a["b"]), x3, tol=1e-8, maxit=300)
    wl.set_coupling(0)
    x.zero_()
    without = wl.solve(P, b, x, tol=1e-8, maxit=300, raise_on_error=False)
    assert with_c["iters"] <= plain["iters"] + 2
    assert without["iters"] > with_c["iters"]
    assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-6 * np.linalg.norm(xo) or without["rc"] != bo.BO_OK


def test_nonzero_initial_guess_and_repeat_solves(bo, ctx, cases):
    case, a, Ao, xo = cases["s0_liquid"]
    A, wl, P = _gpu(bo, ctx, case, a, bo.BO_PREC_FP32)
    rng = np.random.default_rng(3)
    x = _dev(xo * (1 + 1e-3 * rng.standard_normal(xo.size)))
    info = wl.solve(P, _dev(a["b_full"]), x, tol=1e-8, x0_is_zero=False)
    assert info["true_rel_res"] <= 1e-8
    assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-6 * np.linalg.norm(xo)
    # after new well values and a preconditioner update the setup is redone
    bd = a["border"]
    wl.update_values(_dev(bd["apw"].ravel()), _dev(bd["awp"].ravel()), _dev(bd["aww"]))
    P.update()
    x.zero_()
    info2 = wl.solve(P, _dev(a["b_full"]), x, tol=1e-8)
    assert info2["true_rel_res"] <= 1e-8
    assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-6 * np.linalg.norm(xo)
    # zero right-hand side: zero solution, no iterations
    x.fill_(1.0)
    info3 = wl.solve(P, torch.zeros_like(x), x)
    assert info3["iters"] == 0 and float(x.abs().max()) == 0.0


def test_newton_with_rate_wells_follows_the_oracle(bo, ctx):
    case = _case(4, 10, 10, 4, third=True)
    N = case.N
    b0 = float(np.linalg.norm(bogen.assemble(case)["b_full"]))
    xo, io = inexact_newton_wells(case, eps=1e-9 * b0, forcing=1e-10, maxit=30)
    assert io["converged"]
    # the same Alg. 1 with the device bordered solve (near-exact linear solves)
    ph = np.array([w.bhp for w in bogen.rate_wells(case)])
    z = np.concatenate([case.x, ph])
    norms = []
    A = wl = P = None
    for it in range(30):
        a = bogen.assemble(case, x=z[:3 * N], ph=z[3 * N:])
        norms.append(float(np.linalg.norm(a["b_full"])))
        if norms[-1] < 1e-9 * b0:
            break
        if A is None:
            A, wl, P = _gpu(bo, ctx, case, a, bo.BO_PREC_FP64)
        else:
            A.update_values(a["val"])
            bd = a["border"]
            wl.update_values(bd["apw"].ravel(), bd["awp"].ravel(), bd["aww"])
            P.update()
        dz = torch.zeros(z.size, dtype=torch.float64, device="cuda")
        info = wl.solve(P, _dev(a["b_full"]), dz, tol=1e-10, maxit=300)
        assert info["true_rel_res"] <= 1e-10
        z = z + dz.cpu().numpy()
    assert norms[-1] < 1e-9 * b0
    assert len(norms) - 1 == io["iters"]
    for ng, no in zip(norms[:-1], io["norms"][:-1]):
        assert ng == pytest.approx(no, rel=1e-6)
    assert np.linalg.norm(z - xo) <= 1e-9 * np.linalg.norm(xo)


def test_waterflood_1m_cells_with_rate_controlled_wells(bo, ctx):
    # the benchmark's 128 x 128 x 64 Jacobian with all five wells under rate
    # control (four water-rate injectors, one liquid-rate producer)
    case = bogen.with_rate_controls(bogen.waterflood_case(128, 128, 64, seed=42, day=0))
    a = bogen.assemble(case)
    A, wl, P = _gpu(bo, ctx, case, a, bo.BO_PREC_FP32)
    x = torch.zeros(a["b_full"].size, dtype=torch.float64, device="cuda")
    info = wl.solve(P, _dev(a["b_full"]), x, tol=1e-8, maxit=400)
    assert info["rc"] == bo.BO_OK
    Ao = oracle.BsrMatrix(a["rowptr"], a["col"], a["val"])
    r = a["b_full"] - bordered_matvec(Ao, a["border"], x.cpu().numpy())
    assert np.linalg.norm(r) <= 1e-8 * np.linalg.norm(a["b_full"]) * (1 + 1e-6)
    assert info["true_rel_res"] == pytest.approx(np.linalg.norm(r) / np.linalg.norm(a["b_full"]), rel=1e-3, abs=1e-12)


def test_wells_argument_errors(bo, ctx):
    case = _case(0, 8, 6, 3)
    a = bogen.assemble(case)
    A, wl, P = _gpu(bo, ctx, case, a, bo.BO_PREC_FP32)
    bd = a["border"]
    W = bd["aww"].size
    pc, pw = bd["perf_cell"], bd["perf_well"]
    with pytest.raises(bo.BoError) as e:  # a cell perforated twice
        bo.Wells(A, W, np.concatenate([pc, pc[:1]]), np.concatenate([pw, [W - 1]]))
    assert e.value.status == bo.BO_ERR_ARG
    with pytest.raises(bo.BoError) as e:  # perforations not grouped by well
        bo.Wells(A, W, pc, pw[::-1].copy())
    assert e.value.status == bo.BO_ERR_ARG
    with pytest.raises(bo.BoError) as e:  # a cell outside the grid
        bo.Wells(A, W, np.where(np.arange(pc.size) == 0, case.N, pc), pw)
    assert e.value.status == bo.BO_ERR_ARG
    w2 = bo.Wells(A, W, pc, pw)
    with pytest.raises(bo.BoError) as e:  # a constraint without its own p_h
        w2.update_values(bd["apw"].ravel(), bd["awp"].ravel(), np.zeros(W))
    assert e.value.status == bo.BO_ERR_BREAKDOWN
    bad = bd["apw"].ravel().copy()
    bad[1] = np.nan
    with pytest.raises(bo.BoError) as e:
        w2.update_values(bad, bd["awp"].ravel(), bd["aww"])
    assert e.value.status == bo.BO_ERR_NONFINITE
    x = torch.zeros(3 * case.N + W, dtype=torch.float64, device="cuda")
    with pytest.raises(bo.BoError) as e:  # no values yet
        w2.solve(P, _dev(a["b_full"]), x)
    assert e.value.status == bo.BO_ERR_ARG
    # a preconditioner of another matrix
    A2 = bo.Matrix.from_bsr(ctx, bo.grid(case.nx, case.ny, case.nz), a["rowptr"], a["col"], a["val"])
    P2 = bo.Preconditioner(A2, precision=bo.BO_PREC_FP32)
    with pytest.raises(bo.BoError) as e:
        wl.solve(P2, _dev(a["b_full"]), x)
    assert e.value.status == bo.BO_ERR_ARG
    with pytest.raises(bo.BoError) as e:
        wl.set_coupling(2)
    assert e.value.status == bo.BO_ERR_ARG
