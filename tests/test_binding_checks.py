"""The binding checks what the C ABI cannot (plain pointers carry no size or
type): dtype, length, layout and host/device placement of every buffer.
These run without a GPU: the objects below have no handle, so a rejected
argument must fail before the library is called, and an accepted one reaches
the library, which answers BO_ERR_ARG for the missing handle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def bo():
    from paper_1606_00556_gb300.buildlib import build
    build()
    import paper_1606_00556_gb300 as bo
    return bo


class _Ctx:
    h = None
    device = 0


def _prec(bo, N=24):
    g = bo.grid(4, 3, 2)
    m = bo.Matrix(_Ctx(), g, None, (), nval=9 * 100)
    P = object.__new__(bo.Preconditioner)
    P.mat, P.h = m, None
    return P, 3 * N


def _reaches_library(bo, fn):
    with pytest.raises(bo.BoError) as e:
        fn()
    assert not isinstance(e.value, bo.BoArgError) and e.value.status == bo.BO_ERR_ARG


def test_arg_error_is_a_bo_error_and_a_value_error(bo):
    e = bo.BoArgError("x")
    assert isinstance(e, bo.BoError) and isinstance(e, ValueError) and isinstance(e, TypeError)
    assert e.status == bo.BO_ERR_ARG


def test_solve_checks_host_vectors(bo):
    P, n = _prec(bo)
    b = np.ones(n)
    # wrong length of either vector
    with pytest.raises(bo.BoArgError):
        P.solve(np.ones(n - 1), np.zeros(n))
    with pytest.raises(bo.BoArgError):
        P.solve(b, np.zeros(n + 3))
    # x is written in place: it must already be contiguous float64
    with pytest.raises(bo.BoArgError):
        P.solve(b, np.zeros(n, np.float32))
    with pytest.raises(bo.BoArgError):
        P.solve(b, np.zeros(2 * n)[::2])
    ro = np.zeros(n)
    ro.flags.writeable = False
    with pytest.raises(bo.BoArgError):
        P.solve_bicgstab(b, ro)
    # a CPU tensor of the wrong dtype
    with pytest.raises(bo.BoArgError):
        P.solve(torch.ones(n, dtype=torch.float32), torch.zeros(n, dtype=torch.float64))
    # an input of another dtype is converted, and valid buffers reach the library
    _reaches_library(bo, lambda: P.solve(np.ones(n, np.float32), np.zeros(n)))
    _reaches_library(bo, lambda: P.solve_bicgstab(torch.ones(n, dtype=torch.float64), torch.zeros(n, dtype=torch.float64)))


def test_device_only_calls_reject_host_buffers(bo):
    P, n = _prec(bo)
    x, y = torch.zeros(n, dtype=torch.float64), torch.zeros(n, dtype=torch.float64)
    for call in (lambda: P.mat.spmv(x, y), lambda: P.apply(bo.BO_STAGE_CPR, x, y), lambda: P.spmv_decoupled(x, y),
                 lambda: bo.bo_mat_residual_noalloc(P.mat, x, x, y, torch.zeros(2, dtype=torch.float64)),
                 lambda: bo.bo_newton_update(_Ctx(), x, y), lambda: P.set_coarse_space(torch.zeros(n // 3, dtype=torch.float64))):
        with pytest.raises(bo.BoArgError):
            call()


def test_matrix_constructors_check_array_sizes(bo):
    from bogen import pattern
    g = bo.grid(4, 3, 2)
    rp, col = pattern(4, 3, 2)
    val = np.zeros((col.size, 3, 3))
    with pytest.raises(bo.BoArgError):
        bo.Matrix.from_bsr(_Ctx(), g, rp[:-1], col, val)
    with pytest.raises(bo.BoArgError):
        bo.Matrix.from_bsr(_Ctx(), g, rp, col, val[:-1])
    with pytest.raises(bo.BoArgError):
        bo.Matrix.from_bsr(_Ctx(), g, torch.from_numpy(rp.astype(np.int64)), torch.from_numpy(col),
                           torch.from_numpy(val))
    with pytest.raises(bo.BoArgError):  # CSR: one value per column index
        bo.Matrix.from_csr(_Ctx(), g, np.zeros(3 * 24 + 1, np.int32), np.zeros(5, np.int32), np.zeros(4))
    # consistent arrays reach the library (which rejects the missing context)
    _reaches_library(bo, lambda: bo.Matrix.from_bsr(_Ctx(), g, rp, col, val))


def test_value_update_checks_the_count(bo):
    P, _ = _prec(bo)
    with pytest.raises(bo.BoArgError):
        P.mat.update_values(np.zeros(899))
    _reaches_library(bo, lambda: P.mat.update_values(np.zeros(900)))
