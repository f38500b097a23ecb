"""The C-ABI library builds and exports every function include/bosolve.h
declares (no compute calls: runs without a GPU)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "bosolve.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?\w+\**\s+\**(bo_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_1606_00556_gb300.buildlib import build
    return build()


def test_header_declarations_parsed():
    names = _declared()
    assert "bo_solve" in names and "bo_mat_create_bsr" in names and len(names) >= 19


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(bo_\w+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_binding_lists_every_declared_symbol(libpath):
    import ctypes

    import paper_1606_00556_gb300 as bo
    assert sorted(bo.EXPORTS) == _declared()
    L = ctypes.CDLL(libpath)
    for n in _declared():
        assert hasattr(L, n)


def test_library_is_built_for_sm_103a_only():
    # every translation unit and the link step get exactly one -gencode,
    # for sm_103a (no PTX of another architecture, no JIT fallback)
    from paper_1606_00556_gb300 import buildlib
    assert buildlib.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert not any("gencode" in f or "arch" in f for f in buildlib.FLAGS)


def test_product_path_has_no_oracle_or_fallback():
    pkg = os.path.join(ROOT, "paper_1606_00556_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "liboracle" not in txt, f


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    import paper_1606_00556_gb300 as bo
    monkeypatch.setattr(bo, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(bo, "_lib", None)
    with pytest.raises(RuntimeError):
        bo.lib()


def test_host_side_contract_without_a_gpu(libpath):
    # the parts of the boundary that touch no device: status strings, option
    # defaults, process-wide switches and the rejection of missing arguments
    import ctypes

    import paper_1606_00556_gb300 as bo
    L = bo.lib()
    for code in range(0, -9, -1):
        s = L.bo_status_str(code)
        assert isinstance(s, bytes) and len(s) > 0
    po = bo.bo_prec_opts()
    L.bo_prec_opts_default(ctypes.byref(po))
    assert (po.precision, po.amg_nu1, po.amg_nu2, po.amg_coarse_max) == (bo.BO_PREC_FP64, 2, 2, 128)
    assert po.amg_overcorr == 1.3 and po.decoupling == bo.BO_DECOUPLE_QI
    so = bo.bo_solve_opts()
    L.bo_solve_opts_default(ctypes.byref(so))
    assert (so.tol, so.restart, so.maxit, so.mem) == (1e-8, 30, 500, bo.BO_MEM_DEVICE)
    assert L.bo_set_amg_cooperative(3) == bo.BO_ERR_ARG and L.bo_set_amg_cooperative(-1) == bo.BO_ERR_ARG
    assert L.bo_set_amg_cooperative(1) == bo.BO_OK and L.bo_set_amg_cooperative(2) == bo.BO_OK
    assert L.bo_set_gs_fused(2) == bo.BO_ERR_ARG and L.bo_set_gs_fused(1) == bo.BO_OK
    assert L.bo_set_conv_engine(7) == bo.BO_ERR_ARG
    for f in ("bo_solve", "bo_solve_bicgstab"):
        assert getattr(L, f)(None, None, None, None, None) == bo.BO_ERR_ARG
    assert L.bo_solve_batched(None, 0, None, None, None, None) == bo.BO_ERR_ARG
    assert L.bo_prec_update(None) == bo.BO_ERR_ARG
    assert L.bo_prec_destroy(None) == bo.BO_ERR_ARG and L.bo_mat_destroy(None) == bo.BO_ERR_ARG
    assert L.bo_prec_apply(None, 0, None, None) == bo.BO_ERR_ARG
    assert L.bo_newton_update(None, None, None, 0) == bo.BO_ERR_ARG
    assert L.bo_ctx_create(0, None, None) == bo.BO_ERR_ARG


def test_every_entry_point_rejects_missing_handles(libpath):
    # no call dereferences a NULL handle or pointer: each returns BO_ERR_ARG
    # before it touches the device (so this runs without a GPU)
    import ctypes

    import paper_1606_00556_gb300 as bo
    L = bo.lib()
    N = None
    calls = {
        "bo_mat_create_bsr": (N, N, 0, 0, N, N, N, 0, N),
        "bo_mat_create_csr": (N, N, 0, 0, N, N, N, 0, N),
        "bo_mat_update_values": (N, N, 0),
        "bo_mat_spmv": (N, 1.0, N, 0.0, N, 0),
        "bo_mat_residual_noalloc": (N, N, N, N, N),
        "bo_prec_setup": (N, N, N),
        "bo_prec_spmv_decoupled": (N, N, N),
        "bo_prec_amg_levels": (N, N, 0),
        "bo_prec_set_launch_mode": (N, 0),
        "bo_prec_set_amg_tile": (N, 1, 256),
        "bo_prec_set_coarse_space": (N, N, 1, 1, 1),
        "bo_learned_coarse_space": (N, N, ctypes.c_double(1.0), 1, 1, 1),
        "bo_prec_residual_history": (N, N, 0),
        "bo_learned_guess": (N, N, N, N, 1, N, N),
        "bo_update_batched": (N, 0, N, 0),
        "bo_autotune_batched": (N, 0, N, N, N, N, N),
        "bo_dp_create": (N, N, 0, 0, N, N, N, 0, N),
        "bo_dp_update_values": (N, N, 0),
        "bo_dp_solve": (N, N, N, N, N, N),
        "bo_dp_destroy": (N,),
        "bo_dp_solve_batched": (N, N, 0, N, N, N, N),
        "bo_wells_create": (N, 1, 0, N, N, N),
        "bo_wells_update_values": (N, N, N, N, 0),
        "bo_wells_set_coupling": (N, 1),
        "bo_wells_spmv": (N, ctypes.c_double(1.0), N, ctypes.c_double(0.0), N),
        "bo_solve_bordered": (N, N, N, N, N, N),
        "bo_wells_destroy": (N,),
        "bo_ow_create": (N, N, 0, 0, N, N, N, 0, N),
        "bo_ow_update_values": (N, N, 0),
        "bo_ow_spmv": (N, ctypes.c_double(1.0), N, ctypes.c_double(0.0), N),
        "bo_ow_solve": (N, N, N, N, N, N),
        "bo_ow_solve_bicgstab": (N, N, N, N, N, N),
        "bo_ow_destroy": (N,),
        "bo_cnn_create": (N, 8, 8, 8, 1, ctypes.c_uint64(0), N),
        "bo_cnn_destroy": (N,),
        "bo_cnn_get_params": (N, N, 0),
        "bo_cnn_set_params": (N, N, 0),
        "bo_cnn_get_grads": (N, N, 0),
        "bo_cnn_forward": (N, N, 1, N),
        "bo_cnn_backward": (N, N, N, N, 1, 1, N),
        "bo_cnn_adam_step": (N, ctypes.c_float(1e-3)),
        "bo_conv3d_forward": (N, 8, 8, 8, 1, 32, 32, N, N, N, N, 1, N, N),
        "bo_conv3d_backward_data": (N, 8, 8, 8, 1, 32, 32, N, N, N),
        "bo_conv3d_backward_weights": (N, 8, 8, 8, 1, 32, 32, N, N, N, N),
        "bo_ctx_destroy": (N,),
        "bo_model_create": (N, N, N, N, N, N, N, N, 0, N, N, N, N, N, N),
        "bo_model_destroy": (N,),
        "bo_model_assemble": (N, N, N, ctypes.c_double(1.0), N, N, N),
        "bo_newton_solve": (N, N, N, N, ctypes.c_double(1.0), N, N),
    }
    for name, args in calls.items():
        assert getattr(L, name)(*args) == bo.BO_ERR_ARG, name
    assert L.bo_dp_fracture_matrix(None) is None
    assert L.bo_ow_matrix(None) is None
    # the stream pool is 1..16 wide
    assert L.bo_set_batch_streams(0) == bo.BO_ERR_ARG and L.bo_set_batch_streams(17) == bo.BO_ERR_ARG
