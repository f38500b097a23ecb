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


def test_library_is_built_for_sm_103a(libpath):
    # the embedded cubin's target, as the CUDA tools report it (no disassembly)
    r = subprocess.run(["cuobjdump", "--list-elf", libpath], capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip("cuobjdump unavailable")
    assert "sm_103a" in r.stdout


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
