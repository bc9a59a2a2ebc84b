"""CPU: the C-ABI library builds, loads, and exports every function include/eig.h declares."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "eig.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:EIG_API\s+)?(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s+\*?(eig_[a-z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_2305_15552_gb300 import build
    try:
        return build.build()
    except RuntimeError as e:
        pytest.fail(f"build failed: {e}")


def test_header_declares_core_api():
    names = declared_functions()
    for must in ["eig_spmm", "eig_spmm_plan_create", "eig_strerror"]:
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(l.split()[-1] for l in out.splitlines() if l.strip())
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, f"declared but not exported: {missing}"


def test_library_loads_without_gpu(libpath):
    import platform
    from paper_2305_15552_gb300 import binding
    if not binding.__dict__.get("_lib") and platform.machine() in ("x86_64", "aarch64"):
        lib = binding.load_symbols_only(libpath)
        assert lib.eig_strerror(0) == b"EIG_OK"
        assert b"sm_103a" in lib.eig_version()
