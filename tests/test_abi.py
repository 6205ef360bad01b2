"""The C-ABI library loads and exports every symbol its headers declare.
No compute calls: this runs on a machine without a GPU."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(gpch_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    from paper_2605_13209_b300 import build
    return build.build()


def test_header_declares_the_scope_entry_points():
    names = declared_symbols()
    for required in ("gpch_create", "gpch_destroy", "gpch_se_matrix", "gpch_chol_factor", "gpch_chol_solve",
                     "gpch_cg_solve"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_and_version(libpath):
    lib = ctypes.CDLL(libpath)
    lib.gpch_status_string.restype = ctypes.c_char_p
    for code, name in enumerate(["GPCH_OK", "GPCH_INVALID_ARG", "GPCH_NOT_SPD", "GPCH_NOT_CONVERGED",
                                 "GPCH_OOM_BUDGET", "GPCH_TIMEOUT", "GPCH_CUDA_ERROR"]):
        assert lib.gpch_status_string(code).decode() == name
    assert lib.gpch_version() == 1


def test_no_cpu_fallback_without_gpu(libpath):
    """Without a GPU, context creation fails loudly instead of computing on
    the host."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    lib = ctypes.CDLL(libpath)
    h = ctypes.c_void_p()
    assert lib.gpch_create(ctypes.byref(h), 0, 0) == 6   # GPCH_CUDA_ERROR
    from paper_2605_13209_b300 import gpchol
    with pytest.raises(Exception):
        gpchol.Context(0)


def test_product_package_never_imports_oracle():
    pkg = os.path.join(ROOT, "paper_2605_13209_b300")
    for f in glob.glob(os.path.join(pkg, "**", "*.*"), recursive=True):
        if f.endswith((".py", ".cu", ".cuh", ".h")):
            src = open(f).read()
            assert "import oracle" not in src and "from oracle" not in src and "gp_oracle" not in src, f
