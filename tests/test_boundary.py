"""CPU checks of the C-ABI boundary: the library loads, exports every symbol
include/cp.h declares, fills option defaults, and reports errors without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "cp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"typedef[^;]*;", "", src, flags=re.S)
    names = re.findall(r"([A-Za-z_][A-Za-z0-9_]*)\s*\([^;{}]*\)\s*;", src)
    return sorted(set(names))


def test_header_declares_the_named_calls():
    names = header_functions()
    for call in ["cp_mttkrp", "cp_als_sweep", "cp_fg", "ngmres_step", "linesearch", "cp_solve"]:
        assert call in names


def test_library_exports_every_declared_symbol():
    import paper_1105_5331_gb300 as cp
    lib = ctypes.CDLL(cp._binding.LIB_PATH)
    names = header_functions()
    assert names, "no declarations parsed"
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(cp.EXPORTED) == sorted(n for n in names if n in cp.EXPORTED)
    assert set(names) <= set(cp.EXPORTED) | set()


def test_option_defaults_follow_the_paper():
    import paper_1105_5331_gb300 as cp
    ls = cp.cp_ls_opts_default()
    assert (ls.ftol, ls.gtol, ls.stp0, ls.maxfev) == (1e-4, 1e-2, 1.0, 20)
    o = cp.cp_solve_opts_default(7)
    assert (o.R, o.w, o.eps, o.tol, o.prec) == (7, 20, 1e-12, 1e-7, cp.CP_FP64)


def test_errors_cross_the_abi_as_status_codes():
    import paper_1105_5331_gb300 as cp
    lib = cp.library()
    # NULL output pointer is rejected before any CUDA call
    assert lib.cp_ctx_create(0, None, None) == 1
    assert "null argument" in cp.cp_last_error()
    assert lib.cp_tensor_info(None, None, None, None) == 1
    assert lib.cp_solve(None, None, None, None, None) == 1


def test_no_gpu_means_a_cuda_error_not_a_fallback():
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    import paper_1105_5331_gb300 as cp
    with pytest.raises(cp.CpError) as ei:
        cp.cp_ctx_create(0)
    assert ei.value.status in (1, 4)


def test_package_without_its_library_fails_to_import(tmp_path):
    """A copy of the package without the built library must refuse to import
    (no CPU fallback path exists)."""
    import shutil
    import subprocess
    import sys
    src = os.path.join(ROOT, "paper_1105_5331_gb300")
    dst = tmp_path / "paper_1105_5331_gb300"
    shutil.copytree(src, dst, ignore=shutil.ignore_patterns("*.so", "_build", "__pycache__", "csrc"))
    r = subprocess.run([sys.executable, "-c", "import paper_1105_5331_gb300"], cwd=tmp_path,
                       capture_output=True, text=True, env=dict(os.environ, PYTHONPATH=str(tmp_path)))
    assert r.returncode != 0
    assert "ImportError" in r.stderr and "no CPU fallback" in r.stderr
