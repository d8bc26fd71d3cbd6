"""The C-ABI library builds, loads without a GPU and exports every declared entry point."""
import os
import re

import pytest

import __graft_entry__ as entry
import paper_2001_04886_gb300 as pkg
from paper_2001_04886_gb300 import _binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "sstep.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(\w+)\s*\(", src, flags=re.M)))


def test_header_parses():
    names = declared_functions()
    assert "sstep_gmres_solve" in names and "stencil_matrix_create" in names and len(names) >= 13


def test_library_exports_every_declared_symbol():
    entry.build()
    L = pkg.lib()
    for name in declared_functions():
        assert hasattr(L, name), name
        assert name in _binding.SIGNATURES, name


def test_status_strings_and_argument_errors_without_gpu():
    L = pkg.lib()
    assert L.sstep_status_string(-4).decode().startswith("breakdown")
    # argument validation happens before any CUDA call
    import ctypes

    h = ctypes.c_void_p()
    shp = (ctypes.c_int64 * 3)(8, 8, 1)
    assert L.stencil_matrix_create(ctypes.byref(h), 4, shp, (ctypes.c_double * 7)()) == -1
    b = ctypes.c_size_t()
    assert L.sstep_gram_workspace_size(100, 0, 1, ctypes.byref(b)) == -1
    assert L.sstep_gram_workspace_size(100, 4, 5, ctypes.byref(b)) == 0 and b.value > 0


def test_params_struct_layout_matches_header():
    # sstep_params: int s, m, k; double tol; int max_cycles, max_iters; double sigma; double* history; int cap
    import ctypes

    P = _binding.SStepParams
    assert P.tol.offset == 16 and P.sigma.offset == 32 and P.history.offset == 40
    assert P.history_cap.offset == 48 and P.precision.offset == 52 and P.x0_guard.offset == 56
    assert P.basis.offset == 60 and P.precond.offset == 64
    assert ctypes.sizeof(P) == 72
    assert ctypes.sizeof(_binding.SStepResult) == 32


def test_workspace_limit_gives_oom_before_any_device_call():
    """The allocation-failure path without a GPU: a workspace cap below the solve's need
    makes sstep_gmres_solve return SSTEP_ERR_OOM (the pointers are never dereferenced)."""
    import ctypes

    L = pkg.lib()
    h = ctypes.c_void_p()
    shp = (ctypes.c_int64 * 3)(16, 16, 1)
    beta = (ctypes.c_double * 3)(10.0, 10.0, 0.0)
    assert L.stencil_matrix_create_convdiff(ctypes.byref(h), 2, shp, beta) == 0
    p = _binding.SStepParams(s=4, m=20, tol=1e-8, max_cycles=10)
    r = _binding.SStepResult()
    fake = ctypes.c_void_p(0x1000)
    assert L.sstep_set_workspace_limit(1024) == 0
    try:
        rc = L.sstep_gmres_solve(h, fake, fake, ctypes.byref(p), ctypes.byref(r), None)
        assert rc == -3   # SSTEP_ERR_OOM
    finally:
        assert L.sstep_set_workspace_limit(0) == 0
        L.stencil_matrix_destroy(h)
    assert L.sstep_set_workspace_limit(-1) == -1


def test_binding_refuses_host_tensors_without_gpu():
    """Host (CPU) tensors never reach the library: the binding raises before the call."""
    import torch

    A = pkg.StencilMatrix(2, (8, 8), beta=(20.0, 20.0))   # a host-only operator handle
    f = torch.ones(A.n, dtype=torch.float64)
    with pytest.raises(TypeError):
        pkg.sstep_gmres_solve(A, f, torch.zeros_like(f), 4, 20, 1e-8)
    with pytest.raises(TypeError):
        pkg.sstep_omin_solve(A, f, torch.zeros_like(f), 4, 1, 1e-8)
    with pytest.raises(TypeError):
        A.apply(f, torch.empty_like(f))
    A.close()
