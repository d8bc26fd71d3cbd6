"""The C-ABI's host code under AddressSanitizer and UndefinedBehaviorSanitizer (no GPU).

compute-sanitizer is not available for the device side, so the host side is checked
the other way round: the host drivers (capi.cu: argument validation, operator
construction, workspace planning, the Newton-shift QR and Leja ordering) are compiled
with -fsanitize=address,undefined and linked with the library's other objects into a
separate library, which a child interpreter (with the sanitizer runtime preloaded)
drives through every entry point that does its work before the first CUDA call.
Any sanitizer report, or a wrong status, fails the test.
"""
import os
import shutil
import subprocess
import sys
import textwrap

import pytest

import __graft_entry__ as entry
from paper_2001_04886_gb300 import build as libbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _runtime(name):
    gcc = shutil.which("gcc")
    if not gcc:
        return None
    p = subprocess.run([gcc, f"-print-file-name={name}"], capture_output=True, text=True).stdout.strip()
    return p if os.path.isabs(p) and os.path.exists(p) else None


CHILD = textwrap.dedent(r"""
    import ctypes, math, sys
    import numpy as np
    from paper_2001_04886_gb300 import _binding as B

    L = ctypes.CDLL(sys.argv[1])
    G = ctypes.CDLL(None)   # the sanitizer runtimes are live in this process
    assert hasattr(G, "__asan_init") and hasattr(G, "__ubsan_handle_type_mismatch_v1")
    for name, (res, args) in B.SIGNATURES.items():
        fn = getattr(L, name)
        fn.restype, fn.argtypes = res, args
    ERR_ARG, ERR_OOM = -1, -3

    for code in range(-8, 3):
        assert L.sstep_status_string(code) is not None

    h = ctypes.c_void_p()
    shp = lambda *v: (ctypes.c_int64 * 3)(*v)
    coef = (ctypes.c_double * 7)(4.0, -1.1, -0.9, -1.0, -1.0, -1.0, -1.0)
    for dim, s in ((4, shp(8, 8, 1)), (1, shp(8, 8, 1)), (2, shp(0, 8, 1)), (3, shp(8, 8, 0)),
                   (3, shp(-1, 8, 8)), (3, shp(1 << 31, 2, 1)), (3, shp(2048, 2048, 1024))):
        assert L.stencil_matrix_create(ctypes.byref(h), dim, s, coef) == ERR_ARG, (dim, list(s))
    assert L.stencil_matrix_create(None, 2, shp(8, 8, 1), coef) == ERR_ARG
    assert L.stencil_matrix_create(ctypes.byref(h), 2, None, coef) == ERR_ARG
    bad = (ctypes.c_double * 7)(4.0, float("nan"), 0, 0, 0, 0, 0)
    assert L.stencil_matrix_create(ctypes.byref(h), 2, shp(8, 8, 1), bad) == ERR_ARG

    mats = []
    for dim, s in ((2, shp(1, 1, 1)), (2, shp(37, 5, 1)), (3, shp(3, 4, 5)), (3, shp(128, 128, 128))):
        m = ctypes.c_void_p()
        assert L.stencil_matrix_create(ctypes.byref(m), dim, s, coef) == 0
        n, ninf = ctypes.c_int64(), ctypes.c_double()
        assert L.stencil_matrix_info(m, ctypes.byref(n), ctypes.byref(ninf)) == 0
        assert n.value == s[0] * s[1] * (s[2] if dim == 3 else 1) and ninf.value > 0
        mats.append(m)
    m = ctypes.c_void_p()
    beta = (ctypes.c_double * 3)(30, 20, 10)
    assert L.stencil_matrix_create_convdiff(ctypes.byref(m), 3, shp(16, 12, 8), beta) == ERR_ARG   # not a cube
    assert L.stencil_matrix_create_convdiff(ctypes.byref(m), 3, shp(12, 12, 12), beta) == 0
    mats.append(m)

    b = ctypes.c_size_t()
    for ka, kb, want in ((0, 1, ERR_ARG), (65, 1, ERR_ARG), (4, 10, ERR_ARG), (4, 5, 0), (64, 9, 0), (1, 1, 0)):
        assert L.sstep_gram_workspace_size(1000, ka, kb, ctypes.byref(b)) == want, (ka, kb)

    # Newton shifts: random Hessenberg matrices (complex pairs), degenerate ones
    rng = np.random.default_rng(5)
    th = (ctypes.c_double * 8)()
    for K in (1, 2, 3, 8, 17, 40, 64):
        for s in (1, 2, 4, 8):
            G = np.triu(rng.standard_normal((K + 1, K)), -1)
            Gf = np.asfortranarray(G)
            assert L.sstep_newton_shifts(Gf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), K + 1, K, s, th) >= 0
            assert all(math.isfinite(th[i]) for i in range(s))
    Z = np.zeros((9, 8), order="F")
    assert L.sstep_newton_shifts(Z.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 9, 8, 8, th) >= 0
    assert L.sstep_newton_shifts(Z.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 9, 8, 9, th) == ERR_ARG
    assert L.sstep_newton_shifts(Z.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 7, 8, 4, th) == ERR_ARG

    # solver argument checks and the workspace cap all return before any device call
    res = B.SStepResult()
    f = ctypes.c_void_p(16)
    x = ctypes.c_void_p(32)
    def params(**kw):
        p = B.SStepParams(s=4, m=20, k=1, tol=1e-8, max_cycles=10, max_iters=10, sigma=0.0, history=None,
                          history_cap=0, precision=0, x0_guard=0, basis=0, precond=0)
        for k, v in kw.items():
            setattr(p, k, v)
        return p
    A = mats[2]
    hbuf = (ctypes.c_double * 4)()
    for name, kw in (("sstep_gmres_solve", dict(s=0)), ("sstep_gmres_solve", dict(m=18)),
                     ("sstep_gmres_solve", dict(s=9, m=18)), ("sstep_gmres_solve", dict(tol=0.0)),
                     ("sstep_gmres_solve", dict(sigma=-1.0)), ("sstep_gmres_solve", dict(basis=2)),
                     ("sstep_gmres_solve", dict(precision=7)), ("sstep_omin_solve", dict(k=-1)),
                     ("sstep_omin_solve", dict(s=8, k=9)), ("sstep_omin_solve", dict(basis=1)),
                     ("sstep_omin_solve", dict(s=8, k=8, basis=2)), ("sstep_omin_solve", dict(precision=1)),
                     ("gmres_solve", dict(m=0)),
                     ("gmres_solve", dict(history=ctypes.cast(hbuf, ctypes.POINTER(ctypes.c_double)), history_cap=-1))):
        p = params(**kw)
        rc = getattr(L, name)(A, f, x, ctypes.byref(p), ctypes.byref(res), None)
        assert rc == ERR_ARG, (name, kw, rc)
    assert L.sstep_gmres_solve(A, None, x, ctypes.byref(params()), ctypes.byref(res), None) == ERR_ARG
    assert L.sstep_set_workspace_limit(4096) == 0
    for name in ("sstep_gmres_solve", "gmres_solve", "sstep_omin_solve"):
        rc = getattr(L, name)(mats[3], f, x, ctypes.byref(params()), ctypes.byref(res), None)
        assert rc == ERR_OOM, (name, rc)
    assert L.sstep_set_workspace_limit(0) == 0

    for m in mats:
        assert L.stencil_matrix_destroy(m) == 0
    assert L.stencil_matrix_destroy(None) == ERR_ARG
    print("host sanitizer run ok")
""")


def test_host_code_under_address_and_ub_sanitizers(tmp_path):
    asan, ubsan = _runtime("libasan.so"), _runtime("libubsan.so")
    if not (asan and ubsan):
        pytest.skip("the host compiler has no sanitizer runtimes")
    entry.build()
    cc = libbuild.nvcc()
    # nvcc splits -Xcompiler values at commas: one flag each
    san = []
    for fl in ("-fsanitize=address", "-fsanitize=undefined", "-fno-omit-frame-pointer",
               "-fno-sanitize-recover=undefined"):
        san += ["-Xcompiler", fl]
    obj = str(tmp_path / "capi_san.o")
    cmd = [cc, *libbuild.ARCH, *libbuild.FLAGS, *san, "-c", os.path.join(libbuild.CSRC, "capi.cu"), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    others = [os.path.join(libbuild.OUT, s.replace(".cu", ".o")) for s in libbuild.SOURCES if s != "capi.cu"]
    so = str(tmp_path / "libsstep_san.so")
    r = subprocess.run([cc, *libbuild.ARCH, "-shared", "-cudart", "static", "-Xcompiler", "-fsanitize=address",
                        "-Xcompiler", "-fsanitize=undefined", "-o", so, obj, *others], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    env = dict(os.environ)
    env.update(LD_PRELOAD=f"{asan}:{ubsan}", ASAN_OPTIONS="detect_leaks=0:abort_on_error=1",
               UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", CHILD, so], capture_output=True, text=True, env=env, cwd=ROOT,
                       timeout=600)
    report = r.stdout + r.stderr
    assert r.returncode == 0 and "host sanitizer run ok" in r.stdout, report[-4000:]
    assert "AddressSanitizer" not in report and "runtime error" not in report, report[-4000:]
