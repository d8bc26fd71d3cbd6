"""ctypes binding of libsstep.so (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os
import threading

SSTEP_MAX_S = 8
SSTEP_MAX_M = 64
SSTEP_MAX_COLS = 64

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_lib", "libsstep.so")
_lib = None
_lock = threading.Lock()

c_int, c_double, c_void_p, c_int64, c_size_t = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_int64, ctypes.c_size_t
P = ctypes.POINTER


class SStepParams(ctypes.Structure):
    _fields_ = [("s", c_int), ("m", c_int), ("k", c_int), ("tol", c_double), ("max_cycles", c_int),
                ("max_iters", c_int), ("sigma", c_double), ("history", P(c_double)), ("history_cap", c_int),
                ("precision", c_int), ("x0_guard", c_int), ("basis", c_int), ("precond", c_int)]


PRECISIONS = {"fp64": 0, "df64": 1, "fp32": 2}


class SStepResult(ctypes.Structure):
    _fields_ = [("status", c_int), ("cycles", c_int), ("iters", c_int), ("matvecs", c_int),
                ("history_len", c_int), ("relres", c_double)]


# name -> (restype, argtypes); every entry point declared in include/sstep.h
SIGNATURES = {
    "stencil_matrix_create": (c_int, [P(c_void_p), c_int, P(c_int64), P(c_double)]),
    "stencil_matrix_create_fields": (c_int, [P(c_void_p), c_int, P(c_int64), P(c_void_p), c_void_p]),
    "stencil_matrix_create_convdiff": (c_int, [P(c_void_p), c_int, P(c_int64), P(c_double)]),
    "stencil_matrix_create_convdiff_variable": (c_int, [P(c_void_p), c_int64, c_void_p, c_void_p]),
    "stencil_matrix_destroy": (c_int, [c_void_p]),
    "stencil_matrix_info": (c_int, [c_void_p, P(c_int64), P(c_double)]),
    "stencil_matrix_apply": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "sstep_last_shifts": (c_int, [c_void_p, P(c_double), c_int]),
    "stencil_matrix_rbilu0_apply": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "stencil_matrix_ilu0_apply": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "sstep_newton_shifts": (c_int, [P(c_double), c_int, c_int, c_int, P(c_double)]),
    "sstep_set_workspace_limit": (c_int, [c_int64]),
    "stencil_matrix_smooth": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_double, c_void_p]),
    "stencil_matrix_smooth_batched": (c_int, [c_int, P(c_void_p), P(c_void_p), P(c_void_p), P(c_void_p), c_int,
                                              c_double, c_void_p]),
    "sstep_matrix_powers": (c_int, [c_void_p, c_void_p, c_double, c_double, c_int, c_void_p, c_int64, c_void_p]),
    "sstep_gram_workspace_size": (c_int, [c_int64, c_int, c_int, P(c_size_t)]),
    "sstep_gram": (c_int, [c_int64, c_void_p, c_int64, c_int, c_void_p, c_int64, c_int, c_void_p, c_int,
                           c_void_p, c_size_t, c_void_p]),
    "sstep_gram_tc": (c_int, [c_int64, c_void_p, c_int64, c_int, c_void_p, c_int64, c_int, c_void_p, c_int,
                              c_void_p, c_size_t, c_void_p]),
    "sstep_set_tc_wait_limit": (c_int, [ctypes.c_long]),
    "sstep_gram_noalloc": (c_int, [c_int64, c_void_p, c_int64, c_int, c_void_p, c_int64, c_int, c_void_p, c_int,
                                   c_void_p]),
    "sstep_block_update": (c_int, [c_int64, c_void_p, c_int64, c_int, c_void_p, c_int64, c_int, c_void_p, c_int,
                                   c_void_p, c_void_p, c_size_t, c_void_p]),
    "sstep_block_update_tc": (c_int, [c_int64, c_void_p, c_int64, c_int, c_void_p, c_int64, c_int, c_void_p, c_int,
                                      c_void_p, c_void_p, c_size_t, c_void_p]),
    "sstep_gmres_solve": (c_int, [c_void_p, c_void_p, c_void_p, P(SStepParams), P(SStepResult), c_void_p]),
    "gmres_solve": (c_int, [c_void_p, c_void_p, c_void_p, P(SStepParams), P(SStepResult), c_void_p]),
    "sstep_omin_solve": (c_int, [c_void_p, c_void_p, c_void_p, P(SStepParams), P(SStepResult), c_void_p]),
    "sstep_status_string": (ctypes.c_char_p, [c_int]),
    "sstep_batch_create": (c_int, [P(c_void_p), c_int, P(c_void_p), P(SStepParams)]),
    "sstep_batch_solve": (c_int, [c_void_p, P(c_void_p), P(c_void_p), P(SStepResult), c_int, c_void_p]),
    "sstep_batch_tune": (c_int, [c_void_p, P(c_void_p), P(c_void_p), P(c_int), P(c_int), P(c_int), P(c_int),
                                 P(c_int64), c_void_p]),
    "sstep_batch_configure": (c_int, [c_void_p, c_int, c_int, c_int, c_int, c_int64]),
    "sstep_batch_destroy": (c_int, [c_void_p]),
    "x0net_create": (c_int, [P(c_void_p), c_int, c_int, c_int, c_int, c_int]),
    "x0net_destroy": (c_int, [c_void_p]),
    "x0net_num_params": (c_int, [c_void_p, P(c_int64)]),
    "x0net_set_residual_weight": (c_int, [c_void_p, ctypes.c_float, ctypes.c_float]),
    "x0net_set_params": (c_int, [c_void_p, c_void_p, c_void_p]),
    "x0net_get_params": (c_int, [c_void_p, c_void_p, c_void_p]),
    "x0net_get_state": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, P(c_int64), c_void_p]),
    "x0net_set_state": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_void_p]),
    "x0net_forward": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_void_p]),
    "x0net_features": (c_int, [c_int, c_int, c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "x0net_targets": (c_int, [c_int, c_int, c_int, c_void_p, c_void_p, c_void_p, c_void_p]),
    "x0net_predict": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_void_p]),
    "x0net_gradient": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_void_p]),
    "x0net_set_tensor_cores": (c_int, [c_void_p, c_int]),
    "x0net_status": (c_int, [c_void_p, c_void_p]),
    "x0net_set_wait_limit": (c_int, [c_void_p, c_int64]),
    "x0net_train_step": (c_int, [c_void_p, c_void_p, c_void_p, c_int, ctypes.c_float, c_void_p, c_void_p]),
    "sstep_trace_select": (c_int, [ctypes.c_uint]),
    "sstep_trace_enable": (c_int, [c_int]),
    "sstep_trace_kinds": (c_int, []),
    "sstep_trace_kind_name": (ctypes.c_char_p, [c_int]),
    "sstep_trace_read": (c_int, [c_int, P(c_double), P(c_int64)]),
}


class SStepError(RuntimeError):
    def __init__(self, name, status):
        msg = lib().sstep_status_string(status).decode()
        super().__init__(f"{name} failed: {msg} (status {status})")
        self.status = status


def lib():
    """The loaded libsstep.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is None:
        with _lock:
            if _lib is None:
                if not os.path.exists(_LIB_PATH):
                    raise ImportError(
                        f"libsstep.so not found at {_LIB_PATH}; build it with "
                        "`python -c 'import __graft_entry__ as g; g.build()'`")
                L = ctypes.CDLL(_LIB_PATH)
                for name, (res, args) in SIGNATURES.items():
                    fn = getattr(L, name)
                    fn.restype = res
                    fn.argtypes = args
                _lib = L
    return _lib


def _check(name, rc):
    if rc < 0:
        raise SStepError(name, rc)
    return rc


def _ptr(t):
    import torch

    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch tensor")
    if not t.is_cuda or t.dtype != torch.float64:
        raise TypeError("expected a float64 CUDA tensor")
    return c_void_p(t.data_ptr())


def _vec(t, n, name):
    """The device pointer of a contiguous float64 CUDA vector of exactly n entries (the
    kernels read and write n entries from it, so a shorter or strided view is refused)."""
    p = _ptr(t)
    if not t.is_contiguous() or t.numel() != n:
        raise ValueError(f"{name}: expected a contiguous float64 CUDA vector of {n} entries, got shape "
                         f"{tuple(t.shape)}")
    return p


def _stream(stream):
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return c_void_p(stream.cuda_stream)


def _col_major(t, name):
    """(rows, cols, ld) of a tensor viewed as a column-major panel (columns contiguous)."""
    if t.dim() == 1:
        return t.shape[0], 1, t.shape[0]
    if t.dim() != 2:
        raise ValueError(f"{name}: expected a vector or an (n, k) column-major matrix")
    n, k = t.shape
    if t.stride(0) != 1:
        raise ValueError(f"{name}: columns must be contiguous (use .t().contiguous().t())")
    return n, k, max(t.stride(1), n) if k > 1 else n


class StencilMatrix:
    """Handle of a (2d+1)-point stencil operator (include/sstep.h, operator section)."""

    def __init__(self, dim, shape, coef=None, beta=None, fields=None, beta_field=None, stream=None):
        L = lib()
        h = c_void_p()
        shp = (c_int64 * 3)(*(list(shape) + [1] * (3 - len(shape))))
        if beta_field is not None:
            _check("stencil_matrix_create_convdiff_variable",
                   L.stencil_matrix_create_convdiff_variable(ctypes.byref(h), shape[0],
                                                             _vec(beta_field, shape[0] * shape[0], "beta_field"),
                                                             _stream(stream)))
        elif beta is not None:
            b = (c_double * 3)(*list(beta))
            _check("stencil_matrix_create_convdiff", L.stencil_matrix_create_convdiff(ctypes.byref(h), dim, shp, b))
        elif coef is not None:
            c = (c_double * 7)(*list(coef))
            _check("stencil_matrix_create", L.stencil_matrix_create(ctypes.byref(h), dim, shp, c))
        elif fields is not None:
            npts = 1
            for d in shape:
                npts *= int(d)
            if len(fields) != 2 * dim + 1:
                raise ValueError(f"fields: expected {2 * dim + 1} coefficient arrays")
            ptrs = (c_void_p * 7)(*[_vec(f, npts, "fields").value for f in fields])
            _check("stencil_matrix_create_fields",
                   L.stencil_matrix_create_fields(ctypes.byref(h), dim, shp, ptrs, _stream(stream)))
        else:
            raise ValueError("give coef, beta or fields")
        self.handle = h
        self.dim = dim
        self.shape = tuple(shape)
        n = c_int64()
        ninf = c_double()
        _check("stencil_matrix_info", L.stencil_matrix_info(h, ctypes.byref(n), ctypes.byref(ninf)))
        self.n = n.value
        self.norm_inf = ninf.value

    def close(self):
        if self.handle:
            lib().stencil_matrix_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def apply(self, x, y, stream=None):
        return stencil_matrix_apply(self, x, y, stream)

    def rbilu0_apply(self, v, w, stream=None):
        """w = M^-1 v, M the red-black ILU(0) of this operator."""
        return _check("stencil_matrix_rbilu0_apply",
                      lib().stencil_matrix_rbilu0_apply(self.handle, _vec(v, self.n, "v"), _vec(w, self.n, "w"),
                                                        _stream(stream)))

    def ilu0_apply(self, v, w, stream=None):
        """w = M^-1 v, M the natural-ordering ILU(0) of this operator (the paper's)."""
        return _check("stencil_matrix_ilu0_apply",
                      lib().stencil_matrix_ilu0_apply(self.handle, _vec(v, self.n, "v"), _vec(w, self.n, "w"),
                                                      _stream(stream)))

    def smooth(self, f, x, work, sweeps, omega, stream=None):
        return stencil_matrix_smooth(self, f, x, work, sweeps, omega, stream)


def stencil_matrix_apply(A, x, y, stream=None):
    return _check("stencil_matrix_apply", lib().stencil_matrix_apply(A.handle, _vec(x, A.n, "x"), _vec(y, A.n, "y"),
                                                                     _stream(stream)))


def stencil_matrix_smooth_batched(mats, fs, xs, works, sweeps, omega, stream=None):
    """`sweeps` damped Jacobi sweeps on every x in place, all systems per launch."""
    n = len(mats)
    if not (len(fs) == len(xs) == len(works) == n):
        raise ValueError("one f, x and work vector per matrix")
    arr = lambda ts, nm: (c_void_p * n)(*[_vec(t, A.n, nm).value for t, A in zip(ts, mats)])
    hs = (c_void_p * n)(*[A.handle for A in mats])
    return _check("stencil_matrix_smooth_batched",
                  lib().stencil_matrix_smooth_batched(n, hs, arr(fs, "f"), arr(xs, "x"), arr(works, "work"), int(sweeps),
                                                      float(omega),
                                                      _stream(stream)))


def stencil_matrix_smooth(A, f, x, work, sweeps, omega, stream=None):
    """`sweeps` damped Jacobi sweeps on x in place (work: scratch of n doubles)."""
    return _check("stencil_matrix_smooth", lib().stencil_matrix_smooth(A.handle, _vec(f, A.n, "f"), _vec(x, A.n, "x"),
                                                                       _vec(work, A.n, "work"), int(sweeps),
                                                                       float(omega), _stream(stream)))


def sstep_matrix_powers(A, v, scale, sigma, s, Y, stream=None):
    n, k, ld = _col_major(Y, "Y")
    if k < s + 1:
        raise ValueError("Y needs s+1 columns")
    if n != A.n:
        raise ValueError(f"Y: expected {A.n} rows, got {n}")
    return _check("sstep_matrix_powers",
                  lib().sstep_matrix_powers(A.handle, _vec(v, A.n, "v"), scale, sigma, s, _ptr(Y), ld,
                                            _stream(stream)))


def sstep_gram_workspace_size(n, ka, kb):
    b = c_size_t()
    _check("sstep_gram_workspace_size", lib().sstep_gram_workspace_size(n, ka, kb, ctypes.byref(b)))
    return b.value


def _workspace(nbytes, device):
    import torch

    return torch.empty((nbytes + 255) // 8 + 64, dtype=torch.float64, device=device)


def _aligned_ptr(buf):
    p = buf.data_ptr()
    return c_void_p((p + 255) // 256 * 256)


def sstep_gram(V, Y, C=None, work=None, stream=None):
    """C = V^T Y for column-major panels V (n x ka) and Y (n x kb)."""
    import torch

    n, ka, ldv = _col_major(V, "V")
    n2, kb, ldy = _col_major(Y, "Y")
    assert n == n2
    if C is None:
        C = torch.empty((kb, ka), dtype=torch.float64, device=V.device).t()
    nbytes = sstep_gram_workspace_size(n, ka, kb)
    if work is None:
        work = _workspace(nbytes, V.device)
    _check("sstep_gram", lib().sstep_gram(n, _ptr(V), ldv, ka, _ptr(Y), ldy, kb, c_void_p(C.data_ptr()), ka,
                                          _aligned_ptr(work), nbytes, _stream(stream)))
    return C


def sstep_gram_tc(V, Y, C=None, work=None, stream=None):
    """C = V^T Y on the tensor cores (exact 61-bit fixed point, one rounding per entry)."""
    import torch

    n, ka, ldv = _col_major(V, "V")
    n2, kb, ldy = _col_major(Y, "Y")
    assert n == n2
    if C is None:
        C = torch.empty((kb, ka), dtype=torch.float64, device=V.device).t()
    nbytes = sstep_gram_workspace_size(n, ka, kb)
    if work is None:
        work = _workspace(nbytes, V.device)
    _check("sstep_gram_tc", lib().sstep_gram_tc(n, _ptr(V), ldv, ka, _ptr(Y), ldy, kb, c_void_p(C.data_ptr()), ka,
                                                _aligned_ptr(work), nbytes, _stream(stream)))
    return C


def set_tc_wait_limit(limit):
    """Polls per bounded mbarrier wait of the tensor-core Gram pass (0: none; < 0: the default)."""
    return _check("sstep_set_tc_wait_limit", lib().sstep_set_tc_wait_limit(int(limit)))


def sstep_block_update(V, Y, T, work=None, stream=None, tc=False):
    """In place Y <- Y - V T; returns G = Y^T Y of the updated Y (tc: on the tensor cores,
    sstep_block_update_tc)."""
    import torch

    n, kb, ldy = _col_major(Y, "Y")
    if V is None or V.numel() == 0:
        ka, ldv, vp, tp, ldt = 0, n, c_void_p(0), c_void_p(0), 1
    else:
        n2, ka, ldv = _col_major(V, "V")
        assert n == n2
        vp = _ptr(V)
        Tc = T.t().contiguous().t()
        tp = c_void_p(Tc.data_ptr())
        ldt = Tc.stride(1) if Tc.dim() == 2 and Tc.shape[1] > 1 else ka
        T = Tc
    G = torch.empty((kb, kb), dtype=torch.float64, device=Y.device)
    nbytes = sstep_gram_workspace_size(max(n, 1), 1, kb)
    if work is None:
        work = _workspace(nbytes, Y.device)
    name = "sstep_block_update_tc" if tc else "sstep_block_update"
    _check(name, getattr(lib(), name)(n, vp, ldv, ka, _ptr(Y), ldy, kb, tp, ldt, c_void_p(G.data_ptr()),
                                      _aligned_ptr(work), nbytes, _stream(stream)))
    return G.t()


BASES = {"monomial": 0, "newton": 1, "ortho": 2}
PRECONDS = {None: 0, "none": 0, "rbilu0": 1, "ilu0": 2}


def _solve(name, A, f, x, s=1, m=20, k=1, tol=1e-8, max_cycles=1000, max_iters=100000, sigma=0.0,
           history_cap=4096, stream=None, precision="fp64", x0_guard=False, basis="monomial", precond=None):
    import numpy as np

    hist = np.zeros(max(history_cap, 1), dtype=np.float64)
    p = SStepParams(s=s, m=m, k=k, tol=tol, max_cycles=max_cycles, max_iters=max_iters, sigma=sigma,
                    history=hist.ctypes.data_as(P(c_double)) if history_cap > 0 else None,
                    history_cap=history_cap, precision=PRECISIONS[precision], x0_guard=1 if x0_guard else 0,
                    basis=BASES[basis], precond=PRECONDS[precond])
    r = SStepResult()
    rc = getattr(lib(), name)(A.handle, _vec(f, A.n, "f"), _vec(x, A.n, "x"), ctypes.byref(p), ctypes.byref(r),
                              _stream(stream))
    _check(name, rc)
    return dict(status=r.status, cycles=r.cycles, iters=r.iters, matvecs=r.matvecs, relres=r.relres,
                history=hist[: r.history_len].tolist())


def sstep_gmres_solve(A, f, x, s, m, tol, max_cycles=1000, sigma=0.0, history_cap=4096, stream=None,
                      precision="fp64", x0_guard=False, basis="monomial", precond=None):
    """s-step GMRES (Alg. 4.1/4.2); x is updated in place. Returns the result as a dict
    (with "shifts": the Newton-basis shifts used, empty for the monomial basis).

    precision: "fp64", "df64" (double-float basis) or "fp32" (FP32 basis, FP32 iterative refinement).
    basis: "monomial" (as printed) or "newton" (shifts from the first cycle's Ritz values).
    precond: None, "rbilu0" (right ILU(0) in red-black ordering) or "ilu0" (right ILU(0) in the
    natural ordering, the paper's); FP64 basis.
    """
    r = _solve("sstep_gmres_solve", A, f, x, s=s, m=m, tol=tol, max_cycles=max_cycles, sigma=sigma,
               history_cap=history_cap, stream=stream, precision=precision, x0_guard=x0_guard, basis=basis,
               precond=precond)
    buf = (c_double * SSTEP_MAX_S)()
    cnt = _check("sstep_last_shifts", lib().sstep_last_shifts(A.handle, buf, SSTEP_MAX_S))
    r["shifts"] = list(buf[:cnt])
    return r


def gmres_solve(A, f, x, m, tol, max_cycles=1000, history_cap=4096, stream=None, precision="fp64"):
    """Standard GMRES(m) with classical Gram-Schmidt (Alg. 2.2)."""
    return _solve("gmres_solve", A, f, x, m=m, tol=tol, max_cycles=max_cycles, history_cap=history_cap,
                  stream=stream, precision=precision)


def sstep_omin_solve(A, f, x, s, k, tol, max_iters=100000, sigma=0.0, history_cap=4096, stream=None, precond=None,
                     basis="monomial"):
    """s-step Orthomin(k) (Alg. 3.1); s = 1 is Orthomin(k). precond: None, "rbilu0" or "ilu0".
    basis: "monomial" (as printed) or "ortho" (A^T A-orthonormal direction blocks, Sec. 3)."""
    return _solve("sstep_omin_solve", A, f, x, s=s, k=k, tol=tol, max_iters=max_iters, sigma=sigma,
                  history_cap=history_cap, stream=stream, precond=precond, basis=basis)


def sstep_newton_shifts(G, K, s):
    """The library's Newton-basis shifts for a host Hessenberg matrix G ((>= K) x (>= K),
    float64): the Leja-ordered real parts of the eigenvalues of G[:K, :K] (host only)."""
    import numpy as np

    Gf = np.asfortranarray(np.asarray(G, dtype=np.float64))
    out = (c_double * s)()
    _check("sstep_newton_shifts", lib().sstep_newton_shifts(Gf.ctypes.data_as(P(c_double)), Gf.shape[0], K, s, out))
    return list(out)


def trace_enable(on=True):
    """Turn per-launch CUDA-event tracing on or off (resets the totals)."""
    _check("sstep_trace_enable", lib().sstep_trace_enable(1 if on else 0))


def trace_select(kinds=None):
    """Bracket only the named kernel kinds with events (None: every kind)."""
    L = lib()
    if kinds is None:
        mask = 0xFFFFFFFF
    else:
        names = [L.sstep_trace_kind_name(k).decode() for k in range(L.sstep_trace_kinds())]
        mask = 0
        for nm in kinds:
            mask |= 1 << names.index(nm)
    _check("sstep_trace_select", L.sstep_trace_select(mask))


def trace_read():
    """{kind name: (total milliseconds, launches)} since the last trace_enable()."""
    L = lib()
    out = {}
    for k in range(L.sstep_trace_kinds()):
        ms = c_double()
        nl = c_int64()
        _check("sstep_trace_read", L.sstep_trace_read(k, ctypes.byref(ms), ctypes.byref(nl)))
        out[L.sstep_trace_kind_name(k).decode()] = (ms.value, nl.value)
    return out


def library_build_id():
    """A hash of the kernel sources this package builds libsstep.so from (its csrc files
    and the C header): tuned timings are only valid for the kernels they were taken on."""
    import hashlib

    h = hashlib.sha256()
    csrc = os.path.join(os.path.dirname(os.path.abspath(__file__)), "csrc")
    names = sorted(os.listdir(csrc)) if os.path.isdir(csrc) else []
    for nm in names:
        with open(os.path.join(csrc, nm), "rb") as fh:
            h.update(nm.encode() + b"\0" + fh.read())
    return h.hexdigest()[:16]


def tune_cache_key(shapes, s, m, device, tol=1e-8, sigma=0.0, x0_guard=False, build=None, precision="fp64"):
    """The key of a batch's tuned launch configuration: what the timing depends on. The
    device name, s, m, the tolerance, sigma and the x0 guard (they change the cycle counts),
    the basis precision (another kernel), a hash of the systems' grid shapes in batch order
    and the library build (library_build_id)."""
    import hashlib

    h = hashlib.sha256(repr([tuple(int(v) for v in sh) for sh in shapes]).encode()).hexdigest()[:16]
    b = library_build_id() if build is None else build
    prec = "" if precision == "fp64" else f"|prec={precision}"   # (FP64 keys as before)
    return (f"{device}|s={int(s)}|m={int(m)}|tol={float(tol)!r}|sigma={float(sigma)!r}|guard={int(bool(x0_guard))}"
            f"{prec}|n={len(shapes)}|{h}|build={b}")


def tune_cache_get(path, key):
    """The cached configuration for key, or None (no file, no entry, or an unreadable file)."""
    import json

    try:
        with open(path) as fh:
            cfg = json.load(fh).get(key)
    except (OSError, ValueError, AttributeError):
        return None
    names = ("threads", "ctas_per_sm", "largest_first", "cluster", "coop_min_n")
    if not isinstance(cfg, dict) or any(not isinstance(cfg.get(k), int) for k in names):
        return None
    return {k: cfg[k] for k in names}


def tune_cache_put(path, key, cfg):
    """Adds (or replaces) key's configuration, rewriting the file atomically. The
    read-modify-write holds an exclusive lock on path + ".lock", so processes that write
    at the same time keep each other's entries."""
    import fcntl
    import json

    with open(path + ".lock", "a") as lk:
        fcntl.flock(lk, fcntl.LOCK_EX)
        try:
            try:
                with open(path) as fh:
                    data = json.load(fh)
                if not isinstance(data, dict):
                    data = {}
            except (OSError, ValueError):
                data = {}
            data[key] = dict(cfg)
            tmp = f"{path}.{os.getpid()}.tmp"
            with open(tmp, "w") as fh:
                json.dump(data, fh, indent=1, sort_keys=True)
            os.replace(tmp, path)
        finally:
            fcntl.flock(lk, fcntl.LOCK_UN)


def _f64(t, count, name):
    """Pointer of a contiguous float64 CUDA tensor of `count` elements."""
    import torch

    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous() \
            or t.numel() != count:
        raise TypeError(f"{name}: expected a contiguous float64 CUDA tensor of {count} elements")
    return c_void_p(t.data_ptr())


def x0net_features(H, W, f, beta, stream=None):
    """The learned form's inputs, on the device: f and beta (B, H*W float64 CUDA) ->
    (features (B, 2, H, W) float32 = (f / s_f, beta / 20), f_scale (B,) float64 = s_f)."""
    import torch

    B = f.shape[0]
    inp = torch.empty((B, 2, H, W), dtype=torch.float32, device=f.device)
    sf = torch.empty(B, dtype=torch.float64, device=f.device)
    _check("x0net_features", lib().x0net_features(H, W, B, _f64(f, B * H * W, "f"), _f64(beta, B * H * W, "beta"),
                                                   c_void_p(inp.data_ptr()), c_void_p(sf.data_ptr()), _stream(stream)))
    return inp, sf


def x0net_targets(H, W, x, f_scale, stream=None):
    """Training targets x / (kappa s_f) (B, 1, H, W) float32 from solutions x (B, H*W float64)."""
    import torch

    B = x.shape[0]
    t = torch.empty((B, 1, H, W), dtype=torch.float32, device=x.device)
    _check("x0net_targets", lib().x0net_targets(H, W, B, _f64(x, B * H * W, "x"), _f64(f_scale, B, "f_scale"),
                                                 c_void_p(t.data_ptr()), _stream(stream)))
    return t


class BatchSolver:
    """Batched s-step GMRES over many systems (include/sstep.h, batched solves).

    mats: list of StencilMatrix (kept alive by this object). solve() takes lists of
    float64 CUDA tensors f and x (x in/out) and returns one result dict per system.
    """

    PERSISTENT = 0
    PER_SYSTEM = 1

    def __init__(self, mats, s, m, tol, max_cycles=1000, sigma=0.0, x0_guard=False, precision="fp64"):
        """precision: "fp64" (FP64 basis) or "fp32" (FP32 basis, double-float sums, FP64
        residual, x and scalar work: FP32 iterative refinement per system)."""
        if precision not in ("fp64", "fp32"):
            raise ValueError("precision: fp64 or fp32")
        self.mats = list(mats)
        self.n = len(self.mats)
        self.s, self.m = s, m
        self.tol, self.sigma, self.x0_guard, self.precision = tol, sigma, bool(x0_guard), precision
        h = c_void_p()
        arr = (c_void_p * self.n)(*[A.handle.value for A in self.mats])
        p = SStepParams(s=s, m=m, k=0, tol=tol, max_cycles=max_cycles, max_iters=0, sigma=sigma, history=None,
                        history_cap=0, precision=PRECISIONS[precision], x0_guard=1 if x0_guard else 0)
        _check("sstep_batch_create", lib().sstep_batch_create(ctypes.byref(h), self.n, arr, ctypes.byref(p)))
        self.handle = h

    def _ptrs(self, ts, name):
        if len(ts) != self.n:
            raise ValueError(f"{name}: expected {self.n} vectors, one per system")
        return (c_void_p * self.n)(*[_vec(t, A.n, name).value for t, A in zip(ts, self.mats)])

    def solve(self, f, x, mode=0, stream=None):
        res = (SStepResult * self.n)()
        _check("sstep_batch_solve", lib().sstep_batch_solve(self.handle, self._ptrs(f, "f"), self._ptrs(x, "x"), res, mode,
                                                            _stream(stream)))
        return [dict(status=r.status, cycles=r.cycles, iters=r.iters, matvecs=r.matvecs, relres=r.relres) for r in res]

    def tune(self, f, x, stream=None, cache=None):
        """Time the launch configurations on this batch and keep the fastest (the initial
        guesses are restored). cache: a JSON file (default: $SSTEP_TUNE_CACHE, if set) of
        earlier results, keyed by the device and the batch's shape (tune_cache_key); a hit
        configures without timing."""
        cache = cache if cache is not None else os.environ.get("SSTEP_TUNE_CACHE")
        key = None
        if cache:
            import torch

            key = tune_cache_key([A.shape for A in self.mats], self.s, self.m, torch.cuda.get_device_name(),
                                 tol=self.tol, sigma=self.sigma, x0_guard=self.x0_guard, precision=self.precision)
            hit = tune_cache_get(cache, key)
            if hit is not None:
                self.configure(**hit)
                return dict(hit)
        t, c, o, g, nb = c_int(), c_int(), c_int(), c_int(), c_int64()
        _check("sstep_batch_tune", lib().sstep_batch_tune(self.handle, self._ptrs(f, "f"), self._ptrs(x, "x"), ctypes.byref(t),
                                                          ctypes.byref(c), ctypes.byref(o), ctypes.byref(g),
                                                          ctypes.byref(nb), _stream(stream)))
        cfg = dict(threads=t.value, ctas_per_sm=c.value, largest_first=o.value, cluster=g.value,
                   coop_min_n=nb.value)
        if key is not None:
            tune_cache_put(cache, key, cfg)
        return cfg

    def configure(self, threads=256, ctas_per_sm=1, largest_first=1, cluster=1, coop_min_n=0):
        """Set the launch configuration by hand (what tune() would choose)."""
        _check("sstep_batch_configure", lib().sstep_batch_configure(self.handle, threads, ctas_per_sm, largest_first,
                                                                    cluster, coop_min_n))

    def close(self):
        if self.handle:
            lib().sstep_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class X0Net:
    """The learned-initial-guess U-Net (include/sstep.h, learned initial guess).

    Tensors are float32 CUDA tensors: input (B, 2, H, W), output/target (B, 1, H, W).
    """

    def __init__(self, H, W, batch_max, bf16=True, smooth=4, residual_weight=0.0, kappa=1.0):
        h = c_void_p()
        _check("x0net_create", lib().x0net_create(ctypes.byref(h), H, W, batch_max, 1 if bf16 else 0, smooth))
        _check("x0net_set_residual_weight", lib().x0net_set_residual_weight(h, residual_weight, kappa))
        self.handle = h
        n = c_int64()
        _check("x0net_num_params", lib().x0net_num_params(h, ctypes.byref(n)))
        self.num_params = n.value
        self.H, self.W = H, W

    @staticmethod
    def _f32(t):
        import torch

        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
            raise TypeError("expected a contiguous float32 CUDA tensor")
        return c_void_p(t.data_ptr())

    def _io(self, inp, other, name):
        """Pointers of an input (B, 2, H, W) and an output or target (B, 1, H, W) batch."""
        pi, po = self._f32(inp), self._f32(other)
        B = inp.shape[0] if inp.dim() == 4 else -1
        if tuple(inp.shape) != (B, 2, self.H, self.W) or tuple(other.shape) != (B, 1, self.H, self.W):
            raise ValueError(f"expected input (B, 2, {self.H}, {self.W}) and {name} (B, 1, {self.H}, {self.W}), got "
                             f"{tuple(inp.shape)} and {tuple(other.shape)}")
        return pi, po

    def set_params(self, theta, stream=None):
        import torch

        t = torch.as_tensor(theta, dtype=torch.float32).contiguous()
        if not t.is_cuda:
            t = t.cuda()
        _check("x0net_set_params", lib().x0net_set_params(self.handle, c_void_p(t.data_ptr()), _stream(stream)))
        torch.cuda.current_stream().synchronize()

    def get_params(self, stream=None):
        import numpy as np

        out = np.zeros(self.num_params, dtype=np.float32)
        _check("x0net_get_params", lib().x0net_get_params(self.handle, c_void_p(out.ctypes.data), _stream(stream)))
        return out

    def get_state(self, stream=None):
        """The training state: dict(params, m, v) float32 host arrays and step (Adam)."""
        import numpy as np

        st = {k: np.zeros(self.num_params, dtype=np.float32) for k in ("params", "m", "v")}
        step = c_int64()
        _check("x0net_get_state", lib().x0net_get_state(self.handle, c_void_p(st["params"].ctypes.data),
                                                        c_void_p(st["m"].ctypes.data), c_void_p(st["v"].ctypes.data),
                                                        ctypes.byref(step), _stream(stream)))
        st["step"] = int(step.value)
        return st

    def set_state(self, state, stream=None):
        """Restores a state from get_state (or a checkpoint file's contents)."""
        import numpy as np

        arr = {k: np.ascontiguousarray(state[k], dtype=np.float32) for k in ("params", "m", "v")}
        if any(a.shape != (self.num_params,) for a in arr.values()):
            raise ValueError("state arrays must hold num_params floats each")
        _check("x0net_set_state", lib().x0net_set_state(self.handle, c_void_p(arr["params"].ctypes.data),
                                                        c_void_p(arr["m"].ctypes.data), c_void_p(arr["v"].ctypes.data),
                                                        int(state["step"]), _stream(stream)))

    def forward(self, inp, out, stream=None):
        pi, po = self._io(inp, out, "output")
        _check("x0net_forward", lib().x0net_forward(self.handle, pi, po, inp.shape[0],
                                                    _stream(stream)))

    def predict(self, inp, f_scale, x0, stream=None):
        """x0 (B, H*W float64 CUDA) = kappa s_f * the network's output for input (B, 2, H, W):
        the initial guesses (x0net_predict)."""
        pi = self._f32(inp)
        B = inp.shape[0]
        if tuple(inp.shape) != (B, 2, self.H, self.W):
            raise ValueError(f"expected input (B, 2, {self.H}, {self.W}), got {tuple(inp.shape)}")
        _check("x0net_predict", lib().x0net_predict(self.handle, pi, _f64(f_scale, B, "f_scale"),
                                                    B, _f64(x0, B * self.H * self.W, "x0"), _stream(stream)))

    def gradient(self, inp, target, stream=None):
        import numpy as np

        g = np.zeros(self.num_params, dtype=np.float32)
        loss = np.zeros(1, dtype=np.float32)
        pi, pt = self._io(inp, target, "target")
        _check("x0net_gradient", lib().x0net_gradient(self.handle, pi, pt, inp.shape[0],
                                                      c_void_p(loss.ctypes.data), c_void_p(g.ctypes.data),
                                                      _stream(stream)))
        return float(loss[0]), g

    def train_step(self, inp, target, lr, loss_out=None, stream=None):
        lp = self._f32(loss_out) if loss_out is not None else c_void_p(0)
        pi, pt = self._io(inp, target, "target")
        _check("x0net_train_step", lib().x0net_train_step(self.handle, pi, pt, inp.shape[0],
                                                          lr, lp, _stream(stream)))

    def set_tensor_cores(self, on):
        """BF16 mode: 3x3 convolutions on the tensor cores (default) or on the CUDA cores."""
        _check("x0net_set_tensor_cores", lib().x0net_set_tensor_cores(self.handle, 1 if on else 0))

    def set_wait_limit(self, polls):
        """Polls per bounded tensor-core wait (negative: the default); tests set 0."""
        _check("x0net_set_wait_limit", lib().x0net_set_wait_limit(self.handle, int(polls)))

    def status(self, stream=None):
        """Synchronises and raises if a tensor-core kernel's bounded wait ran out."""
        _check("x0net_status", lib().x0net_status(self.handle, _stream(stream)))

    def close(self):
        if self.handle:
            lib().x0net_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
