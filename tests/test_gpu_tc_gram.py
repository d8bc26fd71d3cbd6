"""The tensor-core Gram pass (sstep_gram_tc) against the oracle and against the exact
host emulation of its own fixed-point arithmetic.

Bars: every entry within 1e-14 of the product of the two column norms of the oracle's
FP64 inner products (the parity bar of the Gram pass), equal bit for bit to the host
emulation (every sum is an exact integer, rounded once, so no reduction order enters),
and bitwise reproducible from call to call.
"""
import ctypes
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

from oracle import sstep as osstep
from paper_2001_04886_gb300 import inputs
from tests.gpu_util import dev, to_dev, torch

import paper_2001_04886_gb300 as pkg

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def emu():
    cxx = shutil.which("g++")
    if not cxx:
        pytest.skip("g++ not available")
    d = tempfile.mkdtemp(prefix="ozemu_")
    so = os.path.join(d, "libozemu.so")
    r = subprocess.run([cxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-I",
                        os.path.join(ROOT, "paper_2001_04886_gb300", "csrc"),
                        os.path.join(ROOT, "tests", "ozaki_emulation.cpp"), "-o", so], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    L = ctypes.CDLL(so)
    dp = ctypes.POINTER(ctypes.c_double)
    L.oz_gram.argtypes = [ctypes.c_int64, dp, ctypes.c_int, dp, ctypes.c_int, ctypes.c_int, dp]
    yield L
    shutil.rmtree(d, ignore_errors=True)


def emulate(L, V, Y):
    Vc, Yc = np.asfortranarray(V), np.asfortranarray(Y)
    C = np.zeros(V.shape[1] * Y.shape[1])
    p = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    L.oz_gram(V.shape[0], p(Vc), V.shape[1], p(Yc), Y.shape[1], 8, p(C))
    return C.reshape(Y.shape[1], V.shape[1]).T


def panel(A, d, ld=None):
    """Column-major device panel of A with leading dimension ld (default: the row count)."""
    n, k = A.shape
    ld = ld or n
    buf = torch.zeros((k, ld), dtype=torch.float64, device=d)
    buf[:, :n] = torch.tensor(A.T, dtype=torch.float64, device=d)
    return buf.t()[:n]


def spread_columns(n, k, seed):
    """Columns of different scales and spreads: uniform, decaying over 40 binades, smooth,
    one large spike, and an all-zero column."""
    rng = np.random.default_rng(seed)
    t = np.linspace(0, 1, n)
    cols = []
    for j in range(k):
        kind = j % 5
        if kind == 0:
            c = inputs.x_true(1000 * seed + j, n)
        elif kind == 1:
            c = rng.standard_normal(n) * 2.0 ** (-40 * t) * 10.0 ** (j % 7 - 3)
        elif kind == 2:
            c = np.sin((j + 1) * 3 * t) * 1e-4
        elif kind == 3:
            c = rng.uniform(-1, 1, n)
            c[n // 2] = 1e6
        else:
            c = np.zeros(n) if j == 4 else rng.uniform(-1, 1, n) * 1e-9
        cols.append(c)
    return np.stack(cols, axis=1)


def check(V, Y, C):
    ref = osstep.inner_products(V, Y)
    scale = np.outer(np.linalg.norm(V, axis=0), np.linalg.norm(Y, axis=0))
    scale[scale == 0] = 1.0
    assert np.max(np.abs(C - ref) / scale) <= 1e-14


@pytest.mark.parametrize("n,ka,kb", [(4096, 8, 8), (5000, 32, 9), (1, 1, 1), (63, 3, 2), (1025, 33, 5),
                                     (3000, 64, 9), (2047, 17, 1)])
def test_tc_gram_matches_oracle_and_emulation(emu, n, ka, kb):
    d = dev()
    V = spread_columns(n, ka, 1)
    Y = spread_columns(n, kb, 2)
    Vd, Yd = panel(V, d), panel(Y, d)
    C = pkg.sstep_gram_tc(Vd, Yd)
    C2 = pkg.sstep_gram_tc(Vd, Yd)
    torch.cuda.synchronize()
    got = C.cpu().numpy()
    check(V, Y, got)
    assert np.array_equal(got, emulate(emu, V, Y))        # exact integer sums: bit for bit
    assert np.array_equal(got, C2.cpu().numpy())


@pytest.mark.parametrize("n,ka,kb,ld", [(300001, 33, 9, 300001), (2_097_152, 32, 8, 2_097_152), (100003, 8, 9, 100010)])
def test_tc_gram_large_and_ragged(n, ka, kb, ld):
    """Many chunks of 1024 rows, an odd leading dimension (unaligned columns) and the
    headline block shape at 128^3 (32 earlier columns against 8 powers)."""
    d = dev()
    V = np.stack([inputs.x_true(10 + i, n) for i in range(ka)], axis=1)
    Y = np.stack([inputs.x_true(100 + j, n) * 10.0 ** (j % 5 - 2) for j in range(kb)], axis=1)
    C = pkg.sstep_gram_tc(panel(V, d, ld), panel(Y, d, ld))
    torch.cuda.synchronize()
    check(V, Y, C.cpu().numpy())


def test_tc_gram_symmetric_bit_for_bit():
    """V^T V from exact integer sums is symmetric bit for bit (an FP64 sum need not be)."""
    d = dev()
    n = 200000
    V = np.stack([inputs.x_true(40 + i, n) * 3.0 ** i for i in range(8)], axis=1)
    P = panel(V, d)
    G = pkg.sstep_gram_tc(P, P).cpu().numpy()               # one panel: each column split once
    G2 = pkg.sstep_gram_tc(P, panel(V, d)).cpu().numpy()    # two panels: V and Y split apart
    assert np.array_equal(G, G.T) and np.array_equal(G, G2)
    check(V, V, G)


@pytest.mark.parametrize("n", [1, 113, 9077, 153216, 300001, 2_097_152])
def test_tc_gram_symmetric_nine_columns(emu, n):
    """The 9-column V^T V of the s-step block at s = 8 (its own kernel form, loads three
    stages ahead): bit for bit the same as V and Y split apart, and as the exact emulation.
    The sizes give CTAs of one stage, whole chunks of 9 stages only (153216 = 152 x 9 x 112
    rows) and partial last chunks."""
    d = dev()
    V = spread_columns(n, 9, 3)
    P = panel(V, d)
    G = pkg.sstep_gram_tc(P, P).cpu().numpy()
    G2 = pkg.sstep_gram_tc(P, panel(V, d)).cpu().numpy()
    assert np.array_equal(G, G2) and np.array_equal(G, G.T)
    if n <= 300001:
        assert np.array_equal(G, emulate(emu, V, V))
    check(V, V, G)


def test_tc_gram_symmetric_nine_columns_wait_timeout():
    """The bounded waits of the 9-column form: a poll limit of 0 gives NaN and a normal
    end; the next call with the default limit is exact."""
    d = dev()
    V = spread_columns(300001, 9, 4)
    P = panel(V, d)
    try:
        pkg.set_tc_wait_limit(0)
        bad = pkg.sstep_gram_tc(P, P)
        torch.cuda.synchronize()
        bad = bad.cpu().numpy()
    finally:
        pkg.set_tc_wait_limit(-1)
    assert np.all(np.isnan(bad))
    check(V, V, pkg.sstep_gram_tc(P, P).cpu().numpy())


def test_tc_gram_nonfinite_and_zero():
    d = dev()
    n = 3000
    V = np.stack([inputs.x_true(1, n), np.zeros(n), inputs.x_true(2, n)], axis=1)
    V[17, 2] = np.nan
    Y = np.stack([inputs.x_true(3, n)], axis=1)
    C = pkg.sstep_gram_tc(panel(V, d), panel(Y, d)).cpu().numpy()
    assert np.isfinite(C[0, 0]) and C[1, 0] == 0.0 and np.isnan(C[2, 0])
    check(V[:, :2], Y, C[:2])


def test_tc_gram_n_zero_leaves_padding():
    """n = 0 writes the ka x kb entries only (C = 0), not the rows below ka."""
    import ctypes as ct

    d = dev()
    C = torch.full((3, 4), 7.0, dtype=torch.float64, device=d)   # 3 columns, leading dimension 4
    dummy = torch.zeros(8, dtype=torch.float64, device=d)
    nbytes = pkg.sstep_gram_workspace_size(0, 2, 3)
    work = torch.zeros(nbytes // 8 + 64, dtype=torch.float64, device=d)
    wp = ct.c_void_p((work.data_ptr() + 255) // 256 * 256)
    rc = pkg.lib().sstep_gram_tc(0, ct.c_void_p(dummy.data_ptr()), 0, 2, ct.c_void_p(dummy.data_ptr()), 0, 3,
                                 ct.c_void_p(C.data_ptr()), 4, wp, nbytes, None)
    assert rc == 0
    torch.cuda.synchronize()
    c = C.cpu().numpy()   # c[j, i] = row i of column j
    assert np.all(c[:, :2] == 0.0) and np.all(c[:, 2:] == 7.0)


def test_tc_gram_wait_timeout_gives_nan_and_recovers():
    """A bounded mbarrier wait that runs out (a poll limit of 0: every wait gives up at once)
    makes the result NaN and the kernel still ends normally; with the default limit the
    next call is exact."""
    d = dev()
    n = 50000
    V = np.stack([inputs.x_true(60 + i, n) for i in range(16)], axis=1)
    Y = np.stack([inputs.x_true(70 + j, n) for j in range(4)], axis=1)
    Vd, Yd = panel(V, d), panel(Y, d)
    try:
        pkg.set_tc_wait_limit(0)
        C = pkg.sstep_gram_tc(Vd, Yd)
        torch.cuda.synchronize()
        bad = C.cpu().numpy()
    finally:
        pkg.set_tc_wait_limit(-1)
    assert np.all(np.isnan(bad))
    C = pkg.sstep_gram_tc(Vd, Yd)
    torch.cuda.synchronize()
    check(V, Y, C.cpu().numpy())


# ------------------------------------------------------------------ block update on the tensor cores
@pytest.mark.parametrize("n,ka,kb", [(4096, 12, 5), (5000, 0, 3), (300001, 32, 9), (31, 3, 2), (1, 1, 1),
                                     (130, 16, 8), (2_097_152, 32, 9), (4099, 13, 8), (50000, 27, 4), (777, 17, 9)])
def test_tc_block_update_matches_oracle(n, ka, kb):
    """Y <- Y - V T and G = Y^T Y on the tensor cores against the oracle's block update:
    every updated column to 1e-14 relative (the FP64 kernel's bar) and G to 1e-14 of the
    product of the column norms."""
    from tests.gpu_util import relerr

    d = dev()
    V = np.stack([inputs.x_true(20 + i, n) * 2.0 ** (i % 7 - 3) for i in range(ka)], axis=1) if ka else np.zeros((n, 0))
    Y = np.stack([inputs.x_true(200 + j, n) for j in range(kb)], axis=1)
    T = np.stack([inputs.x_true(300 + j, ka) * 10.0 ** (j % 4 - 2) for j in range(kb)], axis=1) if ka else np.zeros((0, kb))
    Yd = panel(Y, d)
    G = pkg.sstep_block_update(panel(V, d) if ka else None, Yd, to_dev(T, d) if ka else None, tc=True)
    torch.cuda.synchronize()
    Yh, Gr = osstep.block_update(Y, V, T)
    got = Yd.cpu().numpy()
    for j in range(kb):
        assert relerr(got[:, j], Yh[:, j]) <= 1e-14, j
    nrm = np.linalg.norm(Yh, axis=0)
    assert np.max(np.abs(G.cpu().numpy() - Gr) / np.outer(nrm, nrm)) <= 1e-14


def test_tc_block_update_cancellation():
    """Y almost in the span of V (the s-step projection at large s): the updated columns are
    tiny against Y, and their error against the oracle is still at the FP64 level of Y."""
    d = dev()
    n, ka, kb = 100000, 16, 9
    V = np.stack([inputs.x_true(500 + i, n) for i in range(ka)], axis=1)
    T = np.stack([inputs.x_true(600 + j, ka) for j in range(kb)], axis=1)
    Y = V @ T + 1e-9 * np.stack([inputs.x_true(700 + j, n) for j in range(kb)], axis=1)
    Yd = panel(Y, d)
    pkg.sstep_block_update(panel(V, d), Yd, to_dev(T, d), tc=True)
    torch.cuda.synchronize()
    Yh, _ = osstep.block_update(Y, V, T)
    got = Yd.cpu().numpy()
    for j in range(kb):
        assert np.linalg.norm(got[:, j] - Yh[:, j]) <= 1e-15 * 8 * np.linalg.norm(Y[:, j]), j
