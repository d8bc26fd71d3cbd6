"""The fixed-point digit arithmetic of the tensor-core Gram pass, on the CPU.

The library's helpers (csrc/ozaki.cuh) are compiled for the host with a small emulation
driver (tests/ozaki_emulation.cpp). They are checked against exact rational arithmetic:
the digits reconstruct the 53-bit fixed-point value of every entry, and the emulated
Gram matrix is within the error bound stated for sstep_gram_tc of the exact V^T Y. A
coarser digit cut, planted on purpose, breaks that bound.
"""
import ctypes
import os
import shutil
import subprocess
import tempfile
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2001_04886_gb300", "csrc")


@pytest.fixture(scope="module")
def emu():
    cxx = shutil.which("g++")
    if not cxx:
        pytest.skip("g++ not available")
    d = tempfile.mkdtemp(prefix="ozemu_")
    so = os.path.join(d, "libozemu.so")
    r = subprocess.run([cxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-I", CSRC,
                        os.path.join(ROOT, "tests", "ozaki_emulation.cpp"), "-o", so], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    L = ctypes.CDLL(so)
    dp = ctypes.POINTER(ctypes.c_double)
    L.oz_bound.restype = ctypes.c_uint32
    L.oz_bound.argtypes = [dp, ctypes.c_int64]
    L.oz_digits.argtypes = [dp, ctypes.c_int64, ctypes.c_uint32, ctypes.POINTER(ctypes.c_int)]
    L.oz_gram.argtypes = [ctypes.c_int64, dp, ctypes.c_int, dp, ctypes.c_int, ctypes.c_int, dp]
    yield L
    shutil.rmtree(d, ignore_errors=True)


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def gram(L, V, Y, cut=8):
    n, ka = V.shape
    kb = Y.shape[1]
    Vc = np.asfortranarray(V)
    Yc = np.asfortranarray(Y)
    C = np.zeros(ka * kb)
    L.oz_gram(n, _p(Vc), ka, _p(Yc), kb, cut, _p(C))
    return C.reshape(kb, ka).T


def bound_exp(x):
    """ex_max from the definition: the largest biased exponent field over the column."""
    e = 0
    for v in x:
        bits = np.float64(v).view(np.uint64)
        e = max(e, int(bits >> np.uint64(52)) & 0x7FF)
    return e


def sample_columns(rng, n):
    """Columns with the spreads the solver meets: uniform, smooth, decaying over 30
    binades, one spike, exact zeros, and a column of subnormals next to normal values."""
    t = np.linspace(0, 1, n)
    cols = [rng.uniform(-1, 1, n), np.sin(7 * t) * 3e-5, rng.standard_normal(n) * 2.0 ** (-30 * t),
            np.where(np.arange(n) == n // 3, 1e8, rng.uniform(-1, 1, n)), np.zeros(n)]
    c = rng.uniform(-1, 1, n)
    c[::7] = 5e-320
    cols.append(c)
    return np.array(cols).T


def test_digits_reconstruct_the_fixed_point_value(emu):
    """q = trunc(x 2^(1083 - ex_max)) exactly, from the eight balanced digits, for every entry."""
    rng = np.random.default_rng(0)
    X = sample_columns(rng, 257)
    for j in range(X.shape[1]):
        x = np.ascontiguousarray(X[:, j])
        ex = emu.oz_bound(_p(x), len(x))
        assert ex == bound_exp(x)
        dig = (ctypes.c_int * (8 * len(x)))()
        emu.oz_digits(_p(x), len(x), ex, dig)
        d = np.array(dig[:], dtype=np.int64).reshape(-1, 8)
        assert d.min() >= -128 and d.max() <= 127 and np.abs(d[:, 0]).max() <= 32
        for i, v in enumerate(x):
            num, den = Fraction(float(v)).as_integer_ratio()
            if (int(np.float64(v).view(np.uint64) >> np.uint64(52)) & 0x7FF) == 0:
                want = 0   # zero and subnormal entries count as 0
            else:
                scaled = Fraction(num, den) * Fraction(2) ** (1083 - ex)
                want = int(scaled)   # truncation toward zero
            got = sum(int(d[i, t]) * 256 ** (7 - t) for t in range(8))
            assert got == want, (j, i, v)


def exact_gram(V, Y):
    ka, kb = V.shape[1], Y.shape[1]
    C = np.empty((ka, kb), dtype=object)
    Vf = [[Fraction(float(v)) for v in V[:, a]] for a in range(ka)]
    Yf = [[Fraction(float(v)) for v in Y[:, b]] for b in range(kb)]
    for a in range(ka):
        for b in range(kb):
            C[a, b] = sum(p * q for p, q in zip(Vf[a], Yf[b]))
    return C


def error_bound(V, Y):
    """The stated bound: 2^-65 sum(Bv By) + 2^-60 sum(Bv |y| + |v| By) plus the final rounding,
    Bv = 2^(ex_max(v) - 1022) the column's power-of-two bound, plus the products that involve
    a subnormal entry (those entries count as zero)."""
    ka, kb = V.shape[1], Y.shape[1]
    n = V.shape[0]
    bv = [2.0 ** (bound_exp(V[:, a]) - 1022) for a in range(ka)]
    by = [2.0 ** (bound_exp(Y[:, b]) - 1022) for b in range(kb)]
    B = np.empty((ka, kb), dtype=object)
    sub = lambda v: Fraction(abs(float(v))) if abs(v) < 2.0 ** -1022 else Fraction(0)
    for a in range(ka):
        for b in range(kb):
            main = (2.0 ** -65 * n * bv[a] * by[b]
                    + 2.0 ** -60 * (bv[a] * np.abs(Y[:, b]).sum() + np.abs(V[:, a]).sum() * by[b])) * (1 + 2.0 ** -40)
            tiny = sum(sub(v) * abs(Fraction(float(y))) + abs(Fraction(float(v))) * sub(y) for v, y in zip(V[:, a], Y[:, b]))
            B[a, b] = Fraction(float(main)) + tiny
    return B


@pytest.mark.parametrize("n", [1, 63, 1000])
def test_emulated_gram_within_the_stated_bound(emu, n):
    rng = np.random.default_rng(n)
    V = sample_columns(rng, n)
    Y = np.concatenate([sample_columns(rng, n)[:, :3], rng.uniform(-1, 1, (n, 2)) * 1e-3], axis=1)
    C = gram(emu, V, Y)
    ex = exact_gram(V, Y)
    B = error_bound(V, Y)
    for a in range(V.shape[1]):
        for b in range(Y.shape[1]):
            err = abs(Fraction(float(C[a, b])) - ex[a, b])
            assert err <= B[a, b] + abs(ex[a, b]) * Fraction(2) ** -53, (a, b)


def test_emulated_gram_matches_fp64_to_1e14_of_the_column_norms(emu):
    """The parity bar of the Gram entries: 1e-14 of the product of the column norms."""
    rng = np.random.default_rng(5)
    V = rng.uniform(-1, 1, (4000, 6)) * np.array([1, 1e-3, 1e5, 3e-7, 1, 1])
    Y = rng.standard_normal((4000, 4))
    C = gram(emu, V, Y)
    ex = exact_gram(V, Y)
    nrm = np.outer(np.linalg.norm(V, axis=0), np.linalg.norm(Y, axis=0))
    err = np.array([[float(abs(Fraction(float(C[a, b])) - ex[a, b])) for b in range(4)] for a in range(6)])
    assert np.all(err <= 1e-14 * nrm)


def test_spiky_columns_meet_1e14_of_the_column_norms(emu):
    """One large entry among small ones makes the column bound far exceed most entries; the
    dropped pairs and the truncation, measured against the bound, must still stay below
    1e-14 of the product of the column norms over thousands of rows."""
    rng = np.random.default_rng(7)
    n = 5000
    V = rng.uniform(-1, 1, (n, 3))
    Y = rng.uniform(-1, 1, (n, 3))
    V[n // 2, :] = 1e6
    Y[n // 2, :] = 1e6
    Y[:, 2] *= 1e-7
    C = gram(emu, V, Y)
    ex = exact_gram(V, Y)
    nrm = np.outer(np.linalg.norm(V, axis=0), np.linalg.norm(Y, axis=0))
    err = np.array([[float(abs(Fraction(float(C[a, b])) - ex[a, b])) for b in range(3)] for a in range(3)])
    assert np.all(err <= 1e-14 * nrm)


def test_nonfinite_column_gives_nan(emu):
    V = np.ones((10, 2))
    V[3, 1] = np.inf
    Y = np.ones((10, 1))
    C = gram(emu, V, Y)
    assert np.isfinite(C[0, 0]) and np.isnan(C[1, 0]) and C[0, 0] == 10.0


def test_planted_coarse_cut_breaks_the_bound(emu):
    """Keeping only the digit pairs with t_a + t_b <= 6 (a planted slip) leaves errors far
    above the stated bound, so the bound test would catch a wrong cut."""
    rng = np.random.default_rng(9)
    V = rng.uniform(-1, 1, (500, 2))
    Y = rng.uniform(-1, 1, (500, 2))
    ex = exact_gram(V, Y)
    B = error_bound(V, Y)
    C = gram(emu, V, Y, cut=6)
    assert any(abs(Fraction(float(C[a, b])) - ex[a, b]) > B[a, b] for a in range(2) for b in range(2))


def test_integer_rounding_equals_fp64_rounding(emu):
    """The integer-only rounding of a 128-bit integer times 2^e2 (the kernels' epilogue)
    gives the same double as the reference rounding, and that one is the correctly
    rounded value (checked with exact rationals), on ties, carries and random values."""
    emu.oz_round_both.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    rng = np.random.default_rng(4)
    cases = []
    for v in [1, -1, 2 ** 53 + 1, 2 ** 53 + 3, (2 ** 53 - 1) * 2 ** 11 + 2 ** 10, (2 ** 53 - 1) * 2 ** 11 + 2 ** 10 + 1,
              2 ** 120 + 2 ** 67, -(2 ** 100) - 2 ** 47, 2 ** 126 - 1, -(2 ** 126) + 12345]:
        cases.append(v)
    for _ in range(300):
        bits = int(rng.integers(1, 126))
        v = int(rng.integers(0, 2 ** 62)) * 2 ** max(0, bits - 62) + int(rng.integers(0, 2 ** 30))
        cases.append(v if rng.random() < 0.5 else -v)
    out = (ctypes.c_double * 2)()
    for v in cases:
        for e2 in (-1100, -200, 0, 37):
            u = v % (1 << 128)
            emu.oz_round_both(u >> 64, u & ((1 << 64) - 1), e2, out)
            exact = Fraction(v) * Fraction(2) ** e2
            assert out[0] == out[1], (v, e2)
            assert out[0] == float(exact), (v, e2)   # Python's float() of a Fraction rounds correctly


def test_word_form_equals_64_bit_form(emu):
    """The kernels' 32-bit-word fixed-point conversion equals the 64-bit definition for
    every entry: signs, zeros, subnormals, entries at the bound and far below it."""
    emu.oz_biased_both.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.c_int64, ctypes.c_uint32,
                                   ctypes.POINTER(ctypes.c_uint64)]
    rng = np.random.default_rng(7)
    x = np.concatenate([rng.standard_normal(4000) * np.exp2(rng.integers(-80, 8, 4000)),
                        [0.0, -0.0, 5e-324, -5e-324, 2.2e-308, 1.0, -1.0, 0.5, np.nextafter(2.0, 0.0), -1.9999999]])
    out = np.zeros(2 * x.size, dtype=np.uint64)
    for ex in (1023, 1024, 1030, 1100, 1500, 2000):
        m = np.abs(x) < np.exp2(ex - 1022)          # entries within the bound of this exponent
        xs = np.ascontiguousarray(x[m])
        o = np.zeros(2 * xs.size, dtype=np.uint64)
        emu.oz_biased_both(_p(xs), xs.size, ex, o.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))
        assert np.array_equal(o[0::2], o[1::2]), ex
