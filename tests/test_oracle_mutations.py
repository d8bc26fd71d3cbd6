"""Planted mistakes in the oracle must be caught by its pins.

Each case copies one oracle module's source, applies a one-line slip (a dropped
term, a wrong sign or index, a transposed operand), loads the copy as a
separate module and runs the relevant pin on it. The real oracle is untouched.
"""
import importlib.util
import os

import numpy as np
import pytest

import oracle
import oracle.sstep  # noqa: F401  (oracle.sstep is used through the package below)
from oracle import dense, krylov, stencil
from paper_2001_04886_gb300 import inputs

ORACLE_DIR = os.path.dirname(oracle.__file__)


def mutated(modname, old, new):
    src = open(os.path.join(ORACLE_DIR, modname + ".py")).read()
    assert src.count(old) >= 1, old
    src = src.replace(old, new, 1)
    spec = importlib.util.spec_from_loader("oracle._mut_" + modname, loader=None)
    mod = importlib.util.module_from_spec(spec)
    mod.__package__ = "oracle"
    exec(compile(src, modname + "_mut.py", "exec"), mod.__dict__)
    return mod


def brute_force_ok(solve):
    A = stencil.convdiff((4, 4), (20.0, 20.0))
    f = A.apply(inputs.x_true(0, A.n))
    xs = dense.gauss_solve(dense.dense_matrix(A), f)
    try:
        res = solve(A, f)
    except Exception:
        return False
    return res["status"] == 0 and np.linalg.norm(res["x"] - xs) <= 1e-10 * np.linalg.norm(xs)


SSTEP_MUTATIONS = [
    ("col = col / sigma", "col = col"),                                  # dropped 1/sigma in eq. 4
    ("col[:o] = T[:, j + 1]", "col[:o] = T[:, j]"),                      # wrong power index
    ("col = col - G[:, :o] @ T[:, j]", "col = col + G[:, :o] @ T[:, j]"),  # wrong sign
    ("u = Yh[:, s] - Yh[:, :s] @ S", "u = Yh[:, s]"),                    # dropped in-block projection
    ("C = inner_products(U[:, :o], Y[:, 1:])", "C = inner_products(U[:, :o], Y[:, :-1])"),  # shifted powers
    ("lg[rows] = Ls[i] @ G[rows, c]", "lg[rows] = Ls[i].T @ G[rows, c]"),  # transposed factor
]


def sstep_pins_hold(mod):
    """P4 (history equals GMRES(m) over two cycles) and P7 (A V = U G) on a 16x16 system.

    Restarted methods recompute the true residual at every restart, so many
    slips still converge to the right x; the step-by-step history and the
    Arnoldi relation are what expose them.
    """
    A = stencil.convdiff((16, 16), (20.0, 20.0))
    f = A.apply(inputs.x_true(0, A.n))
    z = np.zeros(A.n)
    m = 8
    ref = krylov.gmres(A, f, z, m, 1e-30, 2)["history"]
    for s in (2, 4):
        try:
            tr = {}
            h = mod.sstep_gmres(A, f, z, s, m, 1e-30, 0.125, 2, trace=tr)["history"]
        except Exception:
            return False
        if len(h) != len(ref) or np.max(np.abs(np.array(h) - ref) / np.array(ref)) > 1e-8:
            return False
        U, G = tr["U"], tr["G"]
        AV = np.column_stack([A.apply(U[:, j]) for j in range(G.shape[1])])
        if np.linalg.norm(AV - U @ G) > 1e-10 * np.linalg.norm(AV):
            return False
    return True


def test_sstep_pins_hold_for_real_oracle():
    assert sstep_pins_hold(oracle.sstep)


@pytest.mark.parametrize("old,new", SSTEP_MUTATIONS)
def test_sstep_gmres_mutation_caught(old, new):
    assert not sstep_pins_hold(mutated("sstep", old, new))


OMIN_MUTATIONS = [
    ("B = -_omin_solve(Ls[j], C, ortho)", "B = _omin_solve(Ls[j], C, ortho)"),  # wrong sign of Scalar2
    ("C = AP[j].T @ AR", "C = AR.T @ AP[j]"),                            # transposed C_j
    ("Pn = Pn + P[j] @ B", "Pn = Pn + P[j] @ B.T"),                      # transposed coefficients
    ("x = x + P[-1] @ a", "x = x + P[-1] @ a[::-1]"),                    # wrong column order
]


@pytest.mark.parametrize("old,new", OMIN_MUTATIONS)
def test_sstep_omin_mutation_caught(old, new):
    mod = mutated("sstep", old, new)
    A = stencil.convdiff((16, 16), (20.0, 20.0))
    f = A.apply(inputs.x_true(0, A.n))
    good = oracle.sstep.sstep_omin(A, f, np.zeros(A.n), 3, 1, 1e-9, 0.125, 300)
    try:
        bad = mod.sstep_omin(A, f, np.zeros(A.n), 3, 1, 1e-9, 0.125, 300)
    except Exception:
        return
    # a slip either changes the residual history (A^T A-orthogonality, P7) or
    # leaves x inconsistent with r, which the brute-force solve (P3) exposes
    n = min(len(good["history"]), len(bad["history"]), 20)
    hist_moved = np.max(np.abs(np.array(good["history"][:n]) - bad["history"][:n]) / np.array(good["history"][:n])) > 1e-6
    assert hist_moved or not brute_force_ok(lambda A_, f_: mod.sstep_omin(A_, f_, np.zeros(A_.n), 3, 1, 1e-13, 0.125, 400))


def test_stencil_transposed_caught():
    mod = mutated("stencil", "return Stencil(shape, 2.0 * dim, [-1.0 - cd for cd in c], [-1.0 + cd for cd in c])",
                  "return Stencil(shape, 2.0 * dim, [-1.0 + cd for cd in c], [-1.0 - cd for cd in c])")
    from tests.test_oracle_stencil import test_quadratic_closed_form
    import tests.test_oracle_stencil as ts
    saved = ts.stencil
    ts.stencil = mod
    try:
        with pytest.raises(AssertionError):
            test_quadratic_closed_form((9, 9), (20.0, -7.0))
    finally:
        ts.stencil = saved


def test_gmres_window_and_orth_mutations_caught():
    # a dropped projection: CGS no longer matches the modified Gram-Schmidt cross-check
    mod = mutated("krylov", "w = w - Q[:, : j + 1] @ h", "w = w - Q[:, :j] @ h[:j]")
    A = stencil.convdiff((16, 16), (20.0, 20.0))
    f = A.apply(inputs.x_true(0, A.n))
    for m_, ok in [(mod, False), (krylov, True)]:
        a = np.array(m_.gmres(A, f, np.zeros(A.n), 8, 1e-30, 2)["history"])
        b = np.array(krylov.gmres(A, f, np.zeros(A.n), 8, 1e-30, 2, orth="mgs")["history"])
        assert (np.max(np.abs(a - b) / b) < 1e-9) == ok
    mod = mutated("krylov", "lo = len(P) - min(k, len(P))", "lo = len(P) - 1")
    A = stencil.convdiff((14, 14), (20.0, 20.0))
    f = A.apply(inputs.x_true(0, A.n))
    gcr = mod.omin(A, f, np.zeros(A.n), 10_000, 1e-10, 30)
    gm = krylov.gmres(A, f, np.zeros(A.n), 60, 1e-10, 1)
    a = np.array(gcr["history"][1:25])
    b = np.array(gm["history"][1:25])
    assert np.max(np.abs(a - b) / b) > 1e-6


PRECOND_MUTATIONS = [
    ("dt -= coef_b * self._shift(coef_r / a0.reshape(sh), ax, step).reshape(-1)",
     "dt += coef_b * self._shift(coef_r / a0.reshape(sh), ax, step).reshape(-1)"),   # wrong sign of the fill
    ("s += (am * self._shift(W, ax, -1) + ap * self._shift(W, ax, +1)).reshape(-1)",
     "s += (am * self._shift(W, ax, +1) + ap * self._shift(W, ax, -1)).reshape(-1)"),  # swapped neighbours
    ("out.append((ax, self._mask(am, ax, -1).reshape(-1), ap, -1))",
     "out.append((ax, self._mask(am, ax, +1).reshape(-1), ap, -1))"),                 # wrong boundary mask
    ("w = np.where(self.black, (v - t) / self.dtilde, 0.0)",
     "w = np.where(self.black, (v - t) / self.a0, 0.0)"),                              # unmodified pivot
]


@pytest.mark.parametrize("old,new", PRECOND_MUTATIONS)
def test_precond_mutation_caught(old, new):
    """The red-black ILU(0) pins (L U equals A on its pattern, M^-1 equals the dense solve
    with L U) catch each planted slip."""
    mod = mutated("stencil", old, new)
    from tests.test_oracle_precond import dense_factors

    A = mod.convdiff((4, 4, 4), (30.0, 20.0, 10.0))
    P = mod.RedBlackILU0(A)
    Ap, L, U, perm = dense_factors(A, P)
    LU = L @ U
    pat = Ap != 0
    on_pattern = np.max(np.abs((LU - Ap)[pat])) <= 1e-14 * np.max(np.abs(Ap))
    v = inputs.x_true(3, A.n)
    want = np.zeros(A.n)
    want[perm] = np.linalg.solve(LU, v[perm])
    applies = np.max(np.abs(P.apply_inv(v) - want)) <= 1e-13 * np.max(np.abs(want))
    assert not (on_pattern and applies)
