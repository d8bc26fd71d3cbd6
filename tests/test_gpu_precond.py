"""Red-black ILU(0) right preconditioning on the GPU against the oracle: the
preconditioner application element by element, and preconditioned s-step GMRES
(monomial and Newton bases) with the oracle's cycles, products, history and solution."""
import numpy as np
import pytest

from oracle import sstep as osstep
from oracle import stencil as ostencil
from paper_2001_04886_gb300 import inputs
from tests.gpu_util import dev, to_dev, torch
from tests.parity_bars import first_block_tol

import paper_2001_04886_gb300 as pkg

pytestmark = pytest.mark.gpu


def pair(shape, beta):
    d = dev()
    dim = len(shape)
    if len(set(shape)) == 1:
        return d, ostencil.convdiff(shape, beta), pkg.StencilMatrix(dim, shape, beta=beta)
    h = 1.0 / (shape[0] + 1)
    c = [b * h / 2 for b in beta]
    coef = [2.0 * dim]
    for cd in c:
        coef += [-1.0 - cd, -1.0 + cd]
    return d, ostencil.Stencil(shape, coef[0], coef[1::2], coef[2::2]), pkg.StencilMatrix(dim, shape, coef=coef)


@pytest.mark.parametrize("shape,beta", [((24, 24, 24), (30.0, 20.0, 10.0)), ((37, 29), (20.0, -13.0)),
                                        ((17, 9, 5), (30.0, 20.0, 10.0)), ((1, 1), (5.0, 5.0))])
def test_rbilu0_apply_matches_oracle(shape, beta):
    d, Ao, A = pair(shape, beta)
    v = inputs.x_true(7, Ao.n)
    w = torch.empty(Ao.n, dtype=torch.float64, device=d)
    A.rbilu0_apply(to_dev(v, d), w)
    torch.cuda.synchronize()
    ref = ostencil.RedBlackILU0(Ao).apply_inv(v)
    assert np.max(np.abs(w.cpu().numpy() - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_rbilu0_apply_variable_coefficients():
    d = dev()
    N = 33
    bfield, _ = inputs.fourier_fields(2, N)
    Ao = ostencil.convdiff_variable(N, bfield)
    A = pkg.StencilMatrix(2, (N, N), beta_field=to_dev(bfield, d))
    v = inputs.x_true(8, Ao.n)
    w = torch.empty(Ao.n, dtype=torch.float64, device=d)
    A.rbilu0_apply(to_dev(v, d), w)
    torch.cuda.synchronize()
    ref = ostencil.RedBlackILU0(Ao).apply_inv(v)
    assert np.max(np.abs(w.cpu().numpy() - ref)) <= 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("shape,beta,s,m,basis", [((24, 24, 24), (30.0, 20.0, 10.0), 4, 20, "monomial"),
                                                  ((64, 64), (20.0, 20.0), 4, 20, "monomial"),
                                                  ((24, 24, 24), (30.0, 20.0, 10.0), 8, 40, "newton"),
                                                  ((37, 29), (20.0, -13.0), 2, 10, "monomial")])
def test_preconditioned_solve_matches_oracle(shape, beta, s, m, basis):
    d, Ao, A = pair(shape, beta)
    f = Ao.apply(inputs.x_true(0, Ao.n))
    P = ostencil.RedBlackILU0(Ao)
    xd = torch.zeros(Ao.n, dtype=torch.float64, device=d)
    r = pkg.sstep_gmres_solve(A, to_dev(f, d), xd, s, m, 1e-8, max_cycles=400, precond="rbilu0", basis=basis)
    torch.cuda.synchronize()
    rule = (lambda G, K, s_: list(r["shifts"])) if r["shifts"] else None
    ref = osstep.sstep_gmres(Ao, f, np.zeros(Ao.n), s, m, 1e-8, 1.0, 400, precond=P, basis=basis, shift_rule=rule)
    x = xd.cpu().numpy()
    assert r["status"] == 0 and ref["status"] == 0
    assert r["cycles"] == ref["cycles"] and r["matvecs"] == ref["matvecs"] and r["iters"] == ref["iters"]
    # first s estimates: implementations that round W_1 differently differ by a few
    # u cond(W_1) (the monomial first block of A M^-1; at s = 8 cond ~ 1e10)
    tr = {}
    osstep.sstep_gmres(Ao, f, np.zeros(Ao.n), s, m, 1e-30, 1.0, 1, trace=tr, precond=P)
    htol = first_block_tol(np.linalg.cond(tr["W"][0]))
    h, hr = np.array(r["history"][1 : s + 1]), np.array(ref["history"][1 : s + 1])
    assert np.max(np.abs(h - hr) / hr) <= htol
    # the solution: to 1e-8, or to u cond(W_1) when the first block is worse conditioned
    # (its rounding moves the first cycle's correction, which is most of x, by that much)
    assert np.linalg.norm(x - ref["x"]) <= max(1e-8, htol) * np.linalg.norm(ref["x"])
    assert np.linalg.norm(f - Ao.apply(x)) <= 1e-8 * np.linalg.norm(f)
    # fewer products than the unpreconditioned solve
    x0 = torch.zeros_like(xd)
    r0 = pkg.sstep_gmres_solve(A, to_dev(f, d), x0, s, m, 1e-8, max_cycles=400)
    assert r["matvecs"] < r0["matvecs"]


def test_preconditioner_argument_errors():
    d, Ao, A = pair((12, 12), (10.0, 10.0))
    f = to_dev(Ao.apply(inputs.x_true(1, Ao.n)), d)
    x = torch.zeros_like(f)
    for kw in (dict(precision="df64"), dict(precision="fp32")):
        with pytest.raises(pkg.SStepError):
            pkg.sstep_gmres_solve(A, f, x, 4, 20, 1e-8, precond="rbilu0", **kw)
    with pytest.raises(pkg.SStepError):
        A.rbilu0_apply(f, f)


@pytest.mark.parametrize("s,k", [(1, 4), (2, 2), (4, 1)])
def test_preconditioned_orthomin_matches_oracle(s, k):
    """Right-preconditioned (s-step) Orthomin on the paper's test problem from its
    initial guess: the oracle's step count, products and solution."""
    d = dev()
    N = 48
    P = inputs.paper_problem(N)
    a0, aw, ae, as_, an = P["coef"]
    Ao = ostencil.Stencil((N, N), a0, [aw, as_], [ae, an])
    A = pkg.StencilMatrix(2, (N, N), fields=[to_dev(c, d) for c in P["coef"]])
    xd = to_dev(P["x0"], d)
    r = pkg.sstep_omin_solve(A, to_dev(P["g"], d), xd, s, k, 1e-9, max_iters=20000, precond="rbilu0")
    torch.cuda.synchronize()
    ref = osstep.sstep_omin(Ao, P["g"], P["x0"], s, k, 1e-9, 1.0, 20000, precond=ostencil.RedBlackILU0(Ao))
    x = xd.cpu().numpy()
    assert r["status"] == 0 and ref["status"] == 0
    assert r["iters"] == ref["iters"] and r["matvecs"] == ref["matvecs"]
    assert np.linalg.norm(x - ref["x"]) <= 1e-8 * np.linalg.norm(ref["x"])
    assert np.linalg.norm(P["g"] - Ao.apply(x)) <= 1e-9 * np.linalg.norm(P["g"])
