"""ILU(0) in the natural ordering (the paper's right preconditioner, Sec. 5) on the GPU
against the oracle: the factors and M^-1 v bit for bit (the library sweeps hyperplanes
with the oracle's operations in the oracle's order), and preconditioned s-step GMRES and
s-step Orthomin with the oracle's cycles, products, history and solution."""
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


def paper_pair(N):
    d = dev()
    P = inputs.paper_problem(N)
    a0, aw, ae, as_, an = P["coef"]
    Ao = ostencil.Stencil((N, N), a0, [aw, as_], [ae, an])
    return d, Ao, pkg.StencilMatrix(2, (N, N), fields=[to_dev(c, d) for c in P["coef"]]), P


@pytest.mark.parametrize("shape,beta", [((37, 29), (20.0, -13.0)), ((64, 64), (20.0, 20.0)), ((1, 1), (5.0, 5.0)),
                                        ((40, 1), (20.0, 0.0)), ((9, 7, 5), (30.0, 20.0, 10.0)),
                                        ((16, 16, 16), (30.0, 20.0, 10.0)), ((1, 6, 3), (0.0, 20.0, 10.0))])
def test_ilu0_apply_equals_oracle_bit_for_bit(shape, beta):
    d, Ao, A = pair(shape, beta)
    v = inputs.x_true(7, Ao.n)
    w = torch.empty(Ao.n, dtype=torch.float64, device=d)
    A.ilu0_apply(to_dev(v, d), w)
    w2 = torch.empty_like(w)
    A.ilu0_apply(to_dev(v, d), w2)   # factors kept from the first call
    torch.cuda.synchronize()
    ref = ostencil.NaturalILU0(Ao).apply_inv(v)
    assert np.array_equal(w.cpu().numpy(), ref)
    assert np.array_equal(w2.cpu().numpy(), ref)


def test_ilu0_apply_paper_problem_bit_for_bit():
    d, Ao, A, P = paper_pair(64)
    v = inputs.x_true(9, Ao.n)
    w = torch.empty(Ao.n, dtype=torch.float64, device=d)
    A.ilu0_apply(to_dev(v, d), w)
    torch.cuda.synchronize()
    assert np.array_equal(w.cpu().numpy(), ostencil.NaturalILU0(Ao).apply_inv(v))


def test_ilu0_apply_rejects_in_place():
    d, Ao, A = pair((8, 8), (10.0, 10.0))
    v = to_dev(inputs.x_true(1, Ao.n), d)
    with pytest.raises(pkg.SStepError):
        A.ilu0_apply(v, v)


@pytest.mark.parametrize("N,s,m,basis", [(32, 1, 10, "monomial"), (32, 2, 10, "monomial"), (48, 4, 20, "monomial"),
                                         (48, 4, 20, "newton")])
def test_preconditioned_gmres_matches_oracle(N, s, m, basis):
    """Right-preconditioned (s-step) GMRES on the paper's test problem from its initial
    guess (Table 6.1's settings at s = 1, 2): the oracle's cycles, products, history and
    solution."""
    d, Ao, A, P = paper_pair(N)
    xd = to_dev(P["x0"], d)
    r = pkg.sstep_gmres_solve(A, to_dev(P["g"], d), xd, s, m, 1e-8, max_cycles=2000, precond="ilu0", basis=basis)
    torch.cuda.synchronize()
    rule = (lambda G, K, s_: list(r["shifts"])) if r["shifts"] else None
    M = ostencil.NaturalILU0(Ao)
    ref = osstep.sstep_gmres(Ao, P["g"], P["x0"], s, m, 1e-8, 1.0, 2000, precond=M, basis=basis, shift_rule=rule)
    x = xd.cpu().numpy()
    assert r["status"] == 0 and ref["status"] == 0
    assert (r["cycles"], r["iters"], r["matvecs"]) == (ref["cycles"], ref["iters"], ref["matvecs"])
    tr = {}
    osstep.sstep_gmres(Ao, P["g"], P["x0"], s, m, 1e-30, 1.0, 1, trace=tr, precond=M)
    htol = first_block_tol(np.linalg.cond(tr["W"][0]))
    h, hr = np.array(r["history"][1 : s + 1]), np.array(ref["history"][1 : s + 1])
    assert np.max(np.abs(h - hr) / hr) <= htol
    assert np.linalg.norm(x - ref["x"]) <= max(1e-8, htol) * np.linalg.norm(ref["x"])
    assert np.linalg.norm(P["g"] - Ao.apply(x)) <= 1e-8 * np.linalg.norm(P["g"])


@pytest.mark.parametrize("s,k", [(1, 4), (2, 2)])
def test_preconditioned_orthomin_matches_oracle(s, k):
    d, Ao, A, P = paper_pair(32)
    xd = to_dev(P["x0"], d)
    r = pkg.sstep_omin_solve(A, to_dev(P["g"], d), xd, s, k, 1e-9, max_iters=20000, precond="ilu0")
    torch.cuda.synchronize()
    ref = osstep.sstep_omin(Ao, P["g"], P["x0"], s, k, 1e-9, 1.0, 20000, precond=ostencil.NaturalILU0(Ao))
    x = xd.cpu().numpy()
    assert r["status"] == 0 and ref["status"] == 0
    assert r["iters"] == ref["iters"] and r["matvecs"] == ref["matvecs"]
    assert np.linalg.norm(x - ref["x"]) <= 1e-8 * np.linalg.norm(ref["x"])


def test_natural_ordering_takes_fewer_products_than_red_black():
    """The paper's ordering is the stronger preconditioner on its own problem."""
    d, Ao, A, P = paper_pair(64)
    out = {}
    for pc in ("ilu0", "rbilu0"):
        xd = to_dev(P["x0"], d)
        out[pc] = pkg.sstep_gmres_solve(A, to_dev(P["g"], d), xd, 2, 10, 1e-8, max_cycles=2000, precond=pc)
    assert out["ilu0"]["status"] == out["rbilu0"]["status"] == 0
    assert out["ilu0"]["matvecs"] < out["rbilu0"]["matvecs"]
