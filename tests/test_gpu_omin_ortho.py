"""s-step Orthomin with A^T A-orthonormal direction blocks (Sec. 3) on the GPU.

The library orthonormalises each new block with the triangular factor of its
predicted Gram matrix, folded into the block update; the oracle uses modified
Gram-Schmidt as the paper says. Both give the same blocks in exact arithmetic, so
the library must reach the oracle's step count, products and solution. The
residual histories of the first steps agree to max(1e-10, 100 u cond(A R_0^T A R_0)):
the two orthonormalisations round differently, by about u times the condition of
the raw block they orthonormalise.
"""
import numpy as np
import pytest

from oracle import sstep as osstep
from oracle import stencil as ostencil
from paper_2001_04886_gb300 import inputs
from tests.gpu_util import dev, to_dev, torch

import paper_2001_04886_gb300 as pkg

pytestmark = pytest.mark.gpu

U53 = 2.0 ** -53


def raw_block_condition(Ao, f, s, sigma):
    R, AR = osstep.omin_powers(Ao, f, s, sigma)
    return float(np.linalg.cond(AR.T @ AR))


def compare(res, ref, Ao, f, x, nfirst, hist_tol, tol):
    assert res["status"] == ref["status"] == 0
    assert (res["iters"], res["matvecs"]) == (ref["iters"], ref["matvecs"])
    h, hr = np.array(res["history"]), np.array(ref["history"])
    assert len(h) == len(hr)
    assert np.max(np.abs(h[: nfirst + 1] - hr[: nfirst + 1]) / hr[: nfirst + 1]) <= hist_tol
    assert np.linalg.norm(x - ref["x"]) <= 1e-8 * np.linalg.norm(ref["x"])
    assert np.linalg.norm(f - Ao.apply(x)) <= tol * np.linalg.norm(f)


@pytest.mark.parametrize("shape,beta,s,k", [
    ((64, 64), (20.0, 20.0), 4, 1),
    ((64, 64), (20.0, 20.0), 1, 2),     # Orthomin(2) with normalised directions
    ((32, 32), (20.0, 20.0), 2, 2),
    ((32, 32), (20.0, 20.0), 3, 0),     # s-MR
    ((16, 16, 16), (30.0, 20.0, 10.0), 4, 1),
    ((16, 16, 16), (30.0, 20.0, 10.0), 8, 1),
    ((20, 20, 20), (30.0, 20.0, 10.0), 8, 7),   # (k + 1) s = 64: the largest window
])
def test_ortho_omin_matches_oracle(shape, beta, s, k):
    d = dev()
    Ao = ostencil.convdiff(shape, beta)
    f = Ao.apply(inputs.x_true(0, Ao.n))
    A = pkg.StencilMatrix(len(shape), shape, beta=beta)
    sigma = 1.0 / Ao.norm_inf()
    ref = osstep.sstep_omin(Ao, f, np.zeros(Ao.n), s, k, 1e-8, sigma, 20000, basis="ortho")
    xd = torch.zeros(Ao.n, dtype=torch.float64, device=d)
    res = pkg.sstep_omin_solve(A, to_dev(f, d), xd, s, k, 1e-8, max_iters=20000, sigma=sigma, basis="ortho")
    hist_tol = max(1e-10, 100 * U53 * raw_block_condition(Ao, f, s, sigma))
    compare(res, ref, Ao, f, xd.cpu().numpy(), 4, hist_tol, 1e-8)


def test_ortho_is_the_same_method_as_the_printed_form():
    """Same spans, so the library's two forms take the same steps to the same x."""
    d = dev()
    Ao = ostencil.convdiff((48, 48), (20.0, 10.0))
    f = Ao.apply(inputs.x_true(3, Ao.n))
    A = pkg.StencilMatrix(2, (48, 48), beta=(20.0, 10.0))
    fd = to_dev(f, d)
    xa = torch.zeros(Ao.n, dtype=torch.float64, device=d)
    xb = torch.zeros_like(xa)
    a = pkg.sstep_omin_solve(A, fd, xa, 4, 2, 1e-9)
    b = pkg.sstep_omin_solve(A, fd, xb, 4, 2, 1e-9, basis="ortho")
    assert a["status"] == b["status"] == 0 and a["iters"] == b["iters"]
    ha, hb = np.array(a["history"]), np.array(b["history"])
    assert np.all(np.abs(ha - hb) <= 1e-7 * ha + 1e-14)
    assert float(torch.linalg.norm(xa - xb)) <= 1e-8 * float(torch.linalg.norm(xa))


@pytest.mark.parametrize("s", [4, 8])
def test_ortho_on_the_paper_problem(s):
    """The Sec. 5 problem from the paper's initial guess, without and with the red-black
    ILU(0) right preconditioner: the oracle's steps and solution."""
    d = dev()
    N = 64
    P = inputs.paper_problem(N)
    a0, aw, ae, as_, an = P["coef"]
    Ao = ostencil.Stencil((N, N), a0, [aw, as_], [ae, an])
    A = pkg.StencilMatrix(2, (N, N), fields=[to_dev(c, d) for c in P["coef"]])
    g = P["g"]
    for pre in (None, "rbilu0"):
        sigma = 1.0 if pre else 1.0 / Ao.norm_inf()
        M = ostencil.RedBlackILU0(Ao) if pre else None
        ref = osstep.sstep_omin(Ao, g, P["x0"], s, 1, 1e-9, sigma, 20000, precond=M, basis="ortho")
        xd = to_dev(P["x0"], d)
        res = pkg.sstep_omin_solve(A, to_dev(g, d), xd, s, 1, 1e-9, max_iters=20000, sigma=sigma, precond=pre,
                                   basis="ortho")
        torch.cuda.synchronize()
        x = xd.cpu().numpy()
        assert res["status"] == ref["status"] == 0, pre
        assert (res["iters"], res["matvecs"]) == (ref["iters"], ref["matvecs"]), pre
        assert np.linalg.norm(x - ref["x"]) <= 1e-8 * np.linalg.norm(ref["x"]), pre
        assert np.linalg.norm(g - Ao.apply(x)) <= 1e-9 * np.linalg.norm(g), pre


def test_ortho_argument_errors():
    d = dev()
    A = pkg.StencilMatrix(2, (16, 16), beta=(20.0, 20.0))
    f = torch.ones(A.n, dtype=torch.float64, device=d)
    x = torch.zeros_like(f)
    with pytest.raises(pkg.SStepError):
        pkg.sstep_omin_solve(A, f, x, 8, 8, 1e-8, basis="ortho")      # (k + 1) s = 72 > 64
    with pytest.raises(pkg.SStepError):
        pkg.sstep_omin_solve(A, f, x, 4, 1, 1e-8, basis="newton")     # GMRES only
    with pytest.raises(pkg.SStepError):
        pkg.sstep_gmres_solve(A, f, x, 4, 20, 1e-8, basis="ortho")    # Orthomin only
    assert pkg.sstep_omin_solve(A, f, x, 8, 8, 1e-8)["status"] in (0, 1)   # k s = 64 stays valid printed
