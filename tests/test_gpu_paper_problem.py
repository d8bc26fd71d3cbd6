"""The paper's test problem (Sec. 5) on the GPU: the library (variable-coefficient
stencil, red-black ILU(0), s-step GMRES s = 2, m = 10, the paper's initial guess)
against the oracle on the same system, and the discretisation error against the
analytic solution at the second order that the CPU pins establish."""
import numpy as np
import pytest

from oracle import dense
from oracle import sstep as osstep
from oracle import stencil as ostencil
from paper_2001_04886_gb300 import inputs
from tests.gpu_util import dev, to_dev, torch

import paper_2001_04886_gb300 as pkg

pytestmark = pytest.mark.gpu


def operator(P, N):
    a0, aw, ae, as_, an = P["coef"]
    return ostencil.Stencil((N, N), a0, [aw, as_], [ae, an])


@pytest.mark.parametrize("s,m,precond", [(2, 10, "rbilu0"), (1, 10, "rbilu0"), (2, 10, None)])
def test_paper_problem_matches_oracle_and_converges_at_second_order(s, m, precond):
    d = dev()
    N = 64
    P = inputs.paper_problem(N)
    Ao = operator(P, N)
    A = pkg.StencilMatrix(2, (N, N), fields=[to_dev(c, d) for c in P["coef"]])
    xd = to_dev(P["x0"], d)
    r = pkg.sstep_gmres_solve(A, to_dev(P["g"], d), xd, s, m, 1e-10, max_cycles=5000, precond=precond)
    torch.cuda.synchronize()
    M = ostencil.RedBlackILU0(Ao) if precond else None
    sigma = 1.0 if precond else 1.0 / Ao.norm_inf()
    ref = osstep.sstep_gmres(Ao, P["g"], P["x0"], s, m, 1e-10, sigma, 5000, precond=M)
    x = xd.cpu().numpy()
    assert r["status"] == 0 and ref["status"] == 0
    assert r["cycles"] == ref["cycles"] and r["matvecs"] == ref["matvecs"]
    assert np.linalg.norm(x - ref["x"]) <= 1e-8 * np.linalg.norm(ref["x"])
    # discretisation error: C h^2 with C from a dense solve on the 31^2 grid
    P31 = inputs.paper_problem(31)
    e31 = np.max(np.abs(np.linalg.solve(dense.dense_matrix(operator(P31, 31)), P31["g"]) - P31["u"]))
    predicted = e31 * (32.0 / 65.0) ** 2
    err = np.max(np.abs(x - P["u"]))
    assert 0.5 * predicted <= err <= 1.5 * predicted, (err, predicted)
