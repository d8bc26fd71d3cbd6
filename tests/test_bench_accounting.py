"""The bench's work accounting (the numerator of the reported roofline) against the
oracle's own counts, on the CPU.

bench.py reads the Krylov steps of each restart cycle off the solve's residual
history and charges every kernel kind its algorithmic flops and bytes per block; the
oracle counts the same solve's cycles, steps and products independently.
"""
import numpy as np
import pytest

import bench
from oracle import sstep, stencil
from paper_2001_04886_gb300 import inputs


@pytest.mark.parametrize("s,m,tol", [(4, 20, 1e-8), (8, 40, 1e-8), (2, 10, 1e-10), (8, 16, 1e-6)])
def test_cycle_steps_and_work_match_the_oracle(s, m, tol):
    A = stencil.convdiff((12, 12, 12), (30.0, 20.0, 10.0))
    f = A.apply(inputs.x_true(0, A.n))
    r = sstep.sstep_gmres(A, f, np.zeros(A.n), s, m, tol, 1.0 / A.norm_inf(), 500)
    assert r["status"] == 0
    steps = bench.cycle_steps(r["history"], s, m, tol)
    assert len(steps) == r["cycles"] and sum(steps) == r["iters"]
    assert all(k % s == 0 and 0 < k <= m for k in steps)
    W = bench.sstep_gmres_work(A.n, 3, s, m, r["history"], tol)
    # every Krylov step is one product of 7 multiply-adds per point
    assert W["stencil_powers"][0] == r["iters"] * 14 * A.n
    # products: the steps, plus one explicit residual per restart and the final one
    assert r["matvecs"] == r["iters"] + r["cycles"] + 1
    # block k of a cycle projects s columns on k s earlier ones (Gram and update alike)
    proj = sum(2 * (k * s) * s * A.n for c in steps for k in range(c // s))
    assert W["gram"][0] == proj
    assert W["block_update"][0] == proj + sum(c // s for c in steps) * (s + 1) * (s + 2) * A.n
    assert W["basis_axpy"][0] == 2 * r["iters"] * A.n
