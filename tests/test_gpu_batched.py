"""Batched persistent s-step GMRES against the oracle, system by system.

The batch mixes uneven sizes and convection coefficients as the batched
workload does (sides from a range, beta ~ U[0, 50]), at sizes the oracle solves
quickly. Each system must reach the oracle's solution (relative 1e-8) with the
same number of restart cycles; the persistent launch and the one-solve-per-
system launches must agree.
"""
import numpy as np
import pytest

from oracle import sstep as osstep
from oracle import stencil as ostencil
from paper_2001_04886_gb300 import inputs
from tests.gpu_util import dev, to_dev, torch

import paper_2001_04886_gb300 as pkg

pytestmark = pytest.mark.gpu


def batch(seed, count, lmin, lmax, d):
    systems = inputs.batched_systems(seed, count, lmin, lmax)
    mats, ora, fs, xs = [], [], [], []
    for sy in systems:
        L, beta = sy["L"], sy["beta"]
        Ao = ostencil.convdiff((L, L), (beta, beta))
        f = Ao.apply(inputs.x_true(sy["xseed"], Ao.n))
        mats.append(pkg.StencilMatrix(2, (L, L), beta=(beta, beta)))
        ora.append((Ao, f))
        fs.append(to_dev(f, d))
        xs.append(torch.zeros(Ao.n, dtype=torch.float64, device=d))
    return mats, ora, fs, xs


@pytest.mark.parametrize("s,m", [(4, 20), (8, 16), (1, 10)])
def test_persistent_batch_matches_oracle(s, m):
    d = dev()
    mats, ora, fs, xs = batch(3, 24, 6, 40, d)
    B = pkg.BatchSolver(mats, s, m, 1e-8, max_cycles=400)
    res = B.solve(fs, xs, mode=B.PERSISTENT)
    torch.cuda.synchronize()
    for i, ((Ao, f), r) in enumerate(zip(ora, res)):
        ref = osstep.sstep_gmres(Ao, f, np.zeros(Ao.n), s, m, 1e-8, 1.0 / Ao.norm_inf(), 400)
        x = xs[i].cpu().numpy()
        assert r["status"] == 0 and ref["status"] == 0, (i, r)
        assert r["cycles"] == ref["cycles"], (i, r["cycles"], ref["cycles"])
        assert np.linalg.norm(x - ref["x"]) <= 1e-8 * np.linalg.norm(ref["x"]), i
        assert np.linalg.norm(f - Ao.apply(x)) <= 1e-8 * np.linalg.norm(f)


def test_persistent_equals_per_system_and_tuning():
    d = dev()
    mats, ora, fs, xs = batch(11, 40, 16, 64, d)
    xs2 = [torch.zeros_like(x) for x in xs]
    B = pkg.BatchSolver(mats, 4, 20, 1e-8)
    cfg = B.tune(fs, xs)
    assert cfg["threads"] in (128, 256) and cfg["ctas_per_sm"] in (1, 2, 4)
    assert all(float(x.abs().max()) == 0.0 for x in xs)     # tuning restores the initial guesses
    r1 = B.solve(fs, xs, mode=B.PERSISTENT)
    r2 = B.solve(fs, xs2, mode=B.PER_SYSTEM)
    torch.cuda.synchronize()
    for i in range(len(xs)):
        assert r1[i]["status"] == r2[i]["status"] == 0
        assert r1[i]["cycles"] == r2[i]["cycles"]
        a, b = xs[i].cpu().numpy(), xs2[i].cpu().numpy()
        assert np.linalg.norm(a - b) <= 1e-9 * np.linalg.norm(b)
