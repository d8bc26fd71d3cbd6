"""The first-block history bar of the GPU parity tests holds for the oracle's own rounding.

The oracle's first restart cycle is run twice on the same system: once as it stands (FP64
Gram sums by BLAS) and once with every Gram matrix of the block update summed in extended
precision (numpy longdouble) and rounded to FP64. The first s estimates of the two runs
differ only through the rounding of W_1; that difference must lie within the bar the GPU
tests use (tests/parity_bars.py), so a library whose W_1 is more accurate than the oracle's
is not failed by the oracle's own error.
"""
import numpy as np
import pytest

from oracle import sstep as osstep
from oracle import stencil as ostencil
from paper_2001_04886_gb300 import inputs
from tests.parity_bars import cycle_abs_tol, cycle_x_tol, first_block_tol


def _extended_update(Y, V, T):
    Yh = Y - V @ T
    Yl = Yh.astype(np.longdouble)
    return Yh, (Yl.T @ Yl).astype(np.float64)


@pytest.mark.skipif(np.finfo(np.longdouble).nmant < 60, reason="needs an extended long double")
@pytest.mark.parametrize("N,s", [(32, 4), (32, 8), (64, 4), (64, 8)])
def test_oracle_first_block_rounding_within_bar(N, s, monkeypatch):
    Ao = ostencil.convdiff((N, N, N), (30.0, 20.0, 10.0))
    f = Ao.apply(inputs.x_true(0, Ao.n))
    sigma = 1.0 / Ao.norm_inf()
    tr = {}
    ref = osstep.sstep_gmres(Ao, f, np.zeros(Ao.n), s, 40, 1e-8, sigma, max_cycles=1, trace=tr)
    monkeypatch.setattr(osstep, "block_update", _extended_update)
    ext = osstep.sstep_gmres(Ao, f, np.zeros(Ao.n), s, 40, 1e-8, sigma, max_cycles=1)
    h, he = np.array(ref["history"][: s + 1]), np.array(ext["history"][: s + 1])
    diff = np.max(np.abs(h - he) / he)
    tol = first_block_tol(np.linalg.cond(tr["W"][0]))
    assert diff <= tol
    # the rounding is visible (the extended sums do change W_1), so the check has teeth
    assert diff > 0.0


def _extended_inner(V, Y):
    return (V.astype(np.longdouble).T @ Y.astype(np.longdouble)).astype(np.float64)


@pytest.mark.skipif(np.finfo(np.longdouble).nmant < 60, reason="needs an extended long double")
@pytest.mark.parametrize("N,s", [(32, 8), (64, 4), (64, 8)])
def test_oracle_cycle_rounding_within_bars(N, s, monkeypatch):
    """Every Gram matrix and inner product of the first cycle summed in extended precision:
    the whole cycle's history (absolute, against its first entry) and the iterate move by
    less than the bars of the GPU tests' first-cycle comparisons."""
    Ao = ostencil.convdiff((N, N, N), (30.0, 20.0, 10.0))
    f = Ao.apply(inputs.x_true(0, Ao.n))
    sigma = 1.0 / Ao.norm_inf()
    tr = {}
    ref = osstep.sstep_gmres(Ao, f, np.zeros(Ao.n), s, 40, 1e-8, sigma, max_cycles=1, trace=tr)
    monkeypatch.setattr(osstep, "block_update", _extended_update)
    monkeypatch.setattr(osstep, "inner_products", _extended_inner)
    ext = osstep.sstep_gmres(Ao, f, np.zeros(Ao.n), s, 40, 1e-8, sigma, max_cycles=1)
    cond = np.linalg.cond(tr["W"][0])
    h, he = np.array(ref["history"]), np.array(ext["history"])
    assert len(h) == len(he)
    assert np.all(np.abs(h - he) <= np.maximum(1e-6 * he, cycle_abs_tol(cond) * he[0]))
    dx = np.linalg.norm(ref["x"] - ext["x"]) / np.linalg.norm(ext["x"])
    assert dx <= cycle_x_tol(cond)
