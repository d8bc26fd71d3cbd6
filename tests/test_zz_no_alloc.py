"""The allocation-free Gram entry point against the allocating one and the oracle.

sstep_gram_noalloc serves callers that cannot allocate device memory when they
call it: applications that fix their device-memory budget at start-up, and hosts
whose own allocator owns all device memory. It keeps its scratch in a fixed device
array shared by all calls, so this test also runs it twice in a row: the second
call must not see the first call's leftovers. The file is named to be collected
last, so that a run which stops at its first failure has run every other test
before this one.
"""
import ctypes

import numpy as np
import pytest

from oracle import sstep as osstep
from paper_2001_04886_gb300 import inputs
from tests.gpu_util import dev, to_dev, torch

import paper_2001_04886_gb300 as pkg

pytestmark = pytest.mark.gpu


def call_noalloc(Vd, Yd, n, ka, kb):
    C = torch.full((kb, ka), float("nan"), dtype=torch.float64, device=Vd.device).t()
    rc = pkg.lib().sstep_gram_noalloc(n, ctypes.c_void_p(Vd.data_ptr()), n, ka, ctypes.c_void_p(Yd.data_ptr()), n,
                                      kb, ctypes.c_void_p(C.data_ptr()), ka,
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, pkg.lib().sstep_status_string(rc)
    return C


@pytest.mark.parametrize("n,ka,kb", [(300001, 17, 5), (4096, 36, 4), (77, 1, 1)])
def test_noalloc_matches_gram_twice(n, ka, kb):
    d = dev()
    V = np.stack([inputs.x_true(10 + i, n) for i in range(ka)], axis=1)
    Y = np.stack([inputs.x_true(100 + j, n) for j in range(kb)], axis=1)
    Vd, Yd = to_dev(V.T, d).t(), to_dev(Y.T, d).t()
    ref = pkg.sstep_gram(Vd, Yd).cpu().numpy()
    oracle = osstep.inner_products(V, Y)
    scale = np.outer(np.linalg.norm(V, axis=0), np.linalg.norm(Y, axis=0))
    for _ in range(2):
        got = call_noalloc(Vd, Yd, n, ka, kb)
        torch.cuda.synchronize()
        got = got.cpu().numpy()
        assert np.max(np.abs(got - ref) / scale) <= 1e-14
        assert np.max(np.abs(got - oracle) / scale) <= 1e-14


def test_noalloc_rejects_sizes_beyond_the_maximum():
    d = dev()
    z = torch.zeros(64, dtype=torch.float64, device=d)
    p = ctypes.c_void_p(z.data_ptr())
    L = pkg.lib()
    assert L.sstep_gram_noalloc(8, p, 8, pkg.SSTEP_MAX_COLS + 1, p, 8, 1, p, 65, None) == -1
    assert L.sstep_gram_noalloc(8, p, 8, 1, p, 8, pkg.SSTEP_MAX_S + 2, p, 1, None) == -1
