"""Pins of the U-Net oracle: gradients against central finite differences, and
the building blocks against their definitions on small arrays."""
import numpy as np

from oracle import unet
from paper_2001_04886_gb300 import inputs


def small_problem(B=2, H=8, seed=0):
    theta = unet.init_params(inputs.uniform01(seed, unet.num_params()))
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((B, 2, H, H))
    t = rng.standard_normal((B, 1, H, H))
    return theta, x, t


def test_param_count():
    assert unet.num_params() == sum(co * ci * k * k + co for ci, co, k, _ in unet.LAYERS)
    assert 250_000 < unet.num_params() < 600_000


import pytest


@pytest.mark.parametrize("smooth,res_w,kappa", [(0, 0.0, 1.0), (2, 0.0, 1.0), (2, 3.0, 7.5)])
def test_gradient_matches_central_differences(smooth, res_w, kappa):
    theta, x, t = small_problem()
    _, g = unet.gradient(theta, x, t, smooth=smooth, res_w=res_w, kappa=kappa)
    rng = np.random.default_rng(1)
    idx = rng.choice(theta.size, 60, replace=False)
    # include every layer's bias and first weight
    o = 0
    for ci, co, k, _ in unet.LAYERS:
        idx = np.append(idx, [o, o + co * ci * k * k])
        o += co * ci * k * k + co
    eps = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += eps
        tm[i] -= eps
        fd = (unet.loss(tp, x, t, smooth, res_w, kappa) - unet.loss(tm, x, t, smooth, res_w, kappa)) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1e-3, abs(fd)) + 1e-9, (i, fd, g[i])


def test_conv_matches_direct_sum():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((1, 3, 5, 6))
    W = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    out = unet.conv_fwd(x, W, b)
    for o in range(4):
        for y in range(5):
            for xx in range(6):
                s = b[o]
                for c in range(3):
                    for ky in range(3):
                        for kx in range(3):
                            yy, xq = y + ky - 1, xx + kx - 1
                            if 0 <= yy < 5 and 0 <= xq < 6:
                                s += W[o, c, ky, kx] * x[0, c, yy, xq]
                assert abs(out[0, o, y, xx] - s) < 1e-12


def test_pool_and_up_are_adjoint_pairs():
    rng = np.random.default_rng(3)
    a = rng.standard_normal((2, 3, 8, 8))
    b = rng.standard_normal((2, 3, 4, 4))
    assert abs(np.sum(unet.pool(a) * b) - np.sum(a * unet.pool_bwd(b))) < 1e-12
    assert abs(np.sum(unet.up(b) * a) - np.sum(b * unet.up_bwd(a))) < 1e-12


def test_blur_is_self_adjoint_and_keeps_constants_inside():
    rng = np.random.default_rng(4)
    a = rng.standard_normal((1, 1, 9, 7))
    b = rng.standard_normal((1, 1, 9, 7))
    assert abs(np.sum(unet.blur(a) * b) - np.sum(a * unet.blur(b))) < 1e-12
    c = unet.blur(np.ones((1, 1, 6, 6)))
    assert abs(c[0, 0, 2, 3] - 1.0) < 1e-15 and abs(c[0, 0, 0, 0] - 0.5625) < 1e-15
