"""Host-side pieces of the learned-initial-guess form, on the CPU: the network layout the
training code assumes, its initialisation and the target scale kappa."""
import numpy as np

from oracle import unet as ounet
from paper_2001_04886_gb300 import inputs, learned


def test_layer_table_matches_the_oracle_network():
    assert [(ci, co, k) for ci, co, k, _ in ounet.LAYERS] == list(learned._LAYERS)
    assert sum(co * ci * k * k + co for ci, co, k in learned._LAYERS) == ounet.num_params() == 302705


def test_he_uniform_initialisation():
    u = inputs.uniform01(12345, ounet.num_params())
    theta = learned._init_params(u)
    assert theta.dtype == np.float32
    o = 0
    for ci, co, k in learned._LAYERS:
        nw = co * ci * k * k
        a = np.sqrt(6.0 / (ci * k * k))
        w = theta[o : o + nw]
        assert np.all(np.abs(w) <= a) and np.abs(w).max() > 0.9 * a        # fills U[-a, a]
        assert abs(float(w.mean())) <= 4 * a / np.sqrt(3 * nw)             # centred (4 sigma)
        assert not np.any(theta[o + nw : o + nw + co])                      # zero biases
        o += nw + co
    assert o == len(theta)


def test_kappa_is_the_inverse_smallest_eigenvalue_scale():
    """kappa = 1/(2 pi^2 h^2): times the smallest eigenvalue of the h^2-scaled 2-D
    Laplacian, 4 (2 sin(pi h / 2))^2 / 2 per direction summed, it tends to 1 at second order."""
    for N, tol in ((32, 3e-3), (128, 2e-4)):
        h = 1.0 / (N + 1)
        lam = 2 * 4 * np.sin(np.pi * h / 2) ** 2
        assert abs(learned.kappa(N) * lam - 1.0) <= tol, N
