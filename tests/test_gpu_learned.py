"""The learned-initial-guess form, end to end at a small grid.

The operator built on the device from a beta field matches the oracle's; the x0
guard falls back to x0 = 0 for a useless guess; and a network trained with the
library's kernels on systems solved by the library's GPU solver lowers the mean
number of Krylov steps on held-out systems (the gain the form exists for).
"""
import numpy as np
import pytest

from oracle import sstep as osstep
from oracle import stencil as ostencil
from paper_2001_04886_gb300 import inputs, learned
from tests.gpu_util import dev, to_dev, torch

import paper_2001_04886_gb300 as pkg

pytestmark = pytest.mark.gpu


def test_variable_operator_matches_oracle():
    d = dev()
    N = 40
    beta, f = inputs.fourier_fields(5, N)
    Ao = ostencil.convdiff_variable(N, beta)
    A = pkg.StencilMatrix(2, (N, N), beta_field=to_dev(beta, d))
    x = inputs.x_true(1, Ao.n)
    y = torch.empty(Ao.n, dtype=torch.float64, device=d)
    A.apply(to_dev(x, d), y)
    torch.cuda.synchronize()
    ref = Ao.apply(x)
    assert np.max(np.abs(y.cpu().numpy() - ref)) <= 1e-14 * np.abs(ref).max()
    # and the solver on it matches the oracle's solve
    sig = 1.0 / Ao.norm_inf()
    r = osstep.sstep_gmres(Ao, f, np.zeros(Ao.n), 4, 20, 1e-8, sig, 2000)
    xd = torch.zeros(Ao.n, dtype=torch.float64, device=d)
    res = pkg.sstep_gmres_solve(A, to_dev(f, d), xd, 4, 20, 1e-8, max_cycles=2000, sigma=sig)
    assert res["status"] == 0 and res["cycles"] == r["cycles"]
    assert np.linalg.norm(xd.cpu().numpy() - r["x"]) <= 1e-8 * np.linalg.norm(r["x"])


def test_x0_guard_falls_back_to_zero():
    d = dev()
    N = 24
    beta, f = inputs.fourier_fields(9, N)
    A = pkg.StencilMatrix(2, (N, N), beta_field=to_dev(beta, d))
    fd = to_dev(f, d)
    x0 = torch.zeros(N * N, dtype=torch.float64, device=d)
    ref = pkg.sstep_gmres_solve(A, fd, x0, 4, 20, 1e-8)
    bad = torch.full((N * N,), 1e6, dtype=torch.float64, device=d)
    res = pkg.sstep_gmres_solve(A, fd, bad, 4, 20, 1e-8, x0_guard=True)
    assert res["status"] == 0 and res["cycles"] == ref["cycles"]
    # the batched solver applies the same guard
    B = pkg.BatchSolver([A], 4, 20, 1e-8, x0_guard=True)
    bad.fill_(1e6)
    rb = B.solve([fd], [bad])
    assert rb[0]["status"] == 0 and rb[0]["cycles"] == ref["cycles"]


def test_scalings_on_the_device():
    """The form's scalings by the library against their definitions: s_f = rms of f, the
    features (f / s_f, beta / 20) in FP32, targets x / (kappa s_f) and the initial guess
    kappa s_f * output, kappa = 1 / (2 pi^2 h^2)."""
    d = dev()
    N, B = 24, 3
    fields = [inputs.fourier_fields(30 + i, N) for i in range(B)]
    beta = np.stack([b for b, _ in fields])
    f = np.stack([f_ for _, f_ in fields])
    f[2] = 0.0                                    # f = 0: the scale is taken as 1
    feats, sf = pkg.x0net_features(N, N, to_dev(f, d), to_dev(beta, d))
    torch.cuda.synchronize()
    rms = np.sqrt(np.mean(f * f, axis=1))
    want_sf = np.where(rms > 0, rms, 1.0)
    np.testing.assert_allclose(sf.cpu().numpy(), want_sf, rtol=1e-14, atol=0)
    ft = feats.cpu().numpy()
    np.testing.assert_array_equal(ft[:, 0].reshape(B, -1), (f / want_sf[:, None]).astype(np.float32))
    np.testing.assert_array_equal(ft[:, 1].reshape(B, -1), (beta / 20.0).astype(np.float32))
    kap = 1.0 / (2.0 * np.pi ** 2 * (1.0 / (N + 1)) ** 2)
    x = np.stack([inputs.x_true(40 + i, N * N) for i in range(B)])
    t = pkg.x0net_targets(N, N, to_dev(x, d), sf).cpu().numpy()
    np.testing.assert_allclose(t.reshape(B, -1), (x / (kap * want_sf[:, None])).astype(np.float32), rtol=1e-7, atol=0)
    net = pkg.X0Net(N, N, B, bf16=False, smooth=0)
    net.set_params(np.random.default_rng(0).standard_normal(net.num_params).astype(np.float32) * 0.05)
    out = torch.empty((B, 1, N, N), dtype=torch.float32, device=d)
    net.forward(feats, out)
    x0 = torch.empty((B, N * N), dtype=torch.float64, device=d)
    net.predict(feats, sf, x0)
    torch.cuda.synchronize()
    want = kap * want_sf[:, None] * out.cpu().numpy().reshape(B, -1).astype(np.float64)
    np.testing.assert_allclose(x0.cpu().numpy(), want, rtol=1e-15, atol=0)
    net.close()


def test_trained_network_reduces_krylov_steps():
    dev()
    # training is deterministic (seeded order, fixed-order reductions, no atomics)
    ev = learned.run(N=32, train_seeds=range(2048), test_seeds=range(20000, 20128), epochs=40, batch=32, lr=2e-3,
                     log=None, smooth=4, residual_weight=1.0)
    print(ev)
    assert ev["all_converged"]
    assert ev["predicted"]["accepted_by_guard"] > 0
    # fewer Krylov steps than from x0 = 0 and than from x0 = 0 after the same smoothing sweeps
    assert ev["predicted"]["mean_iters"] < ev["zero"]["mean_iters"]
    assert ev["predicted"]["mean_iters"] < ev["zero_smoothed"]["mean_iters"]


class _DiesAfter:
    """The real network, except that the process 'dies' at a given training step."""

    def __init__(self, net, steps):
        self.net, self.left = net, steps

    def __getattr__(self, name):
        return getattr(self.net, name)

    def train_step(self, *args, **kwargs):
        if self.left == 0:
            raise RuntimeError("the process dies here")
        self.left -= 1
        return self.net.train_step(*args, **kwargs)


def test_training_resumes_bit_for_bit(tmp_path):
    """Checkpoint after every epoch; a run that dies inside epoch 1 and is resumed from
    the file on a fresh network ends with the uninterrupted run's weights, Adam moments
    and step count, bit for bit (every kernel of a step reduces in a fixed order)."""
    d = dev()
    N, B = 16, 4
    g = torch.Generator().manual_seed(8)
    feats = torch.randn(24, 2, N, N, generator=g).to(d)
    targets = torch.randn(24, 1, N, N, generator=g).to(d)

    def fresh():
        net = pkg.X0Net(N, N, B, bf16=True, smooth=2, residual_weight=0.5, kappa=2.0)
        net.set_params(learned._init_params(inputs.uniform01(1, net.num_params)))
        return net

    full = fresh()
    learned.train(full, feats, targets, epochs=3, batch=B, lr=1e-3, seed=2)
    ref = full.get_state()
    ck = tmp_path / "unet.ckpt"
    with pytest.raises(RuntimeError):
        learned.train(_DiesAfter(fresh(), 8), feats, targets, epochs=3, batch=B, lr=1e-3, seed=2, checkpoint=ck)
    assert learned.load_checkpoint(ck)["epoch"] == 1
    resumed = fresh()
    learned.train(resumed, feats, targets, epochs=3, batch=B, lr=1e-3, seed=2, checkpoint=ck, resume=True)
    got = resumed.get_state()
    assert got["step"] == ref["step"] == 18
    for k in ("params", "m", "v"):
        assert np.array_equal(got[k], ref[k]), k
    for net in (full, resumed):
        net.close()
