"""The learned-initial-guess network's CUDA kernels against the FP64 oracle.

FP32 weights: forward and every parameter gradient agree with the oracle to the
FP32 accumulation level. BF16 weights: the same comparison against the oracle run
at the BF16-rounded weights (rounding to nearest even of the FP32 values), which
is exactly what the kernels multiply by.
"""
import numpy as np
import pytest

from oracle import unet as ounet
from paper_2001_04886_gb300 import inputs
from tests.gpu_util import dev, torch

import paper_2001_04886_gb300 as pkg

pytestmark = pytest.mark.gpu
KAPPA = 3.25


def bf16_round(a):
    """float32 values rounded to the nearest bfloat16 (ties to even), returned as float64."""
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def setup(B, H, seed, bf16, smooth=0, res_w=0.0):
    d = dev()
    theta = ounet.init_params(inputs.uniform01(seed, ounet.num_params())).astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((B, 2, H, H)).astype(np.float32)
    t = rng.standard_normal((B, 1, H, H)).astype(np.float32)
    net = pkg.X0Net(H, H, B, bf16=bf16, smooth=smooth, residual_weight=res_w, kappa=KAPPA)
    net.set_params(theta.astype(np.float32))
    xd = torch.tensor(x, device=d).contiguous()
    td = torch.tensor(t, device=d).contiguous()
    return net, theta, x.astype(np.float64), t.astype(np.float64), xd, td


def layer_slices():
    o = 0
    for ci, co, k, _ in ounet.LAYERS:
        n = co * ci * k * k + co
        yield slice(o, o + n)
        o += n


@pytest.mark.parametrize("B,H,smooth,res_w", [(2, 16, 0, 0.0), (3, 32, 0, 0.0), (2, 16, 3, 0.0), (2, 16, 3, 2.0)])
@pytest.mark.parametrize("bf16", [False, True])
def test_forward_and_gradient(B, H, smooth, res_w, bf16):
    net, theta, x, t, xd, td = setup(B, H, 7, bf16, smooth, res_w)
    th = theta.copy()
    if bf16:
        # weights are rounded; biases stay FP32
        for sl, (ci, co, k, _) in zip(layer_slices(), ounet.LAYERS):
            nw = co * ci * k * k
            th[sl.start : sl.start + nw] = bf16_round(theta[sl.start : sl.start + nw])
    out = torch.empty((B, 1, H, H), dtype=torch.float32, device=xd.device)
    net.forward(xd, out)
    torch.cuda.synchronize()
    ref = ounet.forward(th, x, smooth=smooth)
    got = out.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref)
    loss, g = net.gradient(xd, td)
    lref, gref = ounet.gradient(th, x, t, smooth=smooth, res_w=res_w, kappa=KAPPA)
    assert abs(loss - lref) <= 1e-5 * lref
    for sl in layer_slices():
        a, b = g[sl].astype(np.float64), gref[sl]
        assert np.linalg.norm(a - b) <= 1e-4 * np.linalg.norm(b) + 1e-12


def test_training_reduces_loss():
    net, theta, x, t, xd, td = setup(4, 16, 3, True)
    loss0, _ = net.gradient(xd, td)
    lossd = torch.zeros(1, dtype=torch.float32, device=xd.device)
    for _ in range(60):
        net.train_step(xd, td, 1e-3, lossd)
    torch.cuda.synchronize()
    loss1, _ = net.gradient(xd, td)
    assert loss1 < 0.5 * loss0


@pytest.mark.parametrize("B,H,smooth,res_w", [(2, 16, 0, 0.0), (3, 40, 3, 1.0), (2, 128, 2, 0.0)])
def test_tensor_core_convolutions_match_cuda_cores(B, H, smooth, res_w):
    """BF16 mode: the tcgen05 convolutions (FP32 activations split into three BF16 parts)
    and weight gradients (activations and output gradients split, six part products)
    give the CUDA-core result up to the FP32 accumulation inside the tensor core and the
    order of the sums (observed 2e-5 relative on the output at 128^2 over 15 layers):
    forward output, loss and every layer's gradient. H = 40 leaves a ragged pixel tile at
    every level; at H = 16 the coarsest level has 4 pixels of a 128-pixel tile."""
    net, theta, x, t, xd, td = setup(B, H, 11, True, smooth, res_w)
    outs, grads, losses = [], [], []
    for tc in (False, True):
        net.set_tensor_cores(tc)
        out = torch.empty((B, 1, H, H), dtype=torch.float32, device=xd.device)
        net.forward(xd, out)
        loss, g = net.gradient(xd, td)
        net.status()
        outs.append(out.cpu().numpy().astype(np.float64))
        grads.append(g.astype(np.float64))
        losses.append(loss)
    rel = np.linalg.norm(outs[1] - outs[0]) / np.linalg.norm(outs[0])
    print("output rel diff", rel)
    assert rel <= 1e-4
    assert abs(losses[1] - losses[0]) <= 1e-4 * abs(losses[0])
    for sl in layer_slices():
        a, b = grads[1][sl], grads[0][sl]
        assert np.linalg.norm(a - b) <= 1e-3 * np.linalg.norm(b) + 1e-12


def test_tensor_core_wait_timeout_is_reported_and_recoverable():
    """A bounded mbarrier wait that runs out (wait limit 0: no polls) makes the kernel
    drain its MMAs, free its tensor memory and report SSTEP_ERR_TIMEOUT through
    x0net_status; with the default limit restored the same network computes the
    correct output again in the same CUDA context."""
    net, theta, x, t, xd, td = setup(2, 16, 5, True)
    out_ok = torch.empty((2, 1, 16, 16), dtype=torch.float32, device=xd.device)
    net.forward(xd, out_ok)
    net.status()
    net.set_wait_limit(0)
    out = torch.full((2, 1, 16, 16), float("nan"), dtype=torch.float32, device=xd.device)
    net.forward(xd, out)
    with pytest.raises(pkg.SStepError) as ei:
        net.status()
    assert ei.value.status == -6      # SSTEP_ERR_TIMEOUT
    net.set_wait_limit(-1)
    net.status()                      # the flag was cleared by the report
    out2 = torch.empty_like(out_ok)
    net.forward(xd, out2)
    net.status()
    assert torch.equal(out2, out_ok)
    # the backward kernels (tensor-core weight gradient and backward-data convolutions)
    loss_ok, g_ok = net.gradient(xd, td)
    net.status()
    net.set_wait_limit(0)
    with pytest.raises(pkg.SStepError) as ei:
        net.gradient(xd, td)          # the gradient call reports the flag itself
    assert ei.value.status == -6
    with pytest.raises(pkg.SStepError):
        net.status()                  # ... and x0net_status reports it once more and clears it
    net.set_wait_limit(-1)
    loss2, g2 = net.gradient(xd, td)
    net.status()
    assert loss2 == loss_ok and np.array_equal(g2, g_ok)


def test_binding_refuses_batches_of_the_wrong_shape():
    net, theta, x, t, xd, td = setup(2, 16, 5, True)
    out = torch.empty((2, 1, 16, 16), dtype=torch.float32, device=xd.device)
    with pytest.raises(ValueError):
        net.forward(xd, out[:1])
    with pytest.raises(ValueError):
        net.forward(xd[:, :1].contiguous(), out)
    with pytest.raises(ValueError):
        net.gradient(xd, torch.empty((2, 1, 8, 8), dtype=torch.float32, device=xd.device))
    with pytest.raises(TypeError):
        net.forward(xd.double(), out)
    net.forward(xd, out)
    net.status()


def test_full_size_forward_and_gradient_match_the_oracle():
    """The learned form at its full size, in the configuration the bench trains and infers
    with (128^2, BF16 weights on the tensor cores, 4 smoothing passes): a batch of 32
    forwards, two of which (first and last) the oracle recomputes, and one gradient at
    batch 2 against the oracle's."""
    d = dev()
    H, B = 128, 32
    theta = ounet.init_params(inputs.uniform01(21, ounet.num_params())).astype(np.float32).astype(np.float64)
    th = theta.copy()
    for sl, (ci, co, k, _) in zip(layer_slices(), ounet.LAYERS):
        nw = co * ci * k * k
        th[sl.start : sl.start + nw] = bf16_round(theta[sl.start : sl.start + nw])
    rng = np.random.default_rng(22)
    x = rng.standard_normal((B, 2, H, H)).astype(np.float32)
    t = rng.standard_normal((B, 1, H, H)).astype(np.float32)
    net = pkg.X0Net(H, H, B, bf16=True, smooth=4, residual_weight=0.0, kappa=KAPPA)
    net.set_params(theta.astype(np.float32))
    xd = torch.tensor(x, device=d)
    out = torch.empty((B, 1, H, H), dtype=torch.float32, device=d)
    net.forward(xd, out)
    net.status()
    got = out.cpu().numpy().astype(np.float64)
    for i in (0, B - 1):
        ref = ounet.forward(th, x[i : i + 1].astype(np.float64), smooth=4)
        assert np.linalg.norm(got[i : i + 1] - ref) <= 1e-4 * np.linalg.norm(ref), i
    loss, g = net.gradient(xd[:2].contiguous(), torch.tensor(t[:2], device=d))
    lref, gref = ounet.gradient(th, x[:2].astype(np.float64), t[:2].astype(np.float64), smooth=4, res_w=0.0,
                                kappa=KAPPA)
    assert abs(loss - lref) <= 1e-4 * lref
    for sl in layer_slices():
        a, b = g[sl].astype(np.float64), gref[sl]
        assert np.linalg.norm(a - b) <= 1e-3 * np.linalg.norm(b) + 1e-12
    net.close()
