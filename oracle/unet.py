"""FP64 reference of the learned-initial-guess U-Net: forward, loss and backward.

Test infrastructure (see the package header). The network is the 4-level U-Net
of the library (3x3 convolutions with zero padding 1 and ReLU; 2x2 mean pooling;
nearest-neighbour upsampling; skip connections by channel concatenation; a final
1x1 convolution), with the same flat parameter layout: per layer W[co][ci][kh][kw]
then b[co]. Every operation is written from its definition with numpy; the
backward pass is the chain rule applied step by step in reverse. Its gradients are
pinned against central finite differences of the forward pass.
"""
from __future__ import annotations

import numpy as np

# (cin, cout, k, relu) in forward order
LAYERS = [(2, 16, 3, 1), (16, 16, 3, 1), (16, 32, 3, 1), (32, 32, 3, 1), (32, 64, 3, 1), (64, 64, 3, 1),
          (64, 64, 3, 1), (64, 64, 3, 1), (128, 64, 3, 1), (64, 64, 3, 1), (96, 32, 3, 1), (32, 32, 3, 1),
          (48, 16, 3, 1), (16, 16, 3, 1), (16, 1, 1, 0)]


def num_params():
    return sum(co * ci * k * k + co for ci, co, k, _ in LAYERS)


def unpack(theta):
    out, o = [], 0
    for ci, co, k, _ in LAYERS:
        W = theta[o : o + co * ci * k * k].reshape(co, ci, k, k)
        o += co * ci * k * k
        b = theta[o : o + co]
        o += co
        out.append((W, b))
    return out


def conv_fwd(x, W, b):
    """out[b,o,y,x] = sum_{c,ky,kx} W[o,c,ky,kx] x[b,c,y+ky-1,x+kx-1] + bias[o] (zero outside)."""
    k = W.shape[2]
    B, C, H, Wd = x.shape
    if k == 1:
        return np.einsum("oc,bchw->bohw", W[:, :, 0, 0], x) + b[None, :, None, None]
    xp = np.zeros((B, C, H + 2, Wd + 2))
    xp[:, :, 1:-1, 1:-1] = x
    out = np.zeros((B, W.shape[0], H, Wd))
    for ky in range(3):
        for kx in range(3):
            out += np.einsum("oc,bchw->bohw", W[:, :, ky, kx], xp[:, :, ky : ky + H, kx : kx + Wd])
    return out + b[None, :, None, None]


def conv_bwd(x, W, g):
    """Gradients of conv_fwd: dx, dW, db for the output gradient g."""
    k = W.shape[2]
    B, C, H, Wd = x.shape
    if k == 1:
        dW = np.einsum("bohw,bchw->oc", g, x)[:, :, None, None]
        dx = np.einsum("oc,bohw->bchw", W[:, :, 0, 0], g)
        return dx, dW, g.sum(axis=(0, 2, 3))
    xp = np.zeros((B, C, H + 2, Wd + 2))
    xp[:, :, 1:-1, 1:-1] = x
    dxp = np.zeros_like(xp)
    dW = np.zeros_like(W)
    for ky in range(3):
        for kx in range(3):
            dW[:, :, ky, kx] = np.einsum("bohw,bchw->oc", g, xp[:, :, ky : ky + H, kx : kx + Wd])
            dxp[:, :, ky : ky + H, kx : kx + Wd] += np.einsum("oc,bohw->bchw", W[:, :, ky, kx], g)
    return dxp[:, :, 1:-1, 1:-1], dW, g.sum(axis=(0, 2, 3))


def pool(x):
    return 0.25 * (x[:, :, 0::2, 0::2] + x[:, :, 1::2, 0::2] + x[:, :, 0::2, 1::2] + x[:, :, 1::2, 1::2])


def pool_bwd(g):
    return 0.25 * np.repeat(np.repeat(g, 2, axis=2), 2, axis=3)


def up(x):
    return np.repeat(np.repeat(x, 2, axis=2), 2, axis=3)


def up_bwd(g):
    return g[:, :, 0::2, 0::2] + g[:, :, 1::2, 0::2] + g[:, :, 0::2, 1::2] + g[:, :, 1::2, 1::2]


def relu(z):
    return np.maximum(z, 0.0)


def blur(x):
    """One pass of the separable filter [1 2 1]/4 x [1 2 1]/4, zero outside the grid (self-adjoint)."""
    xp = np.zeros((x.shape[0], x.shape[1], x.shape[2] + 2, x.shape[3] + 2))
    xp[:, :, 1:-1, 1:-1] = x
    w = [0.25, 0.5, 0.25]
    H, W = x.shape[2], x.shape[3]
    out = np.zeros_like(x)
    for ky in range(3):
        for kx in range(3):
            out += w[ky] * w[kx] * xp[:, :, ky : ky + H, kx : kx + W]
    return out


def forward(theta, x, keep=False, smooth=0):
    """Output (B, 1, H, W); with keep, also the dict of every layer input and output."""
    P = unpack(theta)
    t = {"x": x}

    def layer(i, inp):
        z = conv_fwd(inp, *P[i])
        return relu(z) if LAYERS[i][3] else z

    t["a1"] = layer(0, x)
    t["e1"] = layer(1, t["a1"])
    t["a2"] = layer(2, pool(t["e1"]))
    t["e2"] = layer(3, t["a2"])
    t["a3"] = layer(4, pool(t["e2"]))
    t["e3"] = layer(5, t["a3"])
    t["ab"] = layer(6, pool(t["e3"]))
    t["bt"] = layer(7, t["ab"])
    t["u3"] = np.concatenate([up(t["bt"]), t["e3"]], axis=1)
    t["a4"] = layer(8, t["u3"])
    t["d3"] = layer(9, t["a4"])
    t["u2"] = np.concatenate([up(t["d3"]), t["e2"]], axis=1)
    t["a5"] = layer(10, t["u2"])
    t["d2"] = layer(11, t["a5"])
    t["u1"] = np.concatenate([up(t["d2"]), t["e1"]], axis=1)
    t["a6"] = layer(12, t["u1"])
    t["d1"] = layer(13, t["a6"])
    t["raw"] = layer(14, t["d1"])
    t["out"] = t["raw"]
    for _ in range(smooth):
        t["out"] = blur(t["out"])
    return (t["out"], t) if keep else t["out"]


def residual(out, x, kappa=1.0):
    """A out - f_hat for the operator the features encode: x[:, 0] = f / s_f, x[:, 1] = beta / 20,
    A the h^2-scaled -Lap u + beta (u_x + u_y) on the interior grid, h = 1/(H+1)."""
    from . import stencil

    B, _, H, W = x.shape
    r = np.zeros_like(out)
    for b in range(B):
        A = stencil.convdiff_variable(H, 20.0 * x[b, 1].reshape(-1))
        r[b, 0] = (kappa * A.apply(out[b, 0].reshape(-1)) - x[b, 0].reshape(-1)).reshape(H, W)
    return r


def residual_adjoint(r, x):
    """A^T r for the same operators (dense transpose of the row definition)."""
    from . import dense, stencil

    B, _, H, W = x.shape
    out = np.zeros_like(r)
    for b in range(B):
        A = stencil.convdiff_variable(H, 20.0 * x[b, 1].reshape(-1))
        out[b, 0] = (dense.dense_matrix(A).T @ r[b, 0].reshape(-1)).reshape(H, W)
    return out


def loss(theta, x, target, smooth=0, res_w=0.0, kappa=1.0):
    out = forward(theta, x, smooth=smooth)
    val = float(np.mean((out - target) ** 2))
    if res_w:
        val += res_w * float(np.mean(residual(out, x, kappa) ** 2))
    return val


def gradient(theta, x, target, smooth=0, res_w=0.0, kappa=1.0):
    """(loss, d loss / d theta) by the chain rule through every layer in reverse."""
    P = unpack(theta)
    out, t = forward(theta, x, keep=True, smooth=smooth)
    n = out.size
    g = 2.0 * (out - target) / n
    lval = float(np.mean((out - target) ** 2))
    if res_w:
        r = residual(out, x, kappa)
        lval += res_w * float(np.mean(r ** 2))
        g = g + res_w * 2.0 * kappa * residual_adjoint(r, x) / n
    for _ in range(smooth):
        g = blur(g)                      # the filter is self-adjoint
    grads = [None] * len(LAYERS)

    def back(i, inp, gout, outp):
        if LAYERS[i][3]:
            gout = gout * (outp > 0)
        dx, dW, db = conv_bwd(inp, P[i][0], gout)
        grads[i] = (dW, db)
        return dx

    gd1 = back(14, t["d1"], g, t["raw"])
    ga6 = back(13, t["a6"], gd1, t["d1"])
    gu1 = back(12, t["u1"], ga6, t["a6"])
    gd2, ge1 = up_bwd(gu1[:, :32]), gu1[:, 32:]
    ga5 = back(11, t["a5"], gd2, t["d2"])
    gu2 = back(10, t["u2"], ga5, t["a5"])
    gd3, ge2 = up_bwd(gu2[:, :64]), gu2[:, 64:]
    ga4 = back(9, t["a4"], gd3, t["d3"])
    gu3 = back(8, t["u3"], ga4, t["a4"])
    gbt, ge3 = up_bwd(gu3[:, :64]), gu3[:, 64:]
    gab = back(7, t["ab"], gbt, t["bt"])
    gp3 = back(6, pool(t["e3"]), gab, t["ab"])
    ge3 = ge3 + pool_bwd(gp3)
    ga3 = back(5, t["a3"], ge3, t["e3"])
    gp2 = back(4, pool(t["e2"]), ga3, t["a3"])
    ge2 = ge2 + pool_bwd(gp2)
    ga2 = back(3, t["a2"], ge2, t["e2"])
    gp1 = back(2, pool(t["e1"]), ga2, t["a2"])
    ge1 = ge1 + pool_bwd(gp1)
    ga1 = back(1, t["a1"], ge1, t["e1"])
    back(0, x, ga1, t["a1"])
    flat = np.concatenate([np.concatenate([dW.ravel(), db]) for dW, db in grads])
    return lval, flat


def init_params(seed_uniform, scale=1.0):
    """He-style initial weights from uniforms u in [0, 1): W ~ U[-a, a], a = sqrt(6 / fan_in); b = 0."""
    theta = np.zeros(num_params())
    o = 0
    for ci, co, k, _ in LAYERS:
        nw = co * ci * k * k
        a = scale * np.sqrt(6.0 / (ci * k * k))
        theta[o : o + nw] = a * (2.0 * seed_uniform[o : o + nw] - 1.0)
        o += nw + co
    return theta
