"""The learned-initial-guess form: a U-Net predicts x0 for the s-step GMRES solve.

Systems: the 2-D operator of -Lap u + beta(x, y)(u_x + u_y) on an N x N grid, beta
and f from 8 random Fourier modes each (inputs.fourier_fields). Training data are
solutions computed by the library's own FP64 s-step GMRES (batched persistent
solver); the network (X0Net) is trained with the library's own forward/backward
and Adam kernels. Evaluation solves held-out systems from x0 = 0 and from the
predicted x0; the solver's x0 guard falls back to x0 = 0 when the predicted
guess's residual exceeds ||f||, so the method is never worse off in iterations
than without the network. Before the guard, the prediction is post-smoothed by a
few damped Jacobi sweeps (stencil_matrix_smooth): the h^2-scaled operator
amplifies the rough part of the prediction's error by up to ~1/(2 pi^2 h^2), and
the sweeps remove that part while keeping the smooth part the network gets right.
The same sweeps applied to x0 = 0 are reported as a control.

Scaling (done on the device by the library: x0net_features, x0net_targets,
x0net_predict): the network sees f / s_f and beta / 20 (s_f = rms of f) and predicts
x / (kappa s_f) with kappa = 1 / (2 pi^2 h^2), the inverse of the smallest
eigenvalue scale of the h^2-scaled operator, so that targets are O(1) on every
grid; since A x = f is linear in f for fixed beta, scaling f scales x.
"""
from __future__ import annotations

import time

import numpy as np

from . import inputs
from ._binding import (BatchSolver, StencilMatrix, X0Net, stencil_matrix_smooth_batched, x0net_features,
                       x0net_targets)

SWEEPS = 32          # damped Jacobi sweeps on the predicted x0
OMEGA = 0.8          # their damping (the smoothing optimum for the 2-D 5-point Laplacian)


def kappa(N):
    h = 1.0 / (N + 1)
    return 1.0 / (2.0 * np.pi ** 2 * h * h)


def make_systems(seeds, N, device):
    """Operators, right-hand sides (FP64, device), features (FP32, device) and f scales
    (FP64, device): the features and scales come from the library (x0net_features)."""
    import torch

    mats, fs, betas = [], [], []
    for sd in seeds:
        beta, f = inputs.fourier_fields(int(sd), N)
        bd = torch.tensor(beta, dtype=torch.float64, device=device)
        mats.append(StencilMatrix(2, (N, N), beta_field=bd))
        fs.append(torch.tensor(f, dtype=torch.float64, device=device))
        betas.append(bd)
    feats, scales = x0net_features(N, N, torch.stack(fs).contiguous(), torch.stack(betas).contiguous())
    return mats, fs, feats, scales


def solve_batch(mats, fs, x0s, s=4, m=20, tol=1e-8, guard=False, tune=False):
    """Batched persistent s-step GMRES; returns (results, milliseconds)."""
    import torch

    B = BatchSolver(mats, s, m, tol, max_cycles=5000, x0_guard=guard)
    if tune:
        B.tune(fs, x0s)
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    res = B.solve(fs, x0s, mode=B.PERSISTENT)
    e1.record(st)
    torch.cuda.synchronize()
    B.close()
    return res, e0.elapsed_time(e1)


def generate(seeds, N, device, chunk=1024, report=None):
    """Training pairs: features (S, 2, N, N) and targets x / (kappa s_f) (S, 1, N, N), FP32 on
    the device. Systems whose solve does not converge are left out; `report` (a dict, if
    given) receives their seeds and statuses."""
    import torch

    feats, targets = [], []
    dropped = []
    for c0 in range(0, len(seeds), chunk):
        part = seeds[c0 : c0 + chunk]
        mats, fs, ft, sc = make_systems(part, N, device)
        xs = [torch.zeros_like(f) for f in fs]
        res, _ = solve_batch(mats, fs, xs)
        keep = []
        for i, r in enumerate(res):
            if r["status"] != 0:
                dropped.append((int(part[i]), r["status"], r["cycles"]))
                continue
            keep.append(i)
        idx = torch.tensor(keep, device=device, dtype=torch.long)
        if keep:   # x / (kappa s_f), by the library (x0net_targets)
            targets.append(x0net_targets(N, N, torch.stack([xs[i] for i in keep]).contiguous(), sc[idx].contiguous()))
        feats.append(ft[idx])
        del mats, fs, xs
    if report is not None:
        report["dropped"] = dropped
    return torch.cat(feats), torch.cat(targets)


# checkpoint file: magic, format version, then little-endian int64 num_params, Adam
# step, epochs done, shuffle seed, and the float32 arrays params, m, v (num_params each)
_CKPT_MAGIC = b"SSX0"
_CKPT_VERSION = 1


def save_checkpoint(path, net, epoch, seed):
    """Writes the network's training state after `epoch` completed epochs (atomically:
    a temporary file renamed over `path`)."""
    import os

    st = net.get_state()
    n = st["params"].shape[0]
    head = np.array([n, st["step"], epoch, seed], dtype="<i8")
    tmp = str(path) + ".tmp"
    with open(tmp, "wb") as fh:
        fh.write(_CKPT_MAGIC)
        fh.write(np.array([_CKPT_VERSION], dtype="<u4").tobytes())
        fh.write(head.tobytes())
        for k in ("params", "m", "v"):
            fh.write(np.ascontiguousarray(st[k], dtype="<f4").tobytes())
    os.replace(tmp, path)


def load_checkpoint(path):
    """Reads a checkpoint: dict(params, m, v, step, epoch, seed); ValueError if the file is
    not one, is of another version or is truncated."""
    with open(path, "rb") as fh:
        raw = fh.read()
    if len(raw) < 40 or raw[:4] != _CKPT_MAGIC:
        raise ValueError(f"{path}: not a checkpoint")
    if int(np.frombuffer(raw[4:8], dtype="<u4")[0]) != _CKPT_VERSION:
        raise ValueError(f"{path}: unsupported checkpoint version")
    n, step, epoch, seed = (int(v) for v in np.frombuffer(raw[8:40], dtype="<i8"))
    if n < 0 or len(raw) != 40 + 12 * n:
        raise ValueError(f"{path}: truncated checkpoint")
    arr = [np.frombuffer(raw[40 + 4 * n * i : 40 + 4 * n * (i + 1)], dtype="<f4").astype(np.float32) for i in range(3)]
    return {"params": arr[0], "m": arr[1], "v": arr[2], "step": step, "epoch": epoch, "seed": seed}


def train(net, feats, targets, epochs, batch=32, lr=1e-3, seed=0, log=None, checkpoint=None, resume=False):
    """Adam on the mean-squared error; learning rate halved for the last third of the epochs.

    checkpoint: a path written after every epoch (save_checkpoint). resume: if that file
    exists, training continues from it (the same seed required): the state is restored
    and the shuffles of the completed epochs are drawn again, so the result equals an
    uninterrupted run. Returns the per-epoch losses of the epochs run here.
    """
    import os

    import torch

    S = feats.shape[0]
    g = torch.Generator(device="cpu").manual_seed(seed)
    lossd = torch.zeros(1, dtype=torch.float32, device=feats.device)
    history = []
    start = 0
    if resume and checkpoint is not None and os.path.exists(checkpoint):
        ck = load_checkpoint(checkpoint)
        if ck["seed"] != seed:
            raise ValueError("checkpoint was written with another shuffle seed")
        net.set_state(ck)
        start = min(ck["epoch"], epochs)
        for _ in range(start):
            torch.randperm(S, generator=g)
    for ep in range(start, epochs):
        rate = lr if ep < (2 * epochs) // 3 else lr / 2
        perm = torch.randperm(S, generator=g).to(feats.device)
        tot, nb = 0.0, 0
        for b0 in range(0, S - batch + 1, batch):
            idx = perm[b0 : b0 + batch]
            net.train_step(feats.index_select(0, idx).contiguous(), targets.index_select(0, idx).contiguous(), rate,
                           lossd)
            if (b0 // batch) % 16 == 0:
                tot += float(lossd.item())
                nb += 1
        net.status()   # raises if a tensor-core kernel's bounded wait ran out
        history.append(tot / max(nb, 1))
        if checkpoint is not None:
            save_checkpoint(checkpoint, net, ep + 1, seed)
        if log:
            log(f"epoch {ep}: loss {history[-1]:.4e}")
    return history


def predict(net, feats, scales, batch=32):
    """x0 = kappa s_f net(features) by the library (x0net_predict): FP64 device vectors, the
    rows of one (S, N*N) tensor."""
    import torch

    N = feats.shape[-1]
    S = feats.shape[0]
    assert feats.dim() == 4 and feats.shape[-2] == N, "features must be (S, 2, N, N)"
    x0 = torch.empty((S, N * N), dtype=torch.float64, device=feats.device)
    for b0 in range(0, S, batch):
        net.predict(feats[b0 : b0 + batch].contiguous(), scales[b0 : b0 + batch].contiguous(), x0[b0 : b0 + batch])
    return list(x0.unbind(0))


def post_smooth(mats, fs, xs, sweeps, omega=OMEGA):
    """`sweeps` damped Jacobi sweeps on every x in place (the library's batched kernel:
    one launch per sweep for all systems)."""
    import torch

    if sweeps <= 0:
        return xs
    works = [torch.empty_like(x) for x in xs]
    stencil_matrix_smooth_batched(mats, fs, xs, works, sweeps, omega)
    return xs


def relres(mats, fs, xs):
    """||f - A x|| / ||f|| per system (library operator, norms on the device)."""
    import torch

    out = []
    for A, f, x in zip(mats, fs, xs):
        y = torch.empty_like(x)
        A.apply(x, y)
        out.append(float((f - y).norm() / f.norm()))
    return out


def _arm(res, ms, sweeps, r0=None):
    d = {"converged": int(sum(r["status"] == 0 for r in res)),
         "mean_cycles": float(np.mean([r["cycles"] for r in res])),
         "mean_iters": float(np.mean([r["iters"] for r in res])),
         "mean_matvecs": float(np.mean([r["matvecs"] for r in res])) + sweeps, "solve_ms": ms}
    if r0 is not None:
        d["median_relres_x0"] = float(np.median(r0))
    return d


def evaluate(net, seeds, N, device, sweeps=SWEEPS):
    """Cycles, Krylov steps and solve time from x0 = 0, from x0 = 0 after the smoothing
    sweeps (control), and from the predicted x0 after the sweeps (with the guard). The
    matvec counts include the sweeps; inference_ms (network and sweeps) is reported
    apart from solve_ms; all_converged covers the x0 = 0 and predicted arms."""
    import torch

    mats, fs, ft, sc = make_systems(seeds, N, device)
    x_zero = [torch.zeros_like(f) for f in fs]
    r0, t0 = solve_batch(mats, fs, x_zero)
    x_zs = post_smooth(mats, fs, [torch.zeros_like(f) for f in fs], sweeps)
    rz0 = relres(mats, fs, x_zs)
    rz, tz = solve_batch(mats, fs, x_zs, guard=True)
    torch.cuda.synchronize()
    ti = time.perf_counter()
    x_pred = post_smooth(mats, fs, predict(net, ft, sc), sweeps)
    torch.cuda.synchronize()
    t_inf = 1e3 * (time.perf_counter() - ti)
    rp0 = relres(mats, fs, x_pred)
    r1, t1 = solve_batch(mats, fs, x_pred, guard=True)
    ok = all(r["status"] == 0 for r in r0 + r1)
    pred = _arm(r1, t1, sweeps, rp0)
    pred["inference_ms"] = t_inf
    pred["accepted_by_guard"] = int(sum(v <= 1.0 for v in rp0))
    return {"systems": len(seeds), "all_converged": ok, "sweeps": sweeps, "omega": OMEGA,
            "zero": _arm(r0, t0, 0), "zero_smoothed": _arm(rz, tz, sweeps, rz0), "predicted": pred}


def run(N=128, train_seeds=range(20000), test_seeds=range(20000, 21000), epochs=8, batch=32, lr=1e-3, log=print,
        smooth=4, residual_weight=0.003, sweeps=SWEEPS):
    """The whole form: generate, train, evaluate. Returns a dict of the measurements."""
    import torch

    dev = torch.device("cuda", torch.cuda.current_device())
    t = time.perf_counter()
    rep = {}
    feats, targets = generate(np.array(list(train_seeds)), N, dev, report=rep)
    t_gen = time.perf_counter() - t
    net = X0Net(N, N, batch, bf16=True, smooth=smooth, residual_weight=residual_weight, kappa=kappa(N))
    from . import inputs as _in

    u = _in.uniform01(12345, net.num_params)
    net.set_params(_init_params(u))
    t = time.perf_counter()
    hist = train(net, feats, targets, epochs, batch, lr, log=log)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t
    ev = evaluate(net, np.array(list(test_seeds)), N, dev, sweeps)
    ev.update({"grid": N, "train_systems": int(feats.shape[0]), "dropped": rep.get("dropped", []), "epochs": epochs,
               "loss_history": hist,
               "generate_s": t_gen, "train_s": t_train, "params": net.num_params})
    net.close()
    return ev


# layer shapes (cin, cout, k) in the library's parameter order
_LAYERS = [(2, 16, 3), (16, 16, 3), (16, 32, 3), (32, 32, 3), (32, 64, 3), (64, 64, 3), (64, 64, 3), (64, 64, 3),
           (128, 64, 3), (64, 64, 3), (96, 32, 3), (32, 32, 3), (48, 16, 3), (16, 16, 3), (16, 1, 1)]


def _init_params(u):
    """Uniform He initialisation W ~ U[-a, a], a = sqrt(6 / fan_in), zero biases (u: uniforms in [0, 1))."""
    theta = np.zeros(len(u), dtype=np.float32)
    o = 0
    for ci, co, k in _LAYERS:
        nw = co * ci * k * k
        a = np.sqrt(6.0 / (ci * k * k))
        theta[o : o + nw] = (a * (2.0 * u[o : o + nw] - 1.0)).astype(np.float32)
        o += nw + co
    return theta
