"""Kernel-level parity of the CUDA path against the oracle (stencil, powers, Gram, update)."""
import numpy as np
import pytest

from oracle import sstep as osstep
from oracle import stencil as ostencil
from paper_2001_04886_gb300 import inputs
from tests.gpu_util import dev, panel, relerr, to_dev, torch

import paper_2001_04886_gb300 as pkg

pytestmark = pytest.mark.gpu

SHAPES = [
    ((64, 64), (20.0, 20.0)),          # 2-D 64^2: n = 4096
    ((37, 29), (20.0, -13.0)),         # ragged 2-D, n not a multiple of 32
    ((3, 3), (20.0, 20.0)),            # tiny
    ((1, 1), (5.0, 5.0)),              # single unknown
    ((24, 24, 24), (30.0, 20.0, 10.0)),
    ((17, 9, 5), (30.0, 20.0, 10.0)),  # ragged 3-D
]


def make(shape, beta, d):
    dim = len(shape)
    if len(set(shape)) == 1:
        Ao = ostencil.convdiff(shape, beta)
        A = pkg.StencilMatrix(dim, shape, beta=beta)
    else:
        h = 1.0 / (shape[0] + 1)
        c = [b * h / 2 for b in beta]
        coef = [2.0 * dim]
        for cd in c:
            coef += [-1.0 - cd, -1.0 + cd]
        Ao = ostencil.Stencil(shape, coef[0], coef[1::2], coef[2::2])
        A = pkg.StencilMatrix(dim, shape, coef=coef)
    return Ao, A


@pytest.mark.parametrize("shape,beta", SHAPES)
def test_stencil_apply(shape, beta):
    d = dev()
    Ao, A = make(shape, beta, d)
    x = inputs.x_true(1, Ao.n)
    y = torch.empty(Ao.n, dtype=torch.float64, device=d)
    A.apply(to_dev(x, d), y)
    torch.cuda.synchronize()
    ref = Ao.apply(x)
    # one rounding per term in a different order: a few ulps of the row's magnitude
    bound = 1e-15 * 8 * np.abs(ref).max() + 1e-300
    assert np.max(np.abs(y.cpu().numpy() - ref)) <= bound
    assert abs(A.norm_inf - Ao.norm_inf()) <= 1e-14 * Ao.norm_inf()


def test_stencil_variable_coefficients():
    d = dev()
    N = 33
    beta, _ = inputs.fourier_fields(4, N)
    Ao = ostencil.convdiff_variable(N, beta)
    fields = [np.broadcast_to(Ao.a0, (Ao.n,)).copy()]
    for k in range(2):
        fields += [np.asarray(Ao.am[k]), np.asarray(Ao.ap[k])]
    A = pkg.StencilMatrix(2, (N, N), fields=[to_dev(fl, d) for fl in fields])
    x = inputs.x_true(2, Ao.n)
    y = torch.empty(Ao.n, dtype=torch.float64, device=d)
    A.apply(to_dev(x, d), y)
    torch.cuda.synchronize()
    ref = Ao.apply(x)
    assert np.max(np.abs(y.cpu().numpy() - ref)) <= 1e-14 * np.abs(ref).max()
    assert abs(A.norm_inf - Ao.norm_inf()) <= 1e-13 * Ao.norm_inf()


@pytest.mark.parametrize("N,kind", [(31, "fourier"), (127, "uniform"), (63, "signed"), (511, "uniform")])
def test_convdiff_variable_closed_form(N, kind):
    """The library's own variable-coefficient operator (beta field in, coefficients built on
    the device) against the closed form of Sec. 5's non-conservative convection-diffusion:
    exact on u = x(1-x) y(1-y) for any beta, so a slip in c = beta h / 2 or its sign fails."""
    from tests.test_oracle_stencil import closed_form_ok, variable_closed_form

    d = dev()
    rng = np.random.default_rng(N)
    if kind == "fourier":
        beta, _ = inputs.fourier_fields(5, N)
    elif kind == "uniform":
        beta = rng.uniform(0.0, 60.0, N * N)
    else:
        beta = rng.uniform(-50.0, 50.0, N * N)
    A = pkg.StencilMatrix(2, (N, N), beta_field=to_dev(beta, d))
    u, expect = variable_closed_form(N, beta)
    y = torch.empty(N * N, dtype=torch.float64, device=d)
    A.apply(to_dev(u, d), y)
    torch.cuda.synchronize()
    Ao = ostencil.convdiff_variable(N, beta)   # only for the rounding scale of each row
    assert closed_form_ok(y.cpu().numpy(), u, expect, Ao)
    assert abs(A.norm_inf - Ao.norm_inf()) <= 1e-13 * Ao.norm_inf()


@pytest.mark.parametrize("shape,beta", [SHAPES[0], SHAPES[1], SHAPES[4], SHAPES[5]])
@pytest.mark.parametrize("s", [1, 4, 8])
def test_matrix_powers(shape, beta, s):
    d = dev()
    Ao, A = make(shape, beta, d)
    v = inputs.x_true(3, Ao.n)
    sigma = 1.0 / Ao.norm_inf()
    Y = panel(Ao.n, s + 1, d)
    pkg.sstep_matrix_powers(A, to_dev(v, d), 0.5, sigma, s, Y)
    torch.cuda.synchronize()
    ref = osstep.matrix_powers(Ao, v, s, sigma, scale=0.5)
    got = Y.cpu().numpy()
    for j in range(s + 1):
        assert relerr(got[:, j], ref[:, j]) <= 1e-14 * (j + 1), j


@pytest.mark.parametrize("n,ka,kb", [(4096, 36, 4), (1000, 8, 9), (77, 1, 1), (300001, 17, 5), (5, 64, 3)])
def test_gram(n, ka, kb):
    d = dev()
    V = np.stack([inputs.x_true(10 + i, n) for i in range(ka)], axis=1)
    Y = np.stack([inputs.x_true(100 + j, n) for j in range(kb)], axis=1)
    Vd = to_dev(V.T, d).t()
    Yd = to_dev(Y.T, d).t()
    C = pkg.sstep_gram(Vd, Yd)
    C2 = pkg.sstep_gram(Vd, Yd)
    torch.cuda.synchronize()
    ref = osstep.inner_products(V, Y)
    scale = np.outer(np.linalg.norm(V, axis=0), np.linalg.norm(Y, axis=0))
    got = C.cpu().numpy()
    assert np.max(np.abs(got - ref) / scale) <= 1e-14
    assert np.array_equal(got, C2.cpu().numpy())   # fixed reduction order: bitwise reproducible


@pytest.mark.parametrize("n,ka,kb", [(4096, 12, 5), (5000, 0, 3), (300001, 33, 9), (31, 3, 2)])
def test_block_update(n, ka, kb):
    d = dev()
    V = np.stack([inputs.x_true(20 + i, n) for i in range(ka)], axis=1) if ka else np.zeros((n, 0))
    Y = np.stack([inputs.x_true(200 + j, n) for j in range(kb)], axis=1)
    T = np.stack([inputs.x_true(300 + j, ka) for j in range(kb)], axis=1) if ka else np.zeros((0, kb))
    Yd = to_dev(Y.T, d).t()
    G = pkg.sstep_block_update(to_dev(V.T, d).t() if ka else None, Yd, to_dev(T, d) if ka else None)
    torch.cuda.synchronize()
    Yh, Gr = osstep.block_update(Y, V, T)
    got = Yd.cpu().numpy()
    for j in range(kb):
        assert relerr(got[:, j], Yh[:, j]) <= 1e-14
    nrm = np.linalg.norm(Yh, axis=0)
    assert np.max(np.abs(G.cpu().numpy() - Gr) / np.outer(nrm, nrm)) <= 1e-14


@pytest.mark.parametrize("shape,beta", [SHAPES[1], SHAPES[3], SHAPES[5]])
@pytest.mark.parametrize("sweeps", [0, 1, 2, 5])
def test_jacobi_smoother(shape, beta, sweeps):
    """Damped Jacobi sweeps against the oracle's; odd and even counts (the result lands in
    x either way), ragged grids and a single unknown."""
    d = dev()
    Ao, A = make(shape, beta, d)
    f = inputs.x_true(5, Ao.n)
    x = inputs.x_true(6, Ao.n)
    xd = to_dev(x, d)
    work = torch.full_like(xd, float("nan"))
    A.smooth(to_dev(f, d), xd, work, sweeps, 0.8)
    torch.cuda.synchronize()
    ref = ostencil.jacobi(Ao, f, x, sweeps, 0.8)
    assert np.max(np.abs(xd.cpu().numpy() - ref)) <= 1e-14 * (1 + np.abs(ref).max())


def test_jacobi_smoother_variable_and_arguments():
    d = dev()
    N = 33
    beta, f = inputs.fourier_fields(7, N)
    Ao = ostencil.convdiff_variable(N, beta)
    A = pkg.StencilMatrix(2, (N, N), beta_field=to_dev(beta, d))
    x = inputs.x_true(8, Ao.n)
    xd, fd = to_dev(x, d), to_dev(f, d)
    work = torch.empty_like(xd)
    A.smooth(fd, xd, work, 3, 0.7)
    torch.cuda.synchronize()
    ref = ostencil.jacobi(Ao, f, x, 3, 0.7)
    assert np.max(np.abs(xd.cpu().numpy() - ref)) <= 1e-13 * (1 + np.abs(ref).max())
    for bad in (dict(sweeps=-1, omega=0.8, w=work), dict(sweeps=2, omega=0.0, w=work),
                dict(sweeps=2, omega=2.0, w=work), dict(sweeps=2, omega=0.8, w=xd)):
        with pytest.raises(pkg.SStepError):
            A.smooth(fd, xd, bad["w"], bad["sweeps"], bad["omega"])


@pytest.mark.parametrize("sweeps", [1, 4, 5])
def test_jacobi_smoother_batched_equals_single(sweeps):
    """The batched smoother (all systems per launch) gives each system's single-system
    result bit for bit: mixed sizes, constant and variable coefficients."""
    d = dev()
    mats, fs, xs = [], [], []
    for i, (shape, beta) in enumerate([SHAPES[1], SHAPES[3], SHAPES[5], SHAPES[0]]):
        _, A = make(shape, beta, d)
        mats.append(A)
        fs.append(to_dev(inputs.x_true(20 + i, A.n), d))
        xs.append(to_dev(inputs.x_true(30 + i, A.n), d))
    bv, fv = inputs.fourier_fields(9, 24)
    mats.append(pkg.StencilMatrix(2, (24, 24), beta_field=to_dev(bv, d)))
    fs.append(to_dev(fv, d))
    xs.append(to_dev(inputs.x_true(40, 576), d))
    single = [x.clone() for x in xs]
    for A, f, x in zip(mats, fs, single):
        A.smooth(f, x, torch.empty_like(x), sweeps, 0.8)
    batched = [x.clone() for x in xs]
    pkg.stencil_matrix_smooth_batched(mats, fs, batched, [torch.empty_like(x) for x in xs], sweeps, 0.8)
    torch.cuda.synchronize()
    for a, b in zip(batched, single):
        assert torch.equal(a, b)
