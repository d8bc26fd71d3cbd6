"""Pins for the oracle's operator (closed forms and an independent dense assembly)."""
import numpy as np
import pytest

from oracle import dense, stencil


def grid_coords(shape):
    N = shape[0]
    h = 1.0 / (N + 1)
    axes = [np.arange(1, n + 1) * h for n in shape]
    # flat order x fastest
    mesh = np.meshgrid(*axes[::-1], indexing="ij")[::-1]
    return [m.reshape(-1) for m in mesh], h


@pytest.mark.parametrize("shape,beta", [((9, 9), (20.0, -7.0)), ((7, 7, 7), (30.0, 20.0, 10.0)), ((12, 12), (0.0, 0.0))])
def test_quadratic_closed_form(shape, beta):
    """P1: centred differences are exact for u quadratic in each variable.

    u = prod_d x_d (1 - x_d) vanishes on the boundary, so the Dirichlet rows
    need no correction: (A u)_p = h^2 [ -Lap u + beta . grad u ](x_p).
    """
    X, h = grid_coords(shape)
    dim = len(shape)
    q = [x * (1 - x) for x in X]
    u = np.prod(q, axis=0)
    lap = np.zeros_like(u)
    grad_term = np.zeros_like(u)
    for d in range(dim):
        others = np.prod([q[e] for e in range(dim) if e != d], axis=0)
        lap += -2.0 * others                     # d^2/dx_d^2 of x(1-x) = -2
        grad_term += beta[d] * (1 - 2 * X[d]) * others
    expect = h * h * (-lap + grad_term)
    A = stencil.convdiff(shape, beta)
    got = A.apply(u)
    assert np.max(np.abs(got - expect)) <= 1e-14 * np.max(np.abs(expect))


@pytest.mark.parametrize("shape,beta", [((10, 10), (20.0, 20.0)), ((6, 6, 6), (10.0, 6.0, -3.0))])
def test_eigenpairs_closed_form(shape, beta):
    """P2: A is diagonally similar to a symmetric matrix with known eigenpairs.

    In 1-D, tridiag(-1-c, 2, -1+c) has eigenvectors rho^i sin(i p pi h),
    rho = sqrt((1+c)/(1-c)), and eigenvalues 2 - 2 sqrt(1-c^2) cos(p pi h);
    the d-dimensional operator is the Kronecker sum (needs |c| < 1).
    """
    N = shape[0]
    dim = len(shape)
    h = 1.0 / (N + 1)
    A = stencil.convdiff(shape, beta)
    idx = [np.arange(1, N + 1)] * dim
    mesh = [m.reshape(-1) for m in np.meshgrid(*idx[::-1], indexing="ij")[::-1]]
    rng = np.random.default_rng(1)
    for _ in range(4):
        p = rng.integers(1, N + 1, size=dim)
        u = np.ones(A.n)
        lam = 0.0
        for d in range(dim):
            c = beta[d] * h / 2
            rho = np.sqrt((1 + c) / (1 - c))
            u *= rho ** mesh[d] * np.sin(mesh[d] * p[d] * np.pi * h)
            lam += 2 - 2 * np.sqrt(1 - c * c) * np.cos(p[d] * np.pi * h)
        res = A.apply(u) - lam * u
        assert np.linalg.norm(res) <= 1e-12 * np.linalg.norm(lam * u)


def test_dense_assembly_matches_apply():
    """Two independent formulations of the same rows agree, constant and variable coefficients."""
    rng = np.random.default_rng(2)
    for St in [stencil.convdiff((5, 5), (20.0, 20.0)), stencil.convdiff((4, 4, 4), (30.0, 20.0, 10.0)),
               stencil.convdiff_variable(6, rng.uniform(-40, 40, 36)),
               stencil.Stencil((5, 3, 4), rng.uniform(1, 2, 60), [rng.uniform(-1, 0, 60) for _ in range(3)],
                               [rng.uniform(-1, 0, 60) for _ in range(3)])]:
        D = dense.dense_matrix(St)
        for _ in range(3):
            x = rng.standard_normal(St.n)
            assert np.allclose(D @ x, St.apply(x), rtol=0, atol=1e-13)
        assert abs(St.norm_inf() - np.abs(D).sum(axis=1).max()) <= 1e-13


def test_norm_inf_is_4d():
    # holds while every cell Peclet number |c_d| = |beta_d| h / 2 is at most 1
    for shape, beta in [((8, 8), (17.0, 17.0)), ((5, 5, 5), (5.0, 4.0, -3.0))]:
        assert abs(stencil.convdiff(shape, beta).norm_inf() - 4 * len(shape)) < 1e-14


def test_gauss_solve_matches_library():
    rng = np.random.default_rng(3)
    M = rng.standard_normal((30, 30)) + 5 * np.eye(30)
    b = rng.standard_normal(30)
    assert np.allclose(dense.gauss_solve(M, b), np.linalg.solve(M, b), rtol=1e-12, atol=1e-12)


# ------------------------------------------------------------------ damped Jacobi (textbook smoother)
def test_jacobi_damps_laplacian_eigenmode_by_closed_form():
    """beta = 0: the sine mode (p, q) has eigenvalue lam = 4 - 2cos(p pi h) - 2cos(q pi h) of the
    h^2-scaled 2-D Laplacian; with f = 0 each sweep multiplies it by 1 - omega lam / 4."""
    N, p, q, omega, sweeps = 9, 2, 7, 0.8, 3
    A = stencil.convdiff((N, N), (0.0, 0.0))
    h = 1.0 / (N + 1)
    i = np.arange(1, N + 1)
    mode = np.outer(np.sin(q * np.pi * h * i), np.sin(p * np.pi * h * i)).reshape(-1)   # rows y, columns x
    lam = 4.0 - 2.0 * np.cos(p * np.pi * h) - 2.0 * np.cos(q * np.pi * h)
    got = stencil.jacobi(A, np.zeros(A.n), mode, sweeps, omega)
    np.testing.assert_allclose(got, (1.0 - omega * lam / 4.0) ** sweeps * mode, rtol=0, atol=1e-14)


def test_jacobi_diagonal_operator_is_solved_in_one_sweep():
    """With no neighbours A = a0 I, and one undamped sweep lands on f / a0 from any start."""
    rng = np.random.default_rng(3)
    A = stencil.Stencil((5, 4, 3), 6.0, [0.0] * 3, [0.0] * 3)
    f, x = rng.standard_normal(A.n), rng.standard_normal(A.n)
    np.testing.assert_allclose(stencil.jacobi(A, f, x, 1, 1.0), f / 6.0, rtol=0, atol=2e-15)


def test_jacobi_matches_dense_iteration_and_keeps_the_solution():
    """Against the iteration written with the dense matrix (assembled entry by entry) on a
    variable-coefficient operator; the exact solution is a fixed point."""
    rng = np.random.default_rng(4)
    N = 6
    A = stencil.convdiff_variable(N, 40.0 * rng.random(N * N))
    D = dense.dense_matrix(A)
    f, x = rng.standard_normal(A.n), rng.standard_normal(A.n)
    want = x.copy()
    for _ in range(4):
        want = want + 0.7 * (f - D @ want) / np.diag(D)
    np.testing.assert_allclose(stencil.jacobi(A, f, x, 4, 0.7), want, rtol=1e-13, atol=1e-13)
    xs = np.linalg.solve(D, f)
    np.testing.assert_allclose(stencil.jacobi(A, f, xs, 3, 0.8), xs, rtol=0, atol=1e-12)


# ------------------------------------------------------------------ variable coefficients (Sec. 5, eq. 10 form)
def variable_closed_form(N, beta_field):
    """h^2 [ -Lap u + beta(x, y) (u_x + u_y) ] at the nodes for u = x(1-x) y(1-y).

    u is quadratic in each variable, so the centred second and first differences of the
    five-point row are exact whatever beta is at the node: the row of the h^2-scaled
    operator equals the continuous operator times h^2, point by point.
    """
    (X, Y), h = grid_coords((N, N))
    u = X * (1 - X) * Y * (1 - Y)
    ux = (1 - 2 * X) * Y * (1 - Y)
    uy = (1 - 2 * Y) * X * (1 - X)
    neg_lap = 2 * Y * (1 - Y) + 2 * X * (1 - X)
    return u, h * h * (neg_lap + np.asarray(beta_field) * (ux + uy))


def row_magnitude(A, u):
    """sum_q |a_pq| |u_q| per row: the scale of the rounding error of any summation order."""
    ab = lambda c: np.abs(c) if not np.isscalar(c) else abs(c)
    return stencil.Stencil(A.shape, ab(A.a0), [ab(c) for c in A.am], [ab(c) for c in A.ap]).apply(np.abs(u))


def closed_form_ok(got, u, expect, Aref):
    """Within 16 ulps of each row's magnitude (the h^2-scaled row cancels by ~1/h^2)."""
    return bool(np.all(np.abs(got - expect) <= 16 * 2.0 ** -53 * row_magnitude(Aref, u)))


def matches_closed_form(A, N, beta_field):
    u, expect = variable_closed_form(N, beta_field)
    return closed_form_ok(A.apply(u), u, expect, A)


@pytest.mark.parametrize("N,kind", [(15, "uniform"), (31, "fourier"), (63, "signed"), (255, "uniform")])
def test_variable_quadratic_closed_form(N, kind):
    """P1 for the variable-coefficient operator: exact on u = x(1-x) y(1-y) for any beta field.

    The fields are a rough random field, the learned form's 8-mode Fourier field and a field
    of both signs; c(p) = beta(x_p, y_p) h / 2 multiplies both first differences of row p.
    N + 1 is a power of two, so the grid coordinates i h are exact and only the roundings
    of u and of the row sum remain (a few ulps of the row magnitude).
    """
    from paper_2001_04886_gb300 import inputs

    rng = np.random.default_rng(11)
    if kind == "uniform":
        beta = rng.uniform(0.0, 60.0, N * N)
    elif kind == "fourier":
        beta, _ = inputs.fourier_fields(7, N)
    else:
        beta = rng.uniform(-50.0, 50.0, N * N)
    assert matches_closed_form(stencil.convdiff_variable(N, beta), N, beta)


def test_variable_closed_form_catches_planted_slips():
    """Each slip a restatement could make fails the closed form: c = beta h instead of
    beta h / 2, the signs of c swapped between u_{p-e} and u_{p+e}, beta applied to x only,
    the field transposed (beta(y, x)), and a centre of 2 d - 1."""
    N = 15
    rng = np.random.default_rng(12)
    beta = rng.uniform(5.0, 60.0, N * N)
    h = 1.0 / (N + 1)
    c = beta * h / 2
    cT = (beta.reshape(N, N).T.reshape(-1)) * h / 2
    planted = {
        "beta h": stencil.Stencil((N, N), 4.0, [-1.0 - 2 * c, -1.0 - 2 * c], [-1.0 + 2 * c, -1.0 + 2 * c]),
        "sign swap": stencil.Stencil((N, N), 4.0, [-1.0 + c, -1.0 + c], [-1.0 - c, -1.0 - c]),
        "x only": stencil.Stencil((N, N), 4.0, [-1.0 - c, -1.0], [-1.0 + c, -1.0]),
        "transposed": stencil.Stencil((N, N), 4.0, [-1.0 - cT, -1.0 - cT], [-1.0 + cT, -1.0 + cT]),
        "centre": stencil.Stencil((N, N), 3.0, [-1.0 - c, -1.0 - c], [-1.0 + c, -1.0 + c]),
    }
    assert matches_closed_form(stencil.convdiff_variable(N, beta), N, beta)
    for name, A in planted.items():
        assert not matches_closed_form(A, N, beta), name
