"""Seeded synthetic inputs shared by the CUDA path's tests/bench and by the oracle.

This module holds only random-number generation and the synthetic input recipes.
It contains none of the solver arithmetic (no operator, no Krylov step), so the
oracle and the CUDA path can both take their inputs from it without sharing any
of the method's code.

Generator: SplitMix64 (G. Steele, D. Lea, C. Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), written out here from its
published definition: the state advances by the golden-ratio increment and each
output is the state passed through the two xor-shift-multiply rounds and a final
xor-shift. Uniform doubles take the top 53 bits: u = (z >> 11) * 2^-53.
"""
from __future__ import annotations

import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Outputs number offset+1 .. offset+count of SplitMix64 started at `seed`."""
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """count doubles in [0, 1) from the top 53 bits of SplitMix64 outputs."""
    z = splitmix64(seed, count, offset)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def x_true(seed: int, n: int) -> np.ndarray:
    """The exact solution x_true[i] = 2u_i - 1 ~ U[-1, 1], in index order."""
    return 2.0 * uniform01(seed, n) - 1.0


class _Stream:
    """Sequential draws from one SplitMix64 stream (used for per-system parameters)."""

    def __init__(self, seed: int):
        self.seed = seed
        self.pos = 0

    def uniform(self, count: int = 1) -> np.ndarray:
        u = uniform01(self.seed, count, self.pos)
        self.pos += count
        return u


def batched_systems(seed: int, count: int, lmin: int = 32, lmax: int = 256):
    """Per-system (side L, beta) for the batched form: L ~ U{lmin..lmax}, beta ~ U[0, 50].

    Draw order per system: L, then beta. Each system's x_true uses its own seed
    (seed * 1_000_003 + system index) so that systems are independent of count.
    """
    st = _Stream(seed)
    out = []
    span = lmax - lmin + 1
    for i in range(count):
        u_l, u_b = st.uniform(2)
        L = lmin + int(math.floor(span * u_l))
        beta = 50.0 * u_b
        out.append({"L": L, "beta": beta, "xseed": seed * 1_000_003 + i})
    return out


def fourier_fields(seed: int, N: int, modes: int = 8):
    """Variable-coefficient 2-D field beta(x, y) and right-hand side f(x, y) on an N x N grid.

    beta = sum_q a_q cos(2 pi (p_q x + r_q y) + phi_q), a_q ~ U[0, 20], p_q, r_q in {0..4},
    phi_q ~ U[0, 2 pi); f = h^2 sum_q b_q sin(pi p'_q x) sin(pi r'_q y), b_q ~ U[-1, 1],
    p'_q, r'_q in {1..4}. Nodes are the interior points x_i = i h, h = 1/(N+1),
    ordered with x fastest. Returns (beta, f) as flat float64 arrays of N*N.
    """
    st = _Stream(seed)
    h = 1.0 / (N + 1)
    coords = np.arange(1, N + 1, dtype=np.float64) * h
    X, Yc = np.meshgrid(coords, coords, indexing="xy")
    beta = np.zeros((N, N))
    for _ in range(modes):
        a, p, r, phi = st.uniform(4)
        beta += 20.0 * a * np.cos(2 * np.pi * (math.floor(5 * p) * X + math.floor(5 * r) * Yc) + 2 * np.pi * phi)
    f = np.zeros((N, N))
    for _ in range(modes):
        b, p, r = st.uniform(3)
        f += (2.0 * b - 1.0) * np.sin(np.pi * (1 + math.floor(4 * p)) * X) * np.sin(np.pi * (1 + math.floor(4 * r)) * Yc)
    return beta.reshape(-1), (h * h) * f.reshape(-1)


def paper_problem(N: int, gamma: float = 50.0, beta: float = 1.0):
    """The test problem of Sec. 5 on an N x N interior grid (h = 1/(N+1), x fastest):

        -(b u_x)_x - (c u_y)_y + (d u)_x + (e u)_y + f u = g  on (0,1)^2, u = 0 on the boundary,
        b = exp(-xy), c = exp(xy), d = beta (x + y), e = gamma (x + y), f = 1 / (1 + xy),

    with g made from the analytic solution u = x exp(xy) sin(pi x) sin(pi y) (the printed
    sin(pi y) sin(pi y) read as sin(pi x) sin(pi y), which vanishes on the boundary).
    Five-point differences in conservative form for the diffusion terms (b, c at the cell
    faces), centred differences of the products d u and e u; every row scaled by h^2.

    Returns dict(coef=[a0, a_west, a_east, a_south, a_north] (n each), g (h^2 g at the
    nodes), u (analytic u at the nodes), x0 (the paper's initial guess x_i = 0.05 mod(i, 50),
    i = 1..n)). Generator of input data only: no arithmetic of the solvers.
    """
    h = 1.0 / (N + 1)
    t = (np.arange(N) + 1) * h
    X, Y = np.meshgrid(t, t)                       # rows: y, columns: x (x fastest)
    b = lambda x, y: np.exp(-x * y)
    c = lambda x, y: np.exp(x * y)
    d = lambda x, y: beta * (x + y)
    e = lambda x, y: gamma * (x + y)
    bw, be = b(X - h / 2, Y), b(X + h / 2, Y)
    cs, cn = c(X, Y - h / 2), c(X, Y + h / 2)
    a0 = bw + be + cs + cn + h * h / (1.0 + X * Y)
    aw = -bw - 0.5 * h * d(X - h, Y)
    ae = -be + 0.5 * h * d(X + h, Y)
    as_ = -cs - 0.5 * h * e(X, Y - h)
    an = -cn + 0.5 * h * e(X, Y + h)
    # g = L u by hand: u = x E S Sy with E = exp(xy), S = sin(pi x), Sy = sin(pi y)
    pi = np.pi
    E, S, C, Sy, Cy = np.exp(X * Y), np.sin(pi * X), np.cos(pi * X), np.sin(pi * Y), np.cos(pi * Y)
    u = X * E * S * Sy
    ux = E * Sy * (S + X * Y * S + pi * X * C)
    uy = X * E * S * (X * Sy + pi * Cy)
    uxx = E * Sy * (2 * Y * S + X * Y * Y * S + 2 * pi * X * Y * C + 2 * pi * C - pi * pi * X * S)
    uyy = X * E * S * (X * X * Sy + 2 * pi * X * Cy - pi * pi * Sy)
    bx, cy = -Y * np.exp(-X * Y), X * np.exp(X * Y)
    g = (-bx * ux - b(X, Y) * uxx - cy * uy - c(X, Y) * uyy + beta * u + d(X, Y) * ux + gamma * u + e(X, Y) * uy
         + u / (1.0 + X * Y))
    n = N * N
    i = np.arange(1, n + 1)
    return dict(coef=[a.reshape(-1).copy() for a in (a0, aw, ae, as_, an)], g=(h * h * g).reshape(-1),
                u=u.reshape(-1), x0=0.05 * np.mod(i, 50).astype(np.float64))
