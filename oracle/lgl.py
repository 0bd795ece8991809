"""Gauss-Lobatto-Legendre (GLL/LGL) nodes, quadrature weights and the nodal
differentiation matrix (Sec. 2.2: n GLL points per direction, spectral
differentiation matrices built from the Lagrange basis, after Costa & Don).

Test infrastructure only (see ``oracle/__init__.py``).

Pinned by ``tests/test_oracle_lgl.py``: tabulated nodes/weights for small N
(``tests/golden/lgl_tabulated.txt``), exactness of the quadrature up to degree
2N-1, and exact differentiation of monomials up to degree N.
"""
import numpy as np


def legendre_pair(N, x):
    """Return (P_N(x), P_{N-1}(x)) by the three-term Bonnet recurrence."""
    x = np.asarray(x, dtype=np.float64)
    p_prev = np.ones_like(x)
    if N == 0:
        return p_prev, np.zeros_like(x)
    p = x.copy()
    for m in range(2, N + 1):
        p_prev, p = p, ((2 * m - 1) * x * p - (m - 1) * p_prev) / m
    return p, p_prev


def lgl_nodes_weights(n):
    """n GLL points on [-1, 1] (order N = n - 1) and their quadrature weights.

    The interior nodes are the roots of P_N'(x).  They are found by Newton's
    method on P_N' started from the Chebyshev-Gauss-Lobatto points; P_N' and
    P_N'' come from the recurrence pair and the Legendre ODE
    (1 - x^2) P'' = 2 x P' - N (N + 1) P.  Weights: w_i = 2 / (N (N+1) P_N(x_i)^2).
    """
    if n < 2:
        raise ValueError("need at least 2 GLL points")
    N = n - 1
    x = -np.cos(np.pi * np.arange(n) / N)
    if N >= 2:
        xi = x[1:-1].copy()
        for _ in range(200):
            p, q = legendre_pair(N, xi)
            dp = N * (xi * p - q) / (xi * xi - 1.0)
            d2p = (2.0 * xi * dp - N * (N + 1) * p) / (1.0 - xi * xi)
            step = dp / d2p
            xi = xi - step
            if np.max(np.abs(step)) < 1e-16:
                break
        x[1:-1] = xi
    x[0], x[-1] = -1.0, 1.0
    if n % 2 == 1:
        x[N // 2] = 0.0
    p, _ = legendre_pair(N, x)
    w = 2.0 / (N * (N + 1) * p * p)
    return x, w


def diff_matrix(x):
    """Nodal differentiation matrix D_ij = l_j'(x_i) of the GLL Lagrange basis.

    Off-diagonal entries use the closed form P_N(x_i) / (P_N(x_j) (x_i - x_j));
    each diagonal entry is minus the sum of its row's off-diagonals, so that
    D applied to a constant is exactly zero (the round-off-limiting form the
    paper points to, after Costa & Don).
    """
    n = len(x)
    N = n - 1
    p, _ = legendre_pair(N, x)
    D = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i != j:
                D[i, j] = p[i] / (p[j] * (x[i] - x[j]))
    for i in range(n):
        D[i, i] = -np.sum(D[i, :])
    return D
