"""Pins of the oracle's GLL nodes, weights and differentiation matrix (Sec. 2.2).

Pinned to tabulated closed forms (tests/golden), to quadrature exactness up to
degree 2N-1 and to exact differentiation of polynomials up to degree N.
"""
import os

import numpy as np
import pytest

from oracle.lgl import lgl_nodes_weights, diff_matrix

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _tabulated():
    out = {}
    with open(os.path.join(GOLDEN, "lgl_tabulated.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            vals = [float(t) for t in line.split()]
            n = int(vals[0])
            out[n] = (np.array(vals[1:1 + n]), np.array(vals[1 + n:1 + 2 * n]))
    return out


@pytest.mark.parametrize("n", [3, 4, 5, 6])
def test_nodes_weights_match_tables(n):
    x_ref, w_ref = _tabulated()[n]
    x, w = lgl_nodes_weights(n)
    np.testing.assert_allclose(x, x_ref, atol=2e-16 * 8)
    np.testing.assert_allclose(w, w_ref, atol=1e-15)


@pytest.mark.parametrize("n", [2, 5, 9, 13, 17, 21])
def test_quadrature_exact_to_degree_2N_minus_1(n):
    x, w = lgl_nodes_weights(n)
    N = n - 1
    assert abs(w.sum() - 2.0) < 1e-14
    for m in range(2 * N):
        exact = 0.0 if m % 2 else 2.0 / (m + 1)
        assert abs(np.dot(w, x ** m) - exact) < 1e-13, m
    # degree 2N is not integrated exactly (Lobatto rule): a sanity check the
    # test above is not vacuous
    assert abs(np.dot(w, x ** (2 * N)) - 2.0 / (2 * N + 1)) > 1e-12


def test_diff_matrix_N2_closed_form():
    D_ref = np.loadtxt(os.path.join(GOLDEN, "diff_matrix_N2.txt"))
    x, _ = lgl_nodes_weights(3)
    np.testing.assert_allclose(diff_matrix(x), D_ref, atol=1e-15)


@pytest.mark.parametrize("n", [3, 6, 9, 13, 17])
def test_diff_matrix_exact_on_polynomials(n):
    x, _ = lgl_nodes_weights(n)
    D = diff_matrix(x)
    N = n - 1
    assert np.abs(D @ np.ones(n)).max() < 1e-12
    for m in range(1, N + 1):
        err = np.abs(D @ x ** m - m * x ** (m - 1)).max()
        assert err < 1e-11 * N * N, (m, err)
    # endpoint diagonal entries of the Legendre collocation derivative
    assert abs(D[0, 0] + N * (N + 1) / 4.0) < 1e-10 * N * N
    assert abs(D[N, N] - N * (N + 1) / 4.0) < 1e-10 * N * N
