"""Pins of the oracle's 3-D Fourier extension (Sec. 5, Alg. 3d).

A separable manufactured solution u = cos(pi x/l_x) cos(pi z) cos(3 y) is
recovered to spectral accuracy (the k^2 = 9 mode carries it), and every mode's
solution equals the 2-D Helmholtz solve for that wavenumber.
"""
import numpy as np

from oracle.smpm import Grid, direct_solve
from oracle import fourier


def test_separable_manufactured_3d():
    g = Grid(4, 2, 10, 2.0, 1.0)
    my, ly = 8, 2.0 * np.pi
    X, Z = g.coords()
    y = np.arange(my) * ly / my
    u2 = np.cos(np.pi * X / 2.0) * np.cos(np.pi * Z)
    u3 = u2[:, None] * np.cos(3.0 * y)[None, :]
    f3 = -(np.pi ** 2 / 4.0 + np.pi ** 2 + 9.0) * u3
    u = fourier.solve_3d(g, f3, ly)
    assert np.abs(u - u3).max() < 1e-8


def test_modes_are_2d_helmholtz_solves():
    g = Grid(3, 2, 5, 1.5, 1.0)
    my, ly = 6, 2.0 * np.pi
    rng = np.random.default_rng(2)
    f3 = rng.uniform(0, 1, (g.r, my))
    fh = fourier.forward(f3)
    uh = fourier.solve_modes(g, fh, ly)
    ks = fourier.wavenumbers(my, ly)
    assert np.allclose(ks, np.arange(my // 2 + 1))
    for j in range(my // 2 + 1):
        ur, _ = direct_solve(g, fh[:, j].real, None, float(ks[j] ** 2))
        assert np.abs(uh[:, j].real - ur).max() < 1e-12 * max(1.0, np.abs(ur).max())
    # Nyquist and mean modes of real data are real
    assert np.abs(fh[:, 0].imag).max() == 0.0 and np.abs(fh[:, -1].imag).max() < 1e-15
