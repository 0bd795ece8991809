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


def test_concatenated_gmres_reaches_the_direct_solution():
    """Alg. 3d as printed (one GMRES on the stacked modes, Sec. 5) reaches the
    plain-definition solution of every mode (rfft, one direct 2-D solve per
    mode and part, irfft), mode 0's regularisation included; the stacked true
    Schur residual is at the GMRES tolerance."""
    from oracle import fourier
    from oracle.smpm import Grid
    g = Grid(6, 2, 6, 2.0, 1.0)
    my, ly = 8, 2.0 * np.pi
    f3 = np.random.default_rng(48).uniform(0, 1, (g.r, my))
    u_ref = fourier.solve_3d(g, f3, ly)
    u, info = fourier.solve_3d_concatenated(g, f3, ly, tol=1e-13)
    assert info["stacked_schur_residual"] < 1e-11
    assert np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref) < 1e-9
    assert np.abs(u - u_ref).max() / np.abs(u_ref).max() < 1e-9
