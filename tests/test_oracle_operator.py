"""Pins of the oracle's SMPM operator (Sec. 2.2, Eq. smpm_poisson).

* Polynomial exactness: a polynomial of degree <= N in each variable is
  reproduced to round-off (the Laplacian is exact, every interface penalty
  vanishes on a C^1 function, every Neumann penalty vanishes for g = n.grad u).
  A wrong sign, a dropped edge term, a wrong normal or a wrong element
  mapping anywhere in the assembly breaks it.
* L 1 = 0 (constant right null vector), a one-dimensional null space.
* The Kronecker-sum structure L = L_x (+) L_z that follows from the
  corner-node and per-edge tau readings (the assembly does not use it).
* Spectral convergence to the manufactured cos-cos solution (config 1 shape).
"""
import numpy as np
import pytest

from oracle.smpm import Grid, assemble_L, rhs, direct_solve, gauge, left_null_dense


def _poly(x, z, lx, lz, k2=0.0):
    """u = 0.3 x^3 - x z^2 + 0.5 z^3 + x z + 2 with its f and Neumann data."""
    u = 0.3 * x ** 3 - x * z ** 2 + 0.5 * z ** 3 + x * z + 2.0
    f = (1.8 * x - 2.0 * x + 3.0 * z) - k2 * u
    ux = lambda x_, z_: 0.9 * x_ ** 2 - z_ ** 2 + z_
    uz = lambda x_, z_: -2.0 * x_ * z_ + 1.5 * z_ ** 2 + x_
    return u, f, ux, uz


def _g_of(g, ux, uz):
    zs, xs = g.z_nodes(), g.x_nodes()
    return {"west": -ux(0.0, zs), "east": ux(g.lx, zs),
            "south": -uz(xs, 0.0), "north": uz(xs, g.lz)}


@pytest.mark.parametrize("shape", [(3, 2, 3, 1.5, 1.0, 1.0), (4, 3, 5, 2.0, 1.0, 1.2),
                                   (2, 4, 6, 0.7, 1.3, 0.8)])
@pytest.mark.parametrize("k2", [0.0, 7.5])
def test_polynomial_reproduced_exactly(shape, k2):
    mx, mz, order, lx, lz, zr = shape
    g = Grid(mx, mz, order, lx, lz, z_ratio=zr)
    X, Z = g.coords()
    u_ex, f, ux, uz = _poly(X, Z, lx, lz, k2)
    gb = _g_of(g, ux, uz)
    L = assemble_L(g, k2)
    # the exact polynomial satisfies every collocation row
    res = L @ u_ex - rhs(g, f, gb)
    assert np.abs(res).max() < 1e-9 * np.abs(L).max()
    u, _ = direct_solve(g, f, gb, k2)
    ref = gauge(g, u_ex) if k2 == 0.0 else u_ex
    assert np.abs(u - ref).max() < 1e-9 * np.abs(ref).max()


def test_wrong_sign_would_fail():
    """The polynomial pin is sensitive: flipping the sign of g breaks it."""
    g = Grid(3, 2, 4, 1.5, 1.0)
    X, Z = g.coords()
    u_ex, f, ux, uz = _poly(X, Z, g.lx, g.lz)
    gb = _g_of(g, ux, uz)
    bad = {k: -v for k, v in gb.items()}
    u, _ = direct_solve(g, f, bad)
    assert np.abs(u - gauge(g, u_ex)).max() > 1e-3


@pytest.mark.parametrize("shape", [(8, 2, 8, 4.0, 1.0, 1.0), (3, 5, 6, 1.0, 2.0, 1.2)])
def test_constant_null_space(shape):
    mx, mz, order, lx, lz, zr = shape
    g = Grid(mx, mz, order, lx, lz, z_ratio=zr)
    L = assemble_L(g)
    assert np.abs(L @ np.ones(g.r)).max() < 1e-10 * abs(L).max()
    uL, s = left_null_dense(L.toarray())
    assert s[-1] / s[0] < 1e-14
    assert s[-2] / s[0] > 1e-9                      # one-dimensional
    assert np.linalg.norm(uL @ L) < 1e-14 * abs(L).max()


@pytest.mark.parametrize("k2", [0.0, 30.0])
def test_kronecker_sum_structure(k2):
    g = Grid(4, 3, 5, 2.0, 1.0, z_ratio=1.2)
    L = assemble_L(g, k2).toarray().reshape(g.nx, g.fz, g.nx, g.fz)
    Lx = L[:, 0, :, 0].copy()
    Lz = L[0, :, 0, :].copy()
    for Z in range(g.fz):
        Lz[Z, Z] = L[0, Z, 0, Z] - Lx[0, 0]
    K = np.einsum("ac,bd->abcd", Lx, np.eye(g.fz)) + np.einsum("ac,bd->abcd", np.eye(g.nx), Lz)
    assert np.abs(K - L).max() < 1e-12 * np.abs(L).max()


def test_spectral_convergence_config1_shape():
    errs = []
    orders = [4, 6, 8, 10, 12]
    for order in orders:
        g = Grid(8, 2, order, 4.0, 1.0)
        X, Z = g.coords()
        ue = np.cos(np.pi * X / 4) * np.cos(np.pi * Z)
        f = -(np.pi ** 2 / 16 + np.pi ** 2) * ue
        u, info = direct_solve(g, f)
        errs.append(np.abs(u - gauge(g, ue)).max())
        # continuous compatibility -> discrete consistency to spectral accuracy
        assert abs(np.dot(info["uL"], f)) / np.linalg.norm(f) < 1e-6
    errs = np.array(errs)
    assert errs[0] > 1e-4 and errs[-1] < 1e-9
    # geometric decay in the order until the round-off plateau (~1e-10 here)
    assert np.all(errs[1:4] < errs[:3] * 1e-2)


def test_helmholtz_spectral_convergence():
    k2 = 9.0
    errs = []
    for order in [4, 8, 12]:
        g = Grid(4, 2, order, 2.0, 1.0, z_ratio=1.2)
        X, Z = g.coords()
        ue = np.cos(np.pi * X / 2) * np.cos(np.pi * Z)
        f = -(np.pi ** 2 / 4 + np.pi ** 2 + k2) * ue
        u, _ = direct_solve(g, f, None, k2)
        errs.append(np.abs(u - ue).max())
    assert errs[0] > 1e-5 and errs[-1] < 1e-9 and errs[1] < errs[0] * 1e-2


def _one_d_spectra(mx, mz, order, hx, lz, zr, tau_scale):
    """Eigenvalues of the 1-D factors of L = L_x (+) L_z (pinned by
    test_kronecker_sum_structure): L_x from a one-element-row grid with m_x
    elements of length hx, L_z from a two-strip grid with the m_z elements of
    the z-mesh.  Each diagonal block read out of L carries the other factor's
    constant diagonal shift; L_x 1 = L_z 1 = 0 gives that shift."""
    out = []
    for g, idx in ((Grid(mx, 1, order, mx * hx, 1.0, tau_scale=tau_scale), "x"),
                   (Grid(2, mz, order, 1.0, lz, z_ratio=zr, tau_scale=tau_scale), "z")):
        L = assemble_L(g).tocsr()
        sel = np.arange(g.nx) * g.fz if idx == "x" else np.arange(g.fz)
        M = L[sel][:, sel].toarray()
        shift = (M @ np.ones(M.shape[0]))[0]
        out.append(np.linalg.eigvals(M) - shift)
    return out


# element shapes of every workload: (m_x used for L_x, m_z, order, h_x, l_z, z_ratio)
PENALTY_SHAPES = [
    (8, 2, 8, 0.5, 1.0, 1.0),        # 8 x 2 elements on 4 x 1, order 8
    (16, 4, 12, 0.25, 1.0, 1.0),     # 256 x 4 on 64 x 1, order 12
    (16, 8, 10, 0.25, 1.0, 1.0),     # 128 x 8 on 32 x 1, order 10 (the Fourier-mode problems)
    (16, 16, 16, 0.0625, 1.0, 1.2),  # 512 x 16 on 32 x 1, order 16, z stretched by 1.2
    (16, 16, 16, 0.0625, 1.0, 1.0),  # 1024 x 16 on 64 x 1, order 16 (serving)
    (16, 16, 12, 0.0625, 1.0, 1.0),  # 512 x 16 / 1024 x 16, order 12 (serving)
    (16, 8, 16, 0.125, 1.0, 1.0),    # 256 x 8 on 32 x 1, order 16 (serving)
    (16, 2, 6, 0.5, 1.0, 1.0),       # 64 x 2 on 32 x 1, order 6 (serving)
]


@pytest.mark.parametrize("shape", PENALTY_SHAPES)
def test_default_penalty_has_no_antidamped_modes(shape):
    """Stability reading of tau: at the default tau_scale no eigenvalue of the
    SMPM operator has a positive real part on the element shapes of every
    workload, orders 6 to 16 and element lengths 1/88 to 1/2 included (so
    every Helmholtz shift k^2 > 0 gives a definite problem).  The spectrum of
    L is the set of sums of the two 1-D spectra, so both are checked."""
    mx, mz, order, hx, lz, zr = shape
    for ev in _one_d_spectra(mx, mz, order, hx, lz, zr, -0.1):
        assert ev.real.max() < 1e-12 * np.abs(ev).max()


@pytest.mark.parametrize("shape", [(16, 16, 16, 0.0625, 1.0, 1.0), (16, 8, 12, 0.125, 1.0, 1.0)])
def test_penalty_pin_is_sensitive(shape):
    """The check above fails for a penalty that is too weak or of the wrong
    sign: tau_scale = -0.02 (below the ~0.028 threshold) and +0.1 both leave
    jump modes with a positive real part."""
    mx, mz, order, hx, lz, zr = shape
    for ts in (-0.02, 0.1):
        worst = max(ev.real.max() / np.abs(ev).max() for ev in _one_d_spectra(mx, mz, order, hx, lz, zr, ts))
        assert worst > 1e-6


@pytest.mark.parametrize("shape", [(8, 2, 8, 4.0, 1.0, 1.0), (8, 4, 12, 2.0, 1.0, 1.0), (4, 4, 10, 1.0, 1.0, 1.2)])
def test_default_penalty_full_spectrum(shape):
    """The same stability statement on the full assembled L of small grids
    (no use of the Kronecker structure)."""
    mx, mz, order, lx, lz, zr = shape
    ev = np.linalg.eigvals(assemble_L(Grid(mx, mz, order, lx, lz, z_ratio=zr)).toarray())
    assert ev.real.max() < 1e-8 * np.abs(ev).max()
