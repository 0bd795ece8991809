"""GPU parity of the batched Fourier-mode solve (Sec. 5, Alg. 3d).

* Small 3-D problem: the y-DFT is taken here (numpy, test harness), all
  my/2+1 modes are solved in one smpm_solve_3d call, the inverse DFT gives the
  3-D field, compared with the oracle's per-mode direct solves.
* Full-size workload shape (128 x 8 elements, order 10, domain 32 x 1,
  m_y = 128 -> 65 modes, k_j = j): a separable manufactured solution carried
  by the k = 3 mode is recovered to spectral accuracy, and for the paper's
  U[0,1] right-hand side every mode's GPU solution satisfies the oracle's own
  assembled (L - k_j^2) system (a property that holds at any size), and
  sampled modes equal the oracle's own DBJ solves at the 1e-9 bar (the GPU
  solved to 1e-11 there, as a solution at residual 1e-10 is only accurate to
  kappa * 1e-10 on this long domain).

Mode 0 of U[0,1] data is incompatible (mean ~0.5): Eq. regularize_poisson
removes its u_L component, which is most of the vector, so the projected data
moves with u_L, and u_L is fixed by L only to ~eps / (sigma_2 / sigma_1) on a
32-long domain.  The library's and the oracle's null vectors (both with
|L^T u_L| ~ 1e-17) put the mode-0 solutions 2.5e-5 apart -- the problem's
conditioning, not an error of either.  Mode 0 is therefore compared with the
oracle on the same data made consistent with the oracle's u_L beforehand
(the library's projection then moves it only to second order), and by
residual in the oracle's system as given.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.smpm import Grid, assemble_L  # noqa: E402
from oracle import fourier  # noqa: E402


def _rel(a, b):
    """Relative error in the 2-norm and in the max-norm, the larger of the two
    (a local error on one face of a long vector shows in the second)."""
    a, b = np.asarray(a), np.asarray(b)
    return max(np.linalg.norm(a - b) / np.linalg.norm(b), np.abs(a - b).max() / np.abs(b).max())


@pytest.fixture(scope="module")
def smpm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1512_01756_gb300 import smpm as m
    m.load()
    return m


def _stack(fh):
    """complex [r, n_modes] -> [n_modes, 2, r] float64"""
    return np.ascontiguousarray(np.stack([fh.real.T, fh.imag.T], axis=1))


def _unstack(U):
    return (U[:, 0, :] + 1j * U[:, 1, :]).T


def test_small_3d_matches_oracle(smpm):
    shape = (6, 2, 6, 2.0, 1.0)
    g = Grid(*shape)
    my, ly = 8, 2.0 * np.pi
    f3 = np.random.default_rng(17).uniform(0, 1, (g.r, my))
    u_ref = fourier.solve_3d(g, f3, ly)
    s = smpm.Solver3D(smpm.make_grid(*shape), my, ly, torch.cuda.current_stream())
    Fh = torch.from_numpy(_stack(fourier.forward(f3))).cuda()
    Uh = torch.empty_like(Fh)
    st = s.solve_3d(Fh, Uh, tol=1e-10)
    torch.cuda.synchronize()
    s.close()
    u = fourier.inverse(_unstack(Uh.cpu().numpy()), my)
    assert st.rel_resid_true <= 1e-10
    assert _rel(u, u_ref) < 1e-9


@pytest.fixture(scope="module")
def full3d(smpm):
    shape = (128, 8, 10, 32.0, 1.0)
    s = smpm.Solver3D(smpm.make_grid(*shape), 128, 2.0 * np.pi, torch.cuda.current_stream())
    yield shape, s
    s.close()


def test_full_size_separable_manufactured(smpm, full3d):
    shape, s = full3d
    g = Grid(*shape)
    X, Z = g.coords()
    my = 128
    y = np.arange(my) * 2.0 * np.pi / my
    u2 = np.cos(np.pi * X / 32.0) * np.cos(np.pi * Z)
    u3 = u2[:, None] * np.cos(3.0 * y)[None, :]
    f3 = -(np.pi ** 2 / 32.0 ** 2 + np.pi ** 2 + 9.0) * u3
    Fh = torch.from_numpy(_stack(fourier.forward(f3))).cuda()
    Uh = torch.empty_like(Fh)
    st = s.solve_3d(Fh, Uh, tol=1e-10)
    torch.cuda.synchronize()
    u = fourier.inverse(_unstack(Uh.cpu().numpy()), my)
    assert st.rel_resid_true <= 1e-10
    assert np.abs(u - u3).max() < 1e-7


def test_full_size_modes_satisfy_oracle_systems(smpm, full3d):
    shape, s = full3d
    g = Grid(*shape)
    my = 128
    f3 = np.random.default_rng(20151208).uniform(0, 1, (g.r, my))
    fh = fourier.forward(f3)
    Fh = torch.from_numpy(_stack(fh)).cuda()
    Uh = torch.empty_like(Fh)
    st = s.solve_3d(Fh, Uh, tol=1e-10)
    torch.cuda.synchronize()
    assert st.rel_resid_true <= 1e-10
    uh = _unstack(Uh.cpu().numpy())
    L = assemble_L(g)
    ks = fourier.wavenumbers(my, 2.0 * np.pi)
    from oracle.schur import left_null_sparse
    uL = left_null_sparse(L)
    for j in range(len(ks)):
        for part in (np.real, np.imag):
            b = part(fh[:, j]).copy()
            if not np.any(b):
                continue
            if j == 0:
                b = b - uL * np.dot(uL, b)
            r = (L @ part(uh[:, j]) - ks[j] ** 2 * part(uh[:, j])) - b
            assert np.linalg.norm(r) / np.linalg.norm(b) < 1e-8, (j, np.linalg.norm(r) / np.linalg.norm(b))
    # the zero mode is returned with zero quadrature mean
    assert abs(np.dot(g.quad_weights(), uh[:, 0].real)) < 1e-10 * np.abs(uh[:, 0].real).max()


def test_full_size_sampled_modes_match_oracle(smpm, full3d):
    from oracle import dbj
    from oracle.schur import StripSchur
    shape, s = full3d
    g = Grid(*shape)
    my = 128
    f3 = np.random.default_rng(20151209).uniform(0, 1, (g.r, my))
    fh = fourier.forward(f3)
    Fh = torch.from_numpy(_stack(fh)).cuda()
    Uh = torch.empty_like(Fh)
    st = s.solve_3d(Fh, Uh, tol=1e-11)
    torch.cuda.synchronize()
    assert st.rel_resid_true <= 1e-11
    uh = _unstack(Uh.cpu().numpy())
    ks = fourier.wavenumbers(my, 2.0 * np.pi)
    for j in (1, 64):
        sch = StripSchur(g, ks[j] ** 2)
        for part in (np.real, np.imag):
            b = part(fh[:, j]).copy()
            if not np.any(b):
                continue
            u_ref, _ = dbj.solve(g, b, k2=ks[j] ** 2, method="dbj", tol=1e-13, schur=sch, coarse="rank1")
            u = part(uh[:, j])
            rel = _rel(u, u_ref)
            print(f"mode {j} {part.__name__}: rel {rel:.2e}")
            assert rel < 1e-9, (j, part.__name__, rel)
    # mode 0 as given (the paper's U[0,1] data, mostly incompatible: each side
    # projects it with its own left null vector, Eq. regularize_poisson)
    b0_raw = fh[:, 0].real.copy()
    u_ref0, _ = dbj.solve(g, b0_raw, method="dbj", tol=1e-13, coarse="rank1")
    rel0 = _rel(uh[:, 0].real, u_ref0)
    print(f"mode 0 (as given): rel {rel0:.2e}")
    # the data is far from compatible (mean ~0.5), so the projection removes
    # most of it and the result moves with the left null vector: in the oracle
    # alone, perturbing the entries of L by one rounding unit moves this
    # solution by 0.8e-9 to 3.9e-9; the two independently computed null
    # vectors are held to 1e-8
    assert rel0 < 1e-8, rel0
    # mode 0 made consistent first (its component along the oracle's u_L
    # removed, Eq. regularize_poisson), through a 2-D handle of the grid
    from oracle.schur import left_null_sparse
    uL = left_null_sparse(assemble_L(g))
    b0 = fh[:, 0].real.copy()
    b0 -= uL * np.dot(uL, b0)
    s2 = smpm.Solver(smpm.make_grid(*shape), 0.0)
    u0 = np.zeros_like(b0)
    st0 = s2.solve(b0, u0, tol=1e-11)
    s2.close()
    assert st0.rel_resid_true <= 1e-11
    u_ref, _ = dbj.solve(g, b0, method="dbj", tol=1e-13, coarse="rank1")
    rel = _rel(u0, u_ref)
    print(f"mode 0 (consistent): rel {rel:.2e}")
    assert rel < 1e-9, rel


def test_small_3d_physical_matches_oracle(smpm):
    """The physical-space call (y-DFTs on the GPU around the batched mode
    solve) against the oracle's rfft / per-mode direct solve / irfft route,
    with Neumann data on the x and z faces varying in y."""
    shape = (6, 2, 6, 2.0, 1.0)
    g = Grid(*shape)
    my, ly = 8, 2.0 * np.pi
    rng = np.random.default_rng(18)
    f3 = rng.uniform(0, 1, (g.r, my))
    u_ref = fourier.solve_3d(g, f3, ly)
    s = smpm.Solver3D(smpm.make_grid(*shape), my, ly)
    u3 = np.zeros((my, g.r))
    st = s.solve_3d_physical(np.ascontiguousarray(f3.T), u3, tol=1e-10)
    s.close()
    assert st.rel_resid_true <= 1e-10
    assert _rel(u3.T, u_ref) < 1e-9


def test_full_size_physical_separable_manufactured(smpm, full3d):
    shape, s = full3d
    g = Grid(*shape)
    X, Z = g.coords()
    my = 128
    y = np.arange(my) * 2.0 * np.pi / my
    u2 = np.cos(np.pi * X / 32.0) * np.cos(np.pi * Z)
    u3 = u2[None, :] * np.cos(5.0 * y)[:, None] + 0.5 * u2[None, :] * np.sin(2.0 * y)[:, None]
    lap = -(np.pi ** 2 / 32.0 ** 2 + np.pi ** 2)
    f3 = u2[None, :] * ((lap - 25.0) * np.cos(5.0 * y)[:, None] + 0.5 * (lap - 4.0) * np.sin(2.0 * y)[:, None])
    F = torch.from_numpy(np.ascontiguousarray(f3)).cuda()
    U = torch.empty_like(F)
    st = s.solve_3d_physical(F, U, tol=1e-10)
    torch.cuda.synchronize()
    assert st.rel_resid_true <= 1e-10
    assert np.abs(U.cpu().numpy() - u3).max() < 1e-7
