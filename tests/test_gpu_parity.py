"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerance: relative solution error 1e-9 in the 2-norm at a GMRES relative
Schur residual of 1e-10 (the oracle's own DBJ-at-1e-10 vs direct-solve floor
is ~1e-11 on these grids, see test_oracle_dbj).  Cases span several GEMM row
tiles, ragged column tiles and a ragged last vector chunk, both boundary strip
classes, odd and even m_x (single-interface last block-Jacobi block or not),
m_x = 2 and 3, stretched z, Helmholtz shifts, nonzero Neumann data, both
deflation groupings, batches of right-hand sides and host or device buffers.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle.smpm import Grid, direct_solve, gauge, assemble_L, rhs  # noqa: E402
from oracle import dbj  # noqa: E402

TOL = 1e-9


@pytest.fixture(scope="module")
def smpm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1512_01756_gb300 import smpm as m
    m.load()
    return m


def _gpu_solve(smpm, shape, f, k2=0.0, gb=None, groups=0, tol=1e-10, host=False, nrhs=1):
    mx, mz, order, lx, lz, zr = shape
    grid = smpm.make_grid(mx, mz, order, lx, lz, z_ratio=zr, deflation_groups=groups)
    s = smpm.Solver(grid, k2, torch.cuda.current_stream())
    if host:
        fh = np.ascontiguousarray(f)
        u = np.empty_like(fh)
        gh = None if gb is None else np.ascontiguousarray(gb)
        st = s.solve(fh, u, g=gh, tol=tol)
    else:
        fd = torch.from_numpy(np.ascontiguousarray(f)).cuda()
        ud = torch.empty_like(fd)
        gd = None if gb is None else torch.from_numpy(np.ascontiguousarray(gb)).cuda()
        st = s.solve(fd, ud, g=gd, tol=tol)
        torch.cuda.synchronize()
        u = ud.cpu().numpy()
    s.close()
    return u, st


def _rel(a, b):
    """Relative error in the 2-norm and in the max-norm, the larger of the two
    (a local error on one face of a long vector shows in the second)."""
    a, b = np.asarray(a), np.asarray(b)
    return max(np.linalg.norm(a - b) / np.linalg.norm(b), np.abs(a - b).max() / np.abs(b).max())


def _g_flat(gd):
    return np.concatenate([gd["west"], gd["east"], gd["south"], gd["north"]])


SHAPES = [
    (8, 2, 8, 4.0, 1.0, 1.0),      # config-1 shape
    (2, 3, 5, 1.0, 1.0, 1.0),      # two strips: both boundary classes only
    (3, 2, 4, 1.5, 1.0, 1.0),      # odd mx: all block-Jacobi blocks full pairs
    (7, 3, 6, 2.0, 1.0, 1.2),      # stretched z, odd mx
    (12, 4, 7, 3.0, 1.0, 1.0),     # nfz = 256: several GEMM row tiles
]


@pytest.mark.parametrize("shape", SHAPES)
def test_random_rhs_matches_direct(smpm, shape):
    g = Grid(*shape[:5], z_ratio=shape[5])
    f = np.random.default_rng(3).uniform(0, 1, g.r)
    u_ref, _ = direct_solve(g, f)
    u, st = _gpu_solve(smpm, shape, f)
    assert st.rel_resid_true <= 1e-10
    assert _rel(u, u_ref) < TOL, (_rel(u, u_ref), st.as_dict())


def test_config1_manufactured(smpm):
    from paper_1512_01756_gb300 import inputs
    shape = (8, 2, 8, 4.0, 1.0, 1.0)
    g = Grid(*shape[:5])
    X, Z = g.coords()
    f, u_ex = inputs.manufactured_cos(X, Z, 4.0, 1.0)
    u_ref, _ = direct_solve(g, f)
    for groups in (0, 1):
        u, st = _gpu_solve(smpm, shape, f, groups=groups)
        assert _rel(u, u_ref) < TOL
        # spectral accuracy against the exact solution (order 8)
        assert np.abs(u - gauge(g, u_ex)).max() < 1e-6


@pytest.mark.parametrize("k2", [0.01, 9.0, 1e4])
def test_helmholtz_matches_direct(smpm, k2):
    shape = (6, 3, 5, 2.0, 1.0, 1.2)
    g = Grid(*shape[:5], z_ratio=shape[5])
    f = np.random.default_rng(5).uniform(-1, 1, g.r)
    u_ref, _ = direct_solve(g, f, None, k2)
    u, st = _gpu_solve(smpm, shape, f, k2=k2)
    assert _rel(u, u_ref) < (1e-8 if k2 < 1 else TOL)


def test_neumann_data_polynomial_exact(smpm):
    """u = 0.3 x^3 - x z^2 + 0.5 z^3 + x z + 2 with its Neumann data is
    reproduced to round-off (checks the g layout and tau g terms)."""
    shape = (4, 3, 5, 2.0, 1.0, 1.2)
    g = Grid(*shape[:5], z_ratio=shape[5])
    X, Z = g.coords()
    u_ex = 0.3 * X ** 3 - X * Z ** 2 + 0.5 * Z ** 3 + X * Z + 2.0
    f = 1.8 * X - 2.0 * X + 3.0 * Z
    ux = lambda x, z: 0.9 * x ** 2 - z ** 2 + z
    uz = lambda x, z: -2.0 * x * z + 1.5 * z ** 2 + x
    zs, xs = g.z_nodes(), g.x_nodes()
    gb = np.concatenate([-ux(0.0, zs), ux(g.lx, zs), -uz(xs, 0.0), uz(xs, g.lz)])
    u, st = _gpu_solve(smpm, shape, f, gb=gb)
    assert np.abs(u - gauge(g, u_ex)).max() < 1e-8 * np.abs(u_ex).max()


def test_batch_equals_single_and_host_buffers(smpm):
    shape = (7, 3, 6, 2.0, 1.0, 1.2)
    g = Grid(*shape[:5], z_ratio=shape[5])
    R = 5
    F = np.random.default_rng(9).uniform(0, 1, (R, g.r))
    grid = smpm.make_grid(*shape[:5], z_ratio=shape[5])
    s = smpm.Solver(grid, 0.0, torch.cuda.current_stream())
    Fd = torch.from_numpy(F).cuda()
    Ud = torch.empty_like(Fd)
    st = s.solve(Fd, Ud, tol=1e-10)
    torch.cuda.synchronize()
    Ub = Ud.cpu().numpy()
    Uh = np.empty_like(F)
    s.solve(F, Uh, tol=1e-10)               # host pointers, staged by the library
    s.close()
    assert st.rel_resid_true <= 1e-10
    for r in range(R):
        u1, _ = _gpu_solve(smpm, shape, F[r])
        assert _rel(Ub[r], u1) < 1e-11
        assert _rel(Uh[r], u1) < 1e-11
        u_ref, _ = direct_solve(g, F[r])
        assert _rel(Ub[r], u_ref) < TOL


def test_many_tiles_ragged_chunks_vs_iterative_oracle(smpm):
    """40 x 3 elements, order 7: 40 strips (two column tiles per class run),
    kp = 1920 (a full and a ragged vector chunk), 192-row strip GEMMs."""
    shape = (40, 3, 7, 10.0, 1.0, 1.0)
    g = Grid(*shape[:5])
    f = np.random.default_rng(11).uniform(0, 1, g.r)
    u_ref, info = dbj.solve(g, f, method="dbj", tol=1e-13)
    u, st = _gpu_solve(smpm, shape, f)
    assert st.rel_resid_true <= 1e-10
    assert _rel(u, u_ref) < TOL
    # full-system residual (Claim 2 bounds it by the Schur residual in exact
    # arithmetic) of the GPU solution with the oracle's own L.  The recovery
    # applies an explicit strip inverse, whose product is accurate but not
    # residual-minimal (~eps cond(A_c) rather than the ~eps of an LU solve), so
    # the bound here is 1e-8 while the solution error above stays below 1e-9.
    L = assemble_L(g)
    b = info["b"]
    res_gpu = np.linalg.norm(L @ u - b) / np.linalg.norm(b)
    assert res_gpu < 1e-8, res_gpu


def test_multi_operator_modes(smpm):
    """Three k^2 values (one of them 0) solved in one batched pass equal the
    per-mode oracle solves (the batched 3-D form of Alg. 3d)."""
    shape = (6, 2, 5, 2.0, 1.0, 1.0)
    g = Grid(*shape[:5])
    k2s = np.array([0.0, 1.0, 4.0])
    ops = np.array([0, 0, 1, 1, 2, 2], dtype=np.int32)
    F = np.random.default_rng(13).uniform(-1, 1, (len(ops), g.r))
    grid = smpm.make_grid(*shape[:5])
    s = smpm.Solver(grid, k2s, torch.cuda.current_stream())
    Fd = torch.from_numpy(F).cuda()
    Ud = torch.empty_like(Fd)
    st = s.solve_multi(ops, Fd, Ud, tol=1e-10)
    torch.cuda.synchronize()
    U = Ud.cpu().numpy()
    s.close()
    for i, o in enumerate(ops):
        u_ref, _ = direct_solve(g, F[i], None, float(k2s[o]))
        assert _rel(U[i], u_ref) < TOL, (i, o)


def test_invalid_arguments(smpm):
    with pytest.raises(smpm.SmpmError):
        smpm.Solver(smpm.make_grid(1, 2, 4, 1.0, 1.0), 0.0)
    with pytest.raises(smpm.SmpmError):
        smpm.Solver(smpm.make_grid(4, 2, 4, 1.0, 1.0), -1.0)
