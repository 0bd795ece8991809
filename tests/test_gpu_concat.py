"""One concatenated Krylov space over every right-hand side of a call
(smpm_grid.krylov = 1; Sec. 5, Implementation, and Alg. 3d line 7: all
wavenumbers solved in one GMRES, every dot product and norm summed over the
modes, one convergence test on the whole residual).

* 3-D: all Fourier modes of a small y-periodic problem (mode 0 with its
  regularisation among them) against the oracle's mode-by-mode direct solve
  and against the per-mode Krylov path, at 1e-9 relative (2-norm and
  max-norm over the whole field).
* 2-D batches of right-hand sides of similar norm, Poisson and Helmholtz, on
  uniform and stretched z: each column against the oracle at 1e-9.
* The serving runtime refuses krylov = 1 (SMPM_EINVAL).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.smpm import Grid, direct_solve  # noqa: E402
from oracle import fourier  # noqa: E402


@pytest.fixture(scope="module")
def smpm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1512_01756_gb300 import smpm as m
    m.load()
    return m


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return max(np.linalg.norm(a - b) / np.linalg.norm(b), np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("shape,my", [((6, 2, 6, 2.0, 1.0), 8), ((8, 2, 8, 4.0, 1.0), 12)])
def test_concatenated_modes_match_oracle_and_per_mode(smpm, shape, my):
    g = Grid(*shape)
    ly = 2.0 * np.pi
    f3 = np.random.default_rng(71).uniform(0, 1, (g.r, my))
    u_ref = fourier.solve_3d(g, f3, ly)
    out, its = {}, {}
    for krylov in (1, 0):
        s = smpm.Solver3D(smpm.make_grid(*shape, krylov=krylov), my, ly)
        u3 = np.zeros((my, g.r))
        st = s.solve_3d_physical(np.ascontiguousarray(f3.T), u3, tol=1e-10)
        s.close()
        assert st.status == 0 and st.rel_resid_true <= 1e-10, (krylov, st.as_dict())
        out[krylov], its[krylov] = u3.T, st.iters
    print(f"iterations: concatenated {its[1]}, per mode (max) {its[0]}")
    assert _rel(out[1], u_ref) < 1e-9, _rel(out[1], u_ref)
    assert _rel(out[1], out[0]) < 1e-9


@pytest.mark.parametrize("shape,k2", [((8, 2, 8, 4.0, 1.0, 1.0), 0.0), ((12, 3, 7, 3.0, 1.0, 1.2), 0.0),
                                      ((10, 2, 6, 2.5, 1.0, 1.0), 40.0)])
def test_concatenated_batch_matches_oracle(smpm, shape, k2):
    mx, mz, order, lx, lz, zr = shape
    g = Grid(mx, mz, order, lx, lz, z_ratio=zr)
    F = np.random.default_rng(72).uniform(0, 1, (4, g.r))
    s = smpm.Solver(smpm.make_grid(mx, mz, order, lx, lz, z_ratio=zr, krylov=1), k2)
    U = np.zeros_like(F)
    st = s.solve(F, U, tol=1e-10)
    s.close()
    assert st.status == 0 and st.rel_resid_true <= 1e-10, st.as_dict()
    assert st.iters > 0
    for i in range(4):
        u_ref, _ = direct_solve(g, F[i], None, k2)
        assert _rel(U[i], u_ref) < 1e-9, (i, _rel(U[i], u_ref))


def test_server_refuses_concatenated(smpm):
    srv = smpm.Server(nworkers=1)
    f = np.zeros(Grid(8, 2, 6, 4.0, 1.0).r)
    with pytest.raises(smpm.SmpmError) as e:
        srv.submit(smpm.make_grid(8, 2, 6, 4.0, 1.0, krylov=1), 0.0, f, np.zeros_like(f))
    assert e.value.code == smpm.SMPM_EINVAL
    srv.close()


def test_bad_krylov_is_einval(smpm):
    with pytest.raises(smpm.SmpmError) as e:
        smpm.Solver(smpm.make_grid(8, 2, 6, 4.0, 1.0, krylov=2), 0.0)
    assert e.value.code == smpm.SMPM_EINVAL
