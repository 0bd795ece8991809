"""The tridiagonal path of the coarse division (one deflation vector per
interface, k^2 > 0: C is tridiagonal and nonsingular, K = C^-1 from a pivoted
tridiagonal LU and one GPU thread per column; Sec. 3.3) against the dense
factorisation of the same C (SMPM_COARSE_DENSE=1): the deflation projection
P x = x - S Z K Z^T x at 1e-12, and solves through it against the oracle at
1e-9.  k^2 = 0 keeps the dense regularised division on both settings."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.smpm import Grid, direct_solve  # noqa: E402


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


SHAPES = [((2, 2, 6, 1.0, 1.0, 1.0), 3.0),      # d = 1
          ((3, 2, 6, 1.5, 1.0, 1.0), 0.7),      # d = 2
          ((8, 2, 8, 4.0, 1.0, 1.0), 5.0),
          ((12, 3, 7, 3.0, 1.0, 1.2), 0.05),
          ((64, 2, 6, 32.0, 1.0, 1.0), 30.0),
          ((64, 2, 6, 32.0, 1.0, 1.0), 0.0)]


@pytest.mark.parametrize("shape,k2", SHAPES)
def test_tridiagonal_coarse_matches_dense(smpm, monkeypatch, shape, k2):
    mx, mz, order, lx, lz, zr = shape
    out = {}
    for dense in (False, True):
        if dense:
            monkeypatch.setenv("SMPM_COARSE_DENSE", "1")
        else:
            monkeypatch.delenv("SMPM_COARSE_DENSE", raising=False)
        s = smpm.Solver(smpm.make_grid(mx, mz, order, lx, lz, z_ratio=zr), k2)
        X = np.random.default_rng(91).standard_normal((6, s.k))
        Y = np.zeros_like(X)
        s.apply("P", X, Y)
        s.close()
        out[dense] = Y
    for i in range(6):
        assert _rel(out[False][i], out[True][i]) < 1e-12, (i, _rel(out[False][i], out[True][i]))


@pytest.mark.parametrize("shape,k2", [s for s in SHAPES if s[0][0] <= 12])
def test_tridiagonal_coarse_solve_matches_oracle(smpm, monkeypatch, shape, k2):
    monkeypatch.delenv("SMPM_COARSE_DENSE", raising=False)
    mx, mz, order, lx, lz, zr = shape
    g = Grid(mx, mz, order, lx, lz, z_ratio=zr)
    F = np.random.default_rng(92).uniform(0, 1, (2, g.r))
    s = smpm.Solver(smpm.make_grid(mx, mz, order, lx, lz, z_ratio=zr), k2)
    U = np.zeros_like(F)
    st = s.solve(F, U, tol=1e-10)
    s.close()
    assert st.status == 0 and st.rel_resid_true <= 1e-10
    for i in range(2):
        u_ref, _ = direct_solve(g, F[i], None, k2)
        assert _rel(U[i], u_ref) < 1e-9, (i, _rel(U[i], u_ref))
