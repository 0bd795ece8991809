"""Slot inverses of uniform-z grids from their two half-size mirror blocks
(Sec. 5 strip solver; each slot matrix L_z + s I commutes with the reversal
of the z-nodes): a handle with 16 k^2 inverts every half of one size in one
Gauss-Jordan launch (the 170-row halves of the 2 x 2 slots in the
global-memory form, the 85-row halves in shared memory), a single-k^2
handle inverts its few large halves with cuSOLVER.  The 16-operator batched
solve must equal each request solved alone (1e-9) and the oracle's DBJ solve
(1e-9), 2-norm and max-norm."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.smpm import Grid  # noqa: E402
from oracle import dbj  # noqa: E402


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


def test_batched_halves_match_single_and_oracle(smpm):
    shape = (4, 10, 16, 0.4, 1.0)            # f_z = 170: 2 x 2 slot halves of 170 rows, 1 x 1 of 85
    g = Grid(*shape)
    k2 = np.exp(np.linspace(np.log(0.05), np.log(5e3), 16))
    F = np.random.default_rng(97).uniform(0, 1, (16, g.r))
    s = smpm.Solver(smpm.make_grid(*shape), k2)
    U = np.zeros_like(F)
    st = s.solve_multi(np.arange(16, dtype=np.int32), F, U, tol=1e-10)
    s.close()
    assert st.status == 0 and st.rel_resid_true <= 1e-10, st.as_dict()
    for i in (0, 7, 15):
        s1 = smpm.Solver(smpm.make_grid(*shape), float(k2[i]))
        u1 = np.zeros(g.r)
        st1 = s1.solve(F[i], u1, tol=1e-10)
        s1.close()
        assert st1.status == 0 and st1.rel_resid_true <= 1e-10
        assert _rel(U[i], u1) < 1e-9, (i, _rel(U[i], u1))
    u_ref, info = dbj.solve(g, F[7], k2=float(k2[7]), method="dbj", tol=1e-13)
    assert info["schur_residual"] < 1e-11
    assert _rel(U[7], u_ref) < 1e-9, _rel(U[7], u_ref)
