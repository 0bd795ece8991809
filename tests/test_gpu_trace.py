"""Tracing: the residual history of the last solve (smpm_residual_history).

* kind 1, the recomputed true residual ||S x_S - b_S|| / ||b_S|| at every
  restart-cycle start: it starts at 1 (zero guess), ends at the solve's
  final relative residual (smpm_last_residuals) below tol, and several
  cycles appear when the restart length is short.
* kind 0, the GMRES residual estimate from the Givens rotations after every
  Arnoldi step (written on the device): one value per step, non-increasing
  within a cycle (GMRES minimises the residual over a growing space), the
  last one of a converged single-cycle solve at or below tol.
* Bad arguments are SMPM_EINVAL.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.smpm import Grid  # noqa: E402


@pytest.fixture(scope="module")
def smpm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1512_01756_gb300 import smpm as m
    m.load()
    return m


@pytest.mark.parametrize("restart,precision", [(64, 0), (4, 0), (64, 2)])
def test_residual_history(smpm, restart, precision):
    shape = (16, 2, 8, 8.0, 1.0)
    g = Grid(*shape)
    F = np.random.default_rng(95).uniform(0, 1, (2, g.r))
    s = smpm.Solver(smpm.make_grid(*shape, restart=restart, precision=precision), 0.3)
    U = np.zeros_like(F)
    st = s.solve(F, U, tol=1e-10)
    assert st.status == 0
    final = s.last_residuals(2)
    for r in range(2):
        true = s.residual_history(r, kind=1)
        assert len(true) >= 1 and abs(true[0] - 1.0) < 1e-12, true
        assert abs(true[-1] - final[r]) <= 1e-15 + 1e-12 * final[r] and true[-1] <= 1e-10
        if restart == 4:
            assert len(true) >= 2
        est = s.residual_history(r, kind=0)
        assert 1 <= len(est) <= st.iters
        first = est[:min(restart, len(est))]
        assert np.all(np.diff(first) <= 1e-14 * first[:-1] + 1e-300), first
        if len(true) == 2 and restart == 64:           # one cycle, then the final check
            assert est[-1] <= 1e-10
    with pytest.raises(smpm.SmpmError) as e:
        s.residual_history(2, kind=0)
    assert e.value.code == smpm.SMPM_EINVAL
    with pytest.raises(smpm.SmpmError):
        s.residual_history(0, kind=3)
    s.close()
