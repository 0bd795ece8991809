"""Persistent Arnoldi kernel (all steps of a restart cycle in one cooperative
launch, phases separated by grid-wide barriers with bounded waits).

* Parity: the persistent path against the step-group path (separate launches,
  SMPM_PERSISTENT unset) and against the oracle, for the plain FP64 solve, the
  mixed-precision solve (FP64 first step group, FP32 block-Jacobi after),
  several restart cycles, batched right-hand sides and the batched Fourier
  modes of the 3-D problem (Sec. 5, Alg. 3d).
* Launches: one cycle costs one persistent launch instead of ~8 per step.
* Failure detection without a fault: the test hook SMPM_PERSIST_STALL makes
  every barrier wait for a block that does not exist, with a 1 ms limit; the
  solve must come back with SMPM_ETIMEOUT, and the next solve on the same
  handle must succeed (the context stays usable).
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


def _solve(smpm, monkeypatch, persistent, shape, F, k2=0.0, **grid_kw):
    monkeypatch.setenv("SMPM_PERSISTENT", "1" if persistent else "0")
    mx, mz, order, lx, lz, zr = shape
    s = smpm.Solver(smpm.make_grid(mx, mz, order, lx, lz, z_ratio=zr, **grid_kw), k2)
    U = np.zeros_like(F)
    l0 = smpm.kernel_launches()
    st = s.solve(F, U, tol=1e-10)
    launches = smpm.kernel_launches() - l0
    s.close()
    return U, st, launches


CASES = [
    ((8, 2, 8, 4.0, 1.0, 1.0), 0.0, 1, {}),
    ((12, 3, 7, 3.0, 1.0, 1.2), 0.0, 3, {}),
    ((10, 2, 6, 2.5, 1.0, 1.0), 40.0, 2, {}),
    ((12, 3, 7, 3.0, 1.0, 1.2), 0.0, 2, {"precision": 1}),
    ((16, 2, 5, 4.0, 1.0, 1.0), 0.0, 2, {"restart": 3}),
]


@pytest.mark.parametrize("case", CASES)
def test_persistent_matches_step_groups_and_oracle(smpm, monkeypatch, case):
    shape, k2, R, kw = case
    g = Grid(*shape[:5], z_ratio=shape[5])
    F = np.random.default_rng(41).uniform(0, 1, (R, g.r))
    if R == 1:
        F = F[0]
    Up, stp, lp = _solve(smpm, monkeypatch, True, shape, F, k2, **kw)
    Us, sts, ls = _solve(smpm, monkeypatch, False, shape, F, k2, **kw)
    assert stp.status == 0 and sts.status == 0
    assert stp.rel_resid_true <= 1e-10 and sts.rel_resid_true <= 1e-10
    assert _rel(Up, Us) < 1e-10, _rel(Up, Us)
    for i, f in enumerate(np.atleast_2d(F)):
        u_ref, _ = direct_solve(g, f, None, k2)
        assert _rel(np.atleast_2d(Up)[i], u_ref) < 1e-9
    if kw.get("restart"):
        assert stp.restarts >= 1
    print(f"launches: persistent {lp}, step groups {ls}")
    assert lp < ls


def test_persistent_batched_fourier_modes(smpm, monkeypatch):
    """All modes of a small 3-D problem in the same persistent launches."""
    shape = (6, 2, 6, 2.0, 1.0)
    g = Grid(*shape)
    my, ly = 8, 2.0 * np.pi
    f3 = np.random.default_rng(44).uniform(0, 1, (g.r, my))
    u_ref = fourier.solve_3d(g, f3, ly)
    out = {}
    for persistent in (True, False):
        monkeypatch.setenv("SMPM_PERSISTENT", "1" if persistent else "0")
        s = smpm.Solver3D(smpm.make_grid(*shape), my, ly)
        u3 = np.zeros((my, g.r))
        st = s.solve_3d_physical(np.ascontiguousarray(f3.T), u3, tol=1e-10)
        s.close()
        assert st.status == 0 and st.rel_resid_true <= 1e-10
        out[persistent] = u3.T
    assert _rel(out[True], out[False]) < 1e-10
    assert _rel(out[True], u_ref) < 1e-9


def test_barrier_timeout_returns_etimeout(smpm, monkeypatch):
    shape = (8, 2, 8, 4.0, 1.0, 1.0)
    g = Grid(*shape[:5])
    f = np.random.default_rng(45).uniform(0, 1, g.r)
    monkeypatch.setenv("SMPM_PERSISTENT", "1")
    s = smpm.Solver(smpm.make_grid(*shape[:5]), 0.0)
    u = np.zeros_like(f)
    monkeypatch.setenv("SMPM_PERSIST_STALL", "1")
    monkeypatch.setenv("SMPM_PERSIST_WAIT_NS", "1000000")
    with pytest.raises(smpm.SmpmError) as e:
        s.solve(f, u, tol=1e-10)
    assert e.value.code == smpm.SMPM_ETIMEOUT
    monkeypatch.delenv("SMPM_PERSIST_STALL")
    monkeypatch.delenv("SMPM_PERSIST_WAIT_NS")
    st = s.solve(f, u, tol=1e-10)             # the handle and the context are still usable
    s.close()
    assert st.status == 0 and st.rel_resid_true <= 1e-10
    u_ref, _ = direct_solve(g, f)
    assert _rel(u, u_ref) < 1e-9
