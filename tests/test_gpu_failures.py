"""Failure detection through the status codes of include/smpm.h, with every
failure made on the host (no GPU fault, trap or hang):

* a NaN planted in f: the Krylov process sees a non-finite residual and the
  solve returns SMPM_EBREAKDOWN;
* max_iter = 3 on a problem that needs more: SMPM_ENOCONV, with a finite best
  iterate in u and its true residual in the stats;
* a serving request whose footprint exceeds the server's device budget: the
  ticket is refused and smpm_poll reports SMPM_ENOMEM, while a request that
  fits is served normally by the same server;
* bad arguments: SMPM_EINVAL with a message.
(The persistent kernel's bounded barrier wait is covered in
test_gpu_persistent.py.)
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


SHAPE = (16, 2, 8, 8.0, 1.0)


def test_nan_in_f_is_breakdown(smpm):
    g = Grid(*SHAPE)
    f = np.random.default_rng(61).uniform(0, 1, g.r)
    f[g.r // 3] = np.nan
    s = smpm.Solver(smpm.make_grid(*SHAPE), 0.0)
    u = np.zeros_like(f)
    with pytest.raises(smpm.SmpmError) as e:
        s.solve(f, u, tol=1e-10)
    assert e.value.code == smpm.SMPM_EBREAKDOWN
    # the handle stays usable
    f[g.r // 3] = 0.5
    st = s.solve(f, u, tol=1e-10)
    s.close()
    assert st.status == 0 and st.rel_resid_true <= 1e-10


def test_iteration_cap_is_noconv_with_best_iterate(smpm):
    g = Grid(*SHAPE)
    f = np.random.default_rng(62).uniform(0, 1, g.r)
    s = smpm.Solver(smpm.make_grid(*SHAPE, max_iter=3), 0.0)
    u = np.zeros_like(f)
    st = s.solve(f, u, tol=1e-10)
    s.close()
    assert st.status == smpm.SMPM_ENOCONV
    assert st.iters <= 3
    assert np.all(np.isfinite(u)) and np.abs(u).max() > 0
    assert np.isfinite(st.rel_resid_true) and 1e-10 < st.rel_resid_true < 1.0


def test_server_refuses_request_over_budget(smpm):
    g = Grid(*SHAPE)
    f = np.random.default_rng(63).uniform(0, 1, g.r)
    srv = smpm.Server(nworkers=1, device_budget_bytes=1 << 20, max_batch=4)
    u = np.zeros_like(f)
    t = srv.submit(smpm.make_grid(*SHAPE), 0.0, f, u, tol=1e-10)
    with pytest.raises(smpm.SmpmError) as e:
        while srv.poll(t) is None:
            pass
    assert e.value.code == smpm.SMPM_ENOMEM
    assert "budget" in str(e.value)
    srv.close()
    srv = smpm.Server(nworkers=1, device_budget_bytes=8 << 30, max_batch=4)
    t = srv.submit(smpm.make_grid(*SHAPE), 0.0, f, u, tol=1e-10)
    st = None
    while st is None:
        st = srv.poll(t)
    srv.close()
    assert st.status == 0 and st.rel_resid_true <= 1e-10


def test_bad_arguments_are_einval(smpm):
    with pytest.raises(smpm.SmpmError) as e:
        smpm.Solver(smpm.make_grid(1, 2, 8, 1.0, 1.0), 0.0)
    assert e.value.code == smpm.SMPM_EINVAL
    with pytest.raises(smpm.SmpmError) as e:
        smpm.Solver(smpm.make_grid(*SHAPE), -1.0)
    assert e.value.code == smpm.SMPM_EINVAL
    s = smpm.Solver(smpm.make_grid(*SHAPE), 0.0)
    f = np.zeros(s.r)
    with pytest.raises(smpm.SmpmError) as e:
        s.solve(f, np.zeros(s.r), tol=-1.0)
    assert e.value.code == smpm.SMPM_EINVAL
    s.close()
