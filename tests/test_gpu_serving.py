"""Serving runtime (smpm_server_*): requests of different grids, orders and k^2
submitted at once are batched and run concurrently; every result must be the
one the same request gives alone (smpm_setup + smpm_solve on its own handle,
same precision), and the one the oracle's direct solve gives (Sec. 2.3;
Helmholtz form of Sec. 5), at relative residual <= 1e-10 and relative error
< 1e-9 -- in FP64 and in the nested mixed precision the serving bench uses.
"""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.smpm import Grid, direct_solve  # noqa: E402

# (mx, mz, order, lx, lz), k^2
REQUESTS = [((8, 2, 6, 4.0, 1.0), 0.0), ((8, 2, 6, 4.0, 1.0), 3.7), ((6, 2, 8, 3.0, 1.0), 0.25),
            ((8, 2, 6, 4.0, 1.0), 150.0), ((6, 2, 8, 3.0, 1.0), 0.0), ((8, 2, 6, 4.0, 1.0), 3.7),
            ((5, 3, 7, 2.5, 1.0), 1e4), ((6, 2, 8, 3.0, 1.0), 41.0), ((8, 2, 6, 4.0, 1.0), 0.02),
            ((5, 3, 7, 2.5, 1.0), 0.0), ((6, 2, 8, 3.0, 1.0), 2.0e3), ((8, 2, 6, 4.0, 1.0), 900.0)]


@pytest.fixture(scope="module")
def smpm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1512_01756_gb300 import smpm as m
    m.load()
    return m


def _rhs(shape, i):
    g = Grid(*shape)
    return np.random.default_rng(4000 + i).uniform(0, 1, g.r)


def _wait(server, tickets, limit_s=120.0):
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        for t in tickets:
            if t not in out:
                st = server.poll(t)
                if st is not None:
                    out[t] = st
        assert time.time() - t0 < limit_s, "requests did not finish"
        time.sleep(0.001)
    return [out[t] for t in tickets]


def _rel(a, b):
    """Relative error in the 2-norm and in the max-norm, the larger of the two
    (a local error on one face of a long vector shows in the second)."""
    a, b = np.asarray(a), np.asarray(b)
    return max(np.linalg.norm(a - b) / np.linalg.norm(b), np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("device_buffers,precision", [(False, 0), (True, 0), (True, 2)])
def test_mix_equals_alone_and_oracle(smpm, device_buffers, precision):
    fs = [_rhs(s, i) for i, (s, _) in enumerate(REQUESTS)]
    if device_buffers:
        fb = [torch.from_numpy(f).cuda() for f in fs]
        ub = [torch.zeros_like(f) for f in fb]
    else:
        fb = fs
        ub = [np.zeros_like(f) for f in fs]
    srv = smpm.Server(nworkers=3, max_batch=4)
    tickets = [srv.submit(smpm.make_grid(*s, precision=precision), k2, fb[i], ub[i], tol=1e-10)
               for i, (s, k2) in enumerate(REQUESTS)]
    stats = _wait(srv, tickets)
    srv.close()
    torch.cuda.synchronize()
    batched = any(st.restarts > 1 for st in stats)
    assert batched, "no two requests shared a batch"
    for i, ((shape, k2), st) in enumerate(zip(REQUESTS, stats)):
        u_mix = ub[i].cpu().numpy() if device_buffers else ub[i]
        assert st.status == 0 and st.rel_resid_true <= 1e-10, (i, st.as_dict())
        # the same request alone, on its own handle
        s = smpm.Solver(smpm.make_grid(*shape, precision=precision), k2)
        u_alone = np.zeros_like(fs[i])
        st1 = s.solve(fs[i], u_alone, tol=1e-10)
        s.close()
        assert st1.rel_resid_true <= 1e-10
        assert _rel(u_mix, u_alone) < 1e-9, (i, _rel(u_mix, u_alone))
        u_ref, _ = direct_solve(Grid(*shape), fs[i], None, k2)
        assert _rel(u_mix, u_ref) < 1e-9, (i, k2, _rel(u_mix, u_ref))


def test_budget_serialises_but_completes(smpm):
    """A budget between the footprint of one request and that of a batch of
    two admits one batch at a time (a larger batch runs alone); everything
    still finishes."""
    shape = (8, 2, 6, 4.0, 1.0)
    one = smpm.request_footprint(smpm.make_grid(*shape), 1, 1)
    two = smpm.request_footprint(smpm.make_grid(*shape), 2, 2)
    assert two > one
    srv = smpm.Server(nworkers=2, device_budget_bytes=(one + two) // 2, max_batch=2)
    fs = [_rhs(shape, 100 + i) for i in range(5)]
    us = [np.zeros_like(f) for f in fs]
    k2s = [0.0, 1.0, 2.0, 0.0, 50.0]
    tickets = [srv.submit(smpm.make_grid(*shape), k2, f, u) for k2, f, u in zip(k2s, fs, us)]
    stats = _wait(srv, tickets)
    srv.close()
    for k2, f, u, st in zip(k2s, fs, us, stats):
        assert st.rel_resid_true <= 1e-10
        u_ref, _ = direct_solve(Grid(*shape), f, None, k2)
        assert _rel(u, u_ref) < 1e-9


def test_bad_requests(smpm):
    srv = smpm.Server(nworkers=1)
    f = np.zeros(10)
    with pytest.raises(smpm.SmpmError):
        srv.submit(smpm.make_grid(8, 2, 6, 4.0, 1.0), 1.0, f, f, tol=0.0)
    with pytest.raises(smpm.SmpmError):
        srv.submit(smpm.make_grid(8, 2, 6, 4.0, 1.0), -1.0, f, f)
    with pytest.raises(smpm.SmpmError):
        srv.poll(123456)
    # an invalid grid fails at setup inside the worker and is reported by poll
    g = np.zeros(4)
    t = srv.submit(smpm.make_grid(1, 1, 6, 4.0, 1.0), 0.0, g, g)
    deadline = time.time() + 30
    while True:
        try:
            st = srv.poll(t)
        except smpm.SmpmError as e:
            assert e.code == smpm.SMPM_EINVAL
            break
        assert st is None, "invalid grid reported success"
        assert time.time() < deadline
        time.sleep(0.001)
    srv.close()


def test_operator_cache_reuses_setup(smpm):
    """A second request with the grid and k^2 of a finished one takes the cached
    operators (no setup) and gives what a fresh handle gives."""
    shape, k2 = (6, 2, 8, 3.0, 1.0), 3.7
    srv = smpm.Server(nworkers=1, max_batch=1)
    f1, f2 = _rhs(shape, 301), _rhs(shape, 302)
    u1, u2 = np.zeros_like(f1), np.zeros_like(f2)
    st1 = _wait(srv, [srv.submit(smpm.make_grid(*shape), k2, f1, u1)])[0]
    st2 = _wait(srv, [srv.submit(smpm.make_grid(*shape), k2, f2, u2)])[0]
    # a different k^2 on the same grid does not hit
    u3 = np.zeros_like(f2)
    st3 = _wait(srv, [srv.submit(smpm.make_grid(*shape), 4.0, f2, u3)])[0]
    srv.close()
    assert st1.setup_ms > 0.0 and st2.setup_ms == 0.0 and st3.setup_ms > 0.0
    s = smpm.Solver(smpm.make_grid(*shape), k2)
    u_fresh = np.zeros_like(f2)
    s.solve(f2, u_fresh, tol=1e-10)
    s.close()
    assert st2.rel_resid_true <= 1e-10 and _rel(u2, u_fresh) < 1e-12
