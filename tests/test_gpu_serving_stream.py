"""Serving runtime on requests shaped like the served workload: long domains
[0, mx/mz] x [0, 1] with mx x mz from 64 x 2 to 1024 x 16 elements, orders 6
to 16, k^2 from 0 to 1e4, f a seeded sum of 32 cos-cos modes; all submitted
at once to one server in the nested mixed precision it serves with.

* Grids the oracle finishes in seconds (up to 128 x 4 elements): each served
  result against the oracle's deflated block-Jacobi solve (Alg. seq, Sec. 3.3)
  at 1e-9 relative, 2-norm and max-norm.
* Larger grids (256 x 8 to 1024 x 16, up to 4.7 million nodes): each served
  result against the same request solved alone in plain FP64 on its own
  handle (1e-9), and against the closed-form solution of the continuous
  problem, u = sum_m c_m cos(k_x x) cos(k_z z) / (-(k_x^2 + k_z^2) - k^2), at
  a tolerance set by the discretisation error of the order and element size
  (measured with the oracle on meshes of the same element size: 1.5e-5 for
  order 6 at h = 1/8, 2e-7 for order 6 at h = 1/16, 1e-7 for order 8 at
  h = 1/8, 2e-12 for order 12 at h = 1/8).
"""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.smpm import Grid  # noqa: E402
from oracle.schur import StripSchur  # noqa: E402
from oracle import dbj  # noqa: E402
from paper_1512_01756_gb300 import inputs  # noqa: E402

# (mx, mz), order, k^2
ORACLE_REQS = [((64, 2), 6, 0.0), ((64, 2), 8, 3.2), ((64, 2), 12, 1.0e4), ((64, 2), 16, 0.0),
               ((128, 4), 6, 150.0), ((128, 4), 8, 0.02), ((64, 2), 8, 3.2), ((128, 4), 6, 0.0)]
# (mx, mz), order, k^2, tolerance against the continuous solution
LARGE_REQS = [((256, 8), 12, 0.0, 1e-9), ((256, 8), 16, 41.0, 1e-9), ((512, 16), 8, 0.0, 1e-7),
              ((1024, 16), 16, 2.5e3, 1e-9), ((1024, 16), 6, 0.0, 1e-5), ((512, 16), 12, 0.3, 1e-9),
              ((256, 8), 12, 0.0, 1e-9), ((1024, 16), 16, 7.0, 1e-9)]


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


def _field(x, z, lx, k2, seed):
    """f and the continuous solution of lap u - k^2 u = f with zero normal
    derivative on the boundary (every mode satisfies it), at the nodes."""
    c, a, b = inputs.cos_modes_spec(seed)
    f = np.zeros_like(x)
    u = np.zeros_like(x)
    for cm, am, bm in zip(c, a, b):
        kx, kz = am * np.pi / lx, bm * np.pi
        phi = np.cos(kx * x) * np.cos(kz * z)
        f += cm * phi
        u += cm * phi / (-(kx * kx + kz * kz) - k2)
    return f, u


def _wait(server, tickets, limit_s=600.0):
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


def test_served_stream_matches_oracle_plain_and_continuous(smpm):
    reqs = []
    for i, ((mx, mz), order, k2) in enumerate(ORACLE_REQS):
        reqs.append({"mx": mx, "mz": mz, "order": order, "k2": k2, "tol": None, "seed": inputs.seed_for(500 + i)})
    for i, ((mx, mz), order, k2, tol) in enumerate(LARGE_REQS):
        reqs.append({"mx": mx, "mz": mz, "order": order, "k2": k2, "tol": tol, "seed": inputs.seed_for(600 + i)})
    for q in reqs:
        q["lx"] = q["mx"] / q["mz"]
        q["grid"] = smpm.make_grid(q["mx"], q["mz"], q["order"], q["lx"], 1.0)
        q["served"] = smpm.make_grid(q["mx"], q["mz"], q["order"], q["lx"], 1.0, precision=2)
        x, z = smpm.grid_coords(q["grid"])
        q["f"], q["u_exact"] = _field(x, z, q["lx"], q["k2"], q["seed"])
        q["u"] = np.zeros_like(q["f"])
    srv = smpm.Server(nworkers=3, max_batch=8)
    tickets = [srv.submit(q["served"], q["k2"], q["f"], q["u"], tol=1e-10) for q in reqs]
    stats = _wait(srv, tickets)
    srv.close()
    for q, st in zip(reqs, stats):
        name = f'{q["mx"]}x{q["mz"]} order {q["order"]} k2 {q["k2"]}'
        assert st.status == 0 and st.rel_resid_true <= 1e-10, (name, st.as_dict())
        if q["tol"] is None:
            g = Grid(q["mx"], q["mz"], q["order"], q["lx"], 1.0)
            X, Z = g.coords()
            f_o, _ = _field(X, Z, q["lx"], q["k2"], q["seed"])
            assert np.abs(f_o - q["f"]).max() <= 1e-12 * np.abs(f_o).max(), name   # same nodes
            u_ref, info = dbj.solve(g, f_o, k2=q["k2"], method="dbj", tol=1e-13,
                                    schur=StripSchur(g, q["k2"]))
            assert info["schur_residual"] < 1e-11, (name, info["schur_residual"])
            assert _rel(q["u"], u_ref) < 1e-9, (name, _rel(q["u"], u_ref))
        else:
            s = smpm.Solver(q["grid"], q["k2"])
            u_alone = np.zeros_like(q["f"])
            st1 = s.solve(q["f"], u_alone, tol=1e-10)
            s.close()
            assert st1.status == 0 and st1.rel_resid_true <= 1e-10, name
            assert _rel(q["u"], u_alone) < 1e-9, (name, _rel(q["u"], u_alone))
            assert _rel(q["u"], q["u_exact"]) < q["tol"], (name, _rel(q["u"], q["u_exact"]))
