"""FP64-accurate Schur and block-Jacobi products on the tensor cores
(SMPM_OZAKI=1: tcgen05 BF16 digit products, exact FP32 accumulation per
anti-diagonal, 64-bit integer combination; ozaki.cu).

* Operators: S x and M^-1 x from the tensor-core path against the FP64 CUDA-core
  path of the same handle and against the oracle's assembled operators, for
  class matrices of one and of several 128-row tiles and K-chunks (2 f_z and
  4 f_z from 36 to 544), at the rounding level of an FP64 product (1e-13
  relative, 2-norm and max-norm).
* Solves: the deflated block-Jacobi GMRES with the tensor-core products
  against the oracle's direct and DBJ solves at 1e-9, Poisson and Helmholtz.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.smpm import Grid, direct_solve  # noqa: E402
from oracle.schur import StripSchur  # noqa: E402
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


def _handle(smpm, monkeypatch, oz, shape, k2=0.0):
    monkeypatch.setenv("SMPM_OZAKI", "1" if oz else "0")
    mx, mz, order, lx, lz, zr = shape
    return smpm.Solver(smpm.make_grid(mx, mz, order, lx, lz, z_ratio=zr), k2)


OP_SHAPES = [
    ((8, 2, 8, 4.0, 1.0, 1.0), 0.0),      # 2 f_z = 36, 4 f_z = 72: one tile
    ((6, 8, 10, 1.5, 1.0, 1.0), 9.0),     # 2 f_z = 176, 4 f_z = 352: two and three tiles
    ((4, 16, 16, 0.5, 1.0, 1.2), 0.0),    # 2 f_z = 544, 4 f_z = 1088: five and nine tiles
]


@pytest.mark.parametrize("shape,k2", OP_SHAPES)
def test_tensor_core_products_match_fp64(smpm, monkeypatch, shape, k2):
    R = 40
    so = _handle(smpm, monkeypatch, True, shape, k2)
    sf = _handle(smpm, monkeypatch, False, shape, k2)
    rng = np.random.default_rng(81)
    X = rng.standard_normal((R, so.k))
    X[3] *= 1e-7                               # columns of very different scales
    X[5] = 0.0
    out = {}
    for name, s in (("oz", so), ("fp64", sf)):
        for kind in ("S", "Minv"):
            Y = np.zeros_like(X)
            s.apply(kind, X, Y)
            out[(name, kind)] = Y
    g = Grid(*shape[:5], z_ratio=shape[5])
    sch = StripSchur(g, k2)
    for kind in ("S", "Minv"):
        a, b = out[("oz", kind)], out[("fp64", kind)]
        for i in range(R):
            if i == 5:
                assert np.all(a[i] == 0.0)
                continue
            assert _rel(a[i], b[i]) < 1e-13, (kind, i, _rel(a[i], b[i]))
    # against the oracle's assembled S: the tensor-core products add nothing
    # to the difference between the two independently built operators (3e-12
    # on the order-16 stretched mesh, from the strip solves)
    for i in (0, 3, 7):
        ref = sch.S @ X[i]
        assert _rel(out[("oz", "S")][i], ref) <= max(1e-12, 1.5 * _rel(out[("fp64", "S")][i], ref))
    so.close()
    sf.close()


SOLVE_CASES = [((8, 2, 8, 4.0, 1.0, 1.0), 0.0), ((12, 4, 9, 3.0, 1.0, 1.2), 0.0), ((10, 3, 7, 2.5, 1.0, 1.0), 30.0)]


@pytest.mark.parametrize("shape,k2", SOLVE_CASES)
def test_tensor_core_solve_matches_oracle(smpm, monkeypatch, shape, k2):
    g = Grid(*shape[:5], z_ratio=shape[5])
    F = np.random.default_rng(82).uniform(0, 1, (3, g.r))
    s = _handle(smpm, monkeypatch, True, shape, k2)
    U = np.zeros_like(F)
    st = s.solve(F, U, tol=1e-10)
    s.close()
    assert st.status == 0 and st.rel_resid_true <= 1e-10
    for i in range(3):
        u_ref, _ = direct_solve(g, F[i], None, k2)
        assert _rel(U[i], u_ref) < 1e-9, (i, _rel(U[i], u_ref))


def test_tensor_core_solve_long_domain(smpm, monkeypatch):
    """A 64 x 4 order-12 long-domain solve (the 256 x 4 workload's element
    shape) against the oracle's DBJ solve."""
    from paper_1512_01756_gb300 import inputs
    shape = (64, 4, 12, 16.0, 1.0, 1.0)
    g = Grid(*shape[:5])
    X, Z = g.coords()
    f, _ = inputs.cos_modes(X, Z, 16.0, 1.0, inputs.cos_modes_spec(inputs.seed_for(1)))
    s = _handle(smpm, monkeypatch, True, shape)
    u = np.zeros_like(f)
    st = s.solve(f, u, tol=1e-10)
    s.close()
    assert st.status == 0 and st.rel_resid_true <= 1e-10
    u_ref, _ = dbj.solve(g, f, method="dbj", tol=1e-13)
    assert _rel(u, u_ref) < 1e-9, _rel(u, u_ref)


# --- FP32-accuracy variant (SMPM_OZAKI bit 2): the FP32 products of the mixed
# forms (precision 1's block-Jacobi, precision 2's inner Schur and
# block-Jacobi products) with 24-bit digit splits (4 digits of 7 or 6 bits,
# 5 of 5 bits for K > 1056)

def _handle_p(smpm, monkeypatch, oz, shape, precision, k2=0.0):
    monkeypatch.setenv("SMPM_OZAKI", str(oz))
    mx, mz, order, lx, lz, zr = shape
    return smpm.Solver(smpm.make_grid(mx, mz, order, lx, lz, z_ratio=zr, precision=precision), k2)


@pytest.mark.parametrize("shape", [(8, 2, 8, 4.0, 1.0, 1.0), (6, 8, 10, 1.5, 1.0, 1.0), (4, 16, 16, 0.5, 1.0, 1.2)])
def test_fp32_tensor_core_block_jacobi(smpm, monkeypatch, shape):
    """precision 2's block-Jacobi apply (FP32 inverses) through the 24-bit
    tensor-core products against the FP32 CUDA-core products of the same
    inverses (rounding-level agreement) and against the FP64 inverses (the
    same distance as the CUDA-core products: both are set by the FP32
    factorisation)."""
    R = 24
    so = _handle_p(smpm, monkeypatch, 2, shape, 2)
    sf = _handle_p(smpm, monkeypatch, 0, shape, 2)
    s64 = _handle_p(smpm, monkeypatch, 0, shape, 0)
    X = np.random.default_rng(83).standard_normal((R, so.k))
    X[2] *= 1e-6
    out = {}
    for name, s in (("oz", so), ("f32", sf), ("f64", s64)):
        Y = np.zeros_like(X)
        s.apply("Minv", X, Y)
        out[name] = Y
        s.close()
    worst_of, worst_f = 0.0, 0.0
    for i in range(R):
        d_of = _rel(out["oz"][i], out["f32"][i])
        e_o, e_f = _rel(out["oz"][i], out["f64"][i]), _rel(out["f32"][i], out["f64"][i])
        worst_of = max(worst_of, d_of)
        worst_f = max(worst_f, e_f)
        assert d_of < 1e-4, (i, d_of)
        assert e_o <= 1.5 * e_f + 1e-6, (i, e_o, e_f)
    print(f"tensor-core vs CUDA-core FP32 products {worst_of:.2e}; FP32 inverses vs FP64 {worst_f:.2e}")


@pytest.mark.parametrize("shape,k2,precision", [((8, 2, 8, 4.0, 1.0, 1.0), 0.0, 2), ((12, 4, 9, 3.0, 1.0, 1.2), 0.0, 2),
                                                ((10, 3, 7, 2.5, 1.0, 1.0), 30.0, 2), ((32, 16, 16, 2.0, 1.0, 1.2), 0.0, 2),
                                                ((12, 4, 9, 3.0, 1.0, 1.2), 0.0, 1)])
def test_fp32_tensor_core_solve_matches_oracle(smpm, monkeypatch, shape, k2, precision):
    """Mixed-precision solves with the FP32 products on the tensor cores
    (SMPM_OZAKI=2) and with every product on them (SMPM_OZAKI=3): 1e-10
    residual, the oracle's solution at 1e-9."""
    g = Grid(*shape[:5], z_ratio=shape[5])
    F = np.random.default_rng(84).uniform(0, 1, (2, g.r))
    refs = [direct_solve(g, F[i], None, k2)[0] for i in range(2)] if g.r <= 20000 else None
    if refs is None:
        ref_s = _handle_p(smpm, monkeypatch, 0, shape, 0, k2)
        U0 = np.zeros_like(F)
        st0 = ref_s.solve(F, U0, tol=1e-11)
        ref_s.close()
        assert st0.rel_resid_true <= 1e-11
        refs = list(U0)
    for oz in (2, 3):
        s = _handle_p(smpm, monkeypatch, oz, shape, precision, k2)
        U = np.zeros_like(F)
        st = s.solve(F, U, tol=1e-10)
        s.close()
        assert st.status == 0 and st.rel_resid_true <= 1e-10, (oz, st.as_dict())
        for i in range(2):
            assert _rel(U[i], refs[i]) < 1e-9, (oz, i, _rel(U[i], refs[i]))
