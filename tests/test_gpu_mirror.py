"""Mirror forms of the dense products.

With uniform h_x an interior strip (and an interior block-Jacobi pair) is
symmetric under the reflection of x about its centre, so its class matrix
commutes with the reversal of its faces and splits into two half-size
products (the symmetric and antisymmetric parts of the column): half the
FLOPs of the dense apply (the oracle's assembled S has that symmetry to
rounding: tests/test_oracle_schur.py).  With uniform h_z the same holds for
the fast strip solver's slot inverses under the reversal of the z-nodes.
Through the C ABI, the mirror-form S x, M^-1 x, B A^-1 b and A^-1 b of a
handle set up with SMPM_MIRROR=1 (mirror form at every size) must equal the
full products of one set up with SMPM_MIRROR=0 to rounding, solves must
agree, and the profiled FLOPs must be about half of the full form's; by
default small batches keep the full products of S and M^-1.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.smpm import Grid  # noqa: E402

SHAPES = [((7, 3, 6, 2.0, 1.0, 1.2), 0.0), ((12, 4, 7, 3.0, 1.0, 1.0), 37.0),
          ((256, 4, 12, 64.0, 1.0, 1.0), 0.0)]


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
    """Relative error in the 2-norm and in the max-norm, the larger of the two
    (a local error on one face of a long vector shows in the second)."""
    a, b = np.asarray(a), np.asarray(b)
    return max(np.linalg.norm(a - b) / np.linalg.norm(b), np.abs(a - b).max() / np.abs(b).max())


def _pair(smpm, monkeypatch, shape, k2, precision=0):
    mx, mz, order, lx, lz, zr = shape
    grid = smpm.make_grid(mx, mz, order, lx, lz, z_ratio=zr, precision=precision)
    monkeypatch.setenv("SMPM_MIRROR", "1")
    s_mir = smpm.Solver(grid, k2)
    monkeypatch.setenv("SMPM_MIRROR", "0")
    s_full = smpm.Solver(grid, k2)
    monkeypatch.delenv("SMPM_MIRROR")
    return s_mir, s_full


@pytest.mark.parametrize("shape,k2", SHAPES)
def test_mirror_products_equal_full(smpm, monkeypatch, shape, k2):
    g = Grid(*shape[:5], z_ratio=shape[5])
    s_mir, s_full = _pair(smpm, monkeypatch, shape, k2)
    X = np.random.default_rng(5).standard_normal((3, g.k))
    a, b = np.empty_like(X), np.empty_like(X)
    s_mir.apply("S", X, a)
    s_full.apply("S", X, b)
    assert max(_rel(a[i], b[i]) for i in range(3)) < 1e-12
    s_mir.apply("Minv", X, a)
    s_full.apply("Minv", X, b)
    assert max(_rel(a[i], b[i]) for i in range(3)) < 1e-10
    # the refined fast strip solves (z-mirror slot products on uniform-z grids)
    Bv = np.random.default_rng(4).standard_normal((3, g.r))
    a, b = np.empty_like(X), np.empty_like(X)
    s_mir.apply("bS", Bv, a)
    s_full.apply("bS", Bv, b)
    assert max(_rel(a[i], b[i]) for i in range(3)) < 1e-11
    ar, br = np.empty_like(Bv), np.empty_like(Bv)
    s_mir.apply("Ainv", Bv, ar)
    s_full.apply("Ainv", Bv, br)
    assert max(_rel(ar[i], br[i]) for i in range(3)) < 1e-11
    # solves of the same right-hand side (both to 1e-11)
    f = np.random.default_rng(6).uniform(0, 1, g.r)
    u1, u2 = np.zeros_like(f), np.zeros_like(f)
    st1 = s_mir.solve(f, u1, tol=1e-11)
    st2 = s_full.solve(f, u2, tol=1e-11)
    s_mir.close()
    s_full.close()
    assert st1.status == 0 and st1.rel_resid_true <= 1e-11 and st2.rel_resid_true <= 1e-11
    assert _rel(u1, u2) < 1e-9


@pytest.mark.parametrize("precision", [1, 2])
def test_mirror_fp32_blocks(smpm, monkeypatch, precision):
    """The FP32 block-Jacobi (precision 1 and 2) and the FP32 Schur blocks of
    the nested form (precision 2) in the mirror form: FP32-rounding agreement
    with the full form, and the mixed solves reach the FP64 solution."""
    shape, k2 = (12, 4, 7, 3.0, 1.0, 1.0), 0.0
    g = Grid(*shape[:5])
    s_mir, s_full = _pair(smpm, monkeypatch, shape, k2, precision)
    X = np.random.default_rng(7).standard_normal((2, g.k))
    a, b = np.empty_like(X), np.empty_like(X)
    s_mir.apply("Minv", X, a)
    s_full.apply("Minv", X, b)
    assert max(_rel(a[i], b[i]) for i in range(2)) < (1e-10 if precision == 1 else 1e-5)
    f = np.random.default_rng(8).uniform(0, 1, g.r)
    u1, u2 = np.zeros_like(f), np.zeros_like(f)
    st1 = s_mir.solve(f, u1, tol=1e-11)
    st2 = s_full.solve(f, u2, tol=1e-11)
    s_mir.close()
    s_full.close()
    assert st1.status == 0 and st1.rel_resid_true <= 1e-11 and st2.rel_resid_true <= 1e-11
    assert _rel(u1, u2) < 1e-9


def test_mirror_halves_the_flops(smpm, monkeypatch):
    """Profiled FLOPs on 256 x 4, order 12.  One S x: the 254 interior strips
    in the mirror form, the two boundary strips (f_z stored rows each) full:
    (2 * 4 + 254 * 4) / (2 * 4 + 254 * 8) = 0.502 of the full form (in units
    of f_z^2 FLOPs per column).  One refined A^-1 b: every slot product in the
    z-mirror form, exactly half."""
    shape = (256, 4, 12, 64.0, 1.0, 1.0)
    g = Grid(*shape[:5])
    s_mir, s_full = _pair(smpm, monkeypatch, shape, 0.0)
    X = np.random.default_rng(9).standard_normal((4, g.k))
    y = np.empty_like(X)
    Bv = np.random.default_rng(10).standard_normal((4, g.r))
    yr = np.empty_like(Bv)
    fl, fl_a = [], []
    for s in (s_mir, s_full):
        for kind, x, out, acc in (("S", X, y, fl), ("Ainv", Bv, yr, fl_a)):
            s.apply(kind, x, out)          # tile-shape tuning happens outside the profile
            s.profile(True)
            s.apply(kind, x, out)
            acc.append(s.profile_read()["flops"])
            s.profile(False)
        s.close()
    fz = g.fz
    assert fl[1] == pytest.approx(4 * (2 * (2 * fz * 2 * fz) + 254 * 2 * (2 * fz) ** 2), rel=1e-12)
    assert fl[0] / fl[1] == pytest.approx(1024 / 2040, rel=1e-9)
    assert fl_a[0] / fl_a[1] == pytest.approx(0.5, rel=1e-9)


def test_small_batches_keep_the_full_products(smpm):
    """By default the x-mirror form of S and M^-1 (one more launch per
    product) is used only where it saves enough FLOPs: not for one right-hand
    side on 8 x 2, order 8; yes for 128 on 256 x 4, order 12."""
    fl = {}
    for shape, R in (((8, 2, 8, 4.0, 1.0), 1), ((256, 4, 12, 64.0, 1.0), 128)):
        g = Grid(*shape)
        s = smpm.Solver(smpm.make_grid(*shape), 0.0, torch.cuda.current_stream())
        X = torch.randn(R, g.k, dtype=torch.float64, device="cuda")
        Y = torch.empty_like(X)
        s.apply("S", X, Y)
        s.profile(True)
        s.apply("S", X, Y)
        p = s.profile_read()
        s.profile(False)
        s.close()
        full = R * (2 * (2 * g.fz * 2 * g.fz) + (g.mx - 2) * 2 * (2 * g.fz) ** 2)
        fl[shape[0]] = (p["launches"], p["flops"] / full)
    assert fl[8] == (1, pytest.approx(1.0, rel=1e-12))
    assert fl[256][0] == 2 and fl[256][1] == pytest.approx(1024 / 2040, rel=1e-9)
