"""Pins of the oracle's Schur complement and null-space handling (Secs. 2.3-2.4).

Algebraic identities L = A + E B, E^T E = I and A block-diagonal per strip;
Claim 1 (u_S = E^T u_L, u_L parallel to A^-T B^T u_S); Claim 2 (the Schur
residual bounds the full residual); the right null vector B 1 of S; the
Schur-route solution equal to the full-system lstsq solution; the paper's
shifted inverse iteration reproducing u_S; the strip-by-strip assembled S equal
to the dense S.
"""
import numpy as np
import pytest

from oracle.smpm import Grid, assemble_L, split, rhs, direct_solve, left_null_dense
from oracle.schur import schur_dense, alg_schur_direct, shifted_inverse_iteration, StripSchur

SHAPES = [(4, 2, 5, 2.0, 1.0, 1.0), (5, 3, 4, 1.0, 1.0, 1.2), (8, 2, 8, 4.0, 1.0, 1.0)]


@pytest.mark.parametrize("shape", SHAPES)
def test_split_identities(shape):
    mx, mz, order, lx, lz, zr = shape
    g = Grid(mx, mz, order, lx, lz, z_ratio=zr)
    L = assemble_L(g)
    A, E, B = split(g, L)
    assert abs((E.T @ E) - np.eye(g.k)).max() == 0.0
    assert abs(A + E @ B - L).max() == 0.0           # L = A + E B exactly
    Ac = A.tocoo()
    assert np.all(g.strip_of(Ac.row) == g.strip_of(Ac.col))
    # B only reads the neighbouring strip's nodes
    Bc = B.tocoo()
    gam = g.gamma_nodes()
    assert np.all(g.strip_of(gam[Bc.row]) != g.strip_of(Bc.col))
    assert B.shape == (g.k, g.r) and g.k == 2 * g.n * g.mz * (g.mx - 1)


@pytest.mark.parametrize("shape", SHAPES[:2])
def test_claim1_and_null_vectors(shape):
    mx, mz, order, lx, lz, zr = shape
    g = Grid(mx, mz, order, lx, lz, z_ratio=zr)
    L = assemble_L(g)
    S, A, E, B = schur_dense(g, L)
    uL, _ = left_null_dense(L.toarray())
    uS = E.T @ uL
    scale = np.abs(S).max()
    assert np.linalg.norm(uS @ S) < 1e-11 * scale * np.linalg.norm(uS)   # Claim 1.1
    v = np.linalg.solve(A.toarray().T, B.T @ uS)                          # Claim 1.2
    v /= np.linalg.norm(v)
    assert min(np.abs(v - uL).max(), np.abs(v + uL).max()) < 1e-10
    # right null vector of S: B 1 (from L 1 = 0)
    b1 = B @ np.ones(g.r)
    assert np.linalg.norm(S @ b1) < 1e-10 * scale * np.linalg.norm(b1)
    # S's null space is one-dimensional
    s = np.linalg.svd(S, compute_uv=False)
    assert s[-1] / s[0] < 1e-13 and s[-2] / s[0] > 1e-10
    # the paper's shifted inverse iteration finds the same u_S
    uS_n = uS / np.linalg.norm(uS)
    uS_n = -uS_n if uS_n[np.argmax(np.abs(uS_n))] < 0 else uS_n
    ii = shifted_inverse_iteration(S, 1e-10 * scale)
    assert np.abs(ii - uS_n).max() < 1e-9


def test_claim2_residual_bound():
    g = Grid(5, 3, 4, 1.0, 1.0, z_ratio=1.2)
    rng = np.random.default_rng(3)
    f = rng.uniform(0, 1, g.r)
    u, parts = alg_schur_direct(g, f)
    S, A, E, B, L = parts["S"], parts["A"], parts["E"], parts["B"], parts["L"]
    ft, uS = parts["b"], parts["uS"]
    bS = B @ np.linalg.solve(A.toarray(), ft)
    for eps in [1e-3, 1e-6, 1e-9]:
        xS = parts["xS"] + eps * rng.standard_normal(g.k)
        uu = np.linalg.solve(A.toarray(), ft - E @ xS)
        lhs = np.linalg.norm(L @ uu - ft)
        rhs_ = np.linalg.norm(S @ xS - (bS - uS * np.dot(uS, bS)))
        assert lhs <= rhs_ * (1 + 1e-8) + 1e-12


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("k2", [0.0, 12.0])
def test_schur_route_equals_full_system(shape, k2):
    mx, mz, order, lx, lz, zr = shape
    g = Grid(mx, mz, order, lx, lz, z_ratio=zr)
    rng = np.random.default_rng(7)
    f = rng.uniform(0, 1, g.r)
    u_full, _ = direct_solve(g, f, None, k2)
    u_schur, _ = alg_schur_direct(g, f, None, k2)
    assert np.linalg.norm(u_schur - u_full) < 1e-10 * np.linalg.norm(u_full)


def test_strip_assembled_S_matches_dense():
    g = Grid(5, 3, 4, 1.0, 1.0, z_ratio=1.2)
    L = assemble_L(g, 3.0)
    S, _, _, _ = schur_dense(g, L)
    sch = StripSchur(g, 3.0)
    assert np.abs(sch.S.toarray() - S).max() < 1e-12 * np.abs(S).max()
    # each interface row couples only to its own and neighbouring interfaces
    fz2 = 2 * g.fz
    Sc = sch.S.tocoo()
    assert np.all(np.abs(Sc.row // fz2 - Sc.col // fz2) <= 1)


@pytest.mark.parametrize("shape,k2", [((6, 2, 5, 3.0, 1.0, 1.0), 2.5), ((5, 3, 4, 1.0, 1.0, 1.2), 0.0)])
def test_schur_commutes_with_x_reflection(shape, k2):
    """With uniform h_x the domain is symmetric under x -> l_x - x, which maps
    interface j to m_x - 2 - j and swaps the two sides of every interface
    (each side keeps its z order); the assembled S commutes with that
    permutation.  This is the symmetry the library's mirror-form products of
    the interior strips and block-Jacobi pairs rest on (Sec. 3.1, Sec. 3.2)."""
    mx, mz, order, lx, lz, zr = shape
    g = Grid(mx, mz, order, lx, lz, z_ratio=zr)
    S = schur_dense(g, assemble_L(g, k2))[0]
    fz = g.fz

    def mirror(i):
        j, rem = divmod(i, 2 * fz)
        s, z = divmod(rem, fz)
        return (g.mx - 2 - j) * 2 * fz + (1 - s) * fz + z

    P = np.array([mirror(i) for i in range(g.k)])
    assert sorted(P) == list(range(g.k))
    assert np.abs(S[np.ix_(P, P)] - S).max() < 1e-12 * np.abs(S).max()
    # and it is not a symmetry of the stretched z direction's reversal
    if zr != 1.0:
        Q = np.array([(i // fz) * fz + (fz - 1 - i % fz) for i in range(g.k)])
        assert np.abs(S[np.ix_(Q, Q)] - S).max() > 1e-3 * np.abs(S).max()


@pytest.mark.parametrize("shape,k2", [((4, 2, 5, 2.0, 1.0, 1.0), 0.0), ((5, 4, 4, 2.0, 1.0, 1.0), 7.5)])
def test_schur_commutes_with_z_reversal(shape, k2):
    """With uniform h_z (and the Neumann condition at both z-ends) the domain
    is symmetric under z -> l_z - z, which reverses the z-nodes of every face
    and keeps the faces in place; the assembled S commutes with it.  The
    library's z-mirror form of the fast strip solver's slot products rests on
    this symmetry of L_z (Sec. 2.2, Sec. 5)."""
    mx, mz, order, lx, lz, zr = shape
    g = Grid(mx, mz, order, lx, lz, z_ratio=zr)
    S = schur_dense(g, assemble_L(g, k2))[0]
    fz = g.fz
    P = np.array([(i // fz) * fz + (fz - 1 - i % fz) for i in range(g.k)])
    assert np.abs(S[np.ix_(P, P)] - S).max() < 1e-12 * np.abs(S).max()
    # the same map is not a symmetry once z is stretched
    gs = Grid(mx, mz, order, lx, lz, z_ratio=1.3)
    Ss = schur_dense(gs, assemble_L(gs, k2))[0]
    assert np.abs(Ss[np.ix_(P, P)] - Ss).max() > 1e-3 * np.abs(Ss).max()


def test_null_vector_on_stiff_stretched_mesh():
    """Left null vector of L on the order-16 mesh stretched by 1.2 (elements
    from 0.011 to 0.18 high, penalty rows ~1e12): the data of a zero-mean
    manufactured solution with g = 0 is compatible with the continuous
    problem, so the discrete compatibility u_L^T b must vanish to the
    discretisation error (spectrally small at order 16), and L^T u_L = 0 to
    round-off of the rows.  The same inverse iteration on the unequilibrated
    L (the shift a fixed fraction of max |L|, above the smallest nonzero
    eigenvalue here) converges to a mixture and misses it by orders of
    magnitude -- that planted variant must fail."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    from oracle.schur import left_null_sparse
    g = Grid(32, 16, 16, 2.0, 1.0, z_ratio=1.2)
    X, Z = g.coords()
    ue = np.cos(np.pi * X / g.lx) * np.cos(np.pi * Z / g.lz)
    f = -(np.pi ** 2 / g.lx ** 2 + np.pi ** 2 / g.lz ** 2) * ue
    L = assemble_L(g).tocsr()
    b = rhs(g, f)
    uL = left_null_sparse(L)
    rowmax = abs(L).max(axis=1).toarray().ravel()
    assert np.abs((L.T @ uL)).max() < 1e-13 * rowmax.max()
    assert abs(np.dot(uL, b)) < 1e-11 * np.linalg.norm(b)
    # planted mistake: no row equilibration
    T = (L.T - 1e-12 * abs(L).max() * sp.identity(g.r)).tocsc()
    lu = spla.splu(T)
    v = np.random.default_rng(0).standard_normal(g.r)
    for _ in range(4):
        v = lu.solve(v)
        v /= np.linalg.norm(v)
    assert abs(np.dot(v, b)) > 1e-7 * np.linalg.norm(b)
