"""Schur complement of the SMPM operator and its null-space handling (Secs. 2.3-2.4).

Test infrastructure only (see ``oracle/__init__.py``).

* S = I + B A^-1 E, b_S = B A^-1 f (Eq. operator_decomp); recovery
  u_i = A_i^-1 (f_i - (E x_S)_i).
* Left null vectors: u_L of L (Eq. regularize_poisson), u_S of S, related by
  Claim 1 (u_S = E^T u_L, u_L = A^-T B^T u_S); the Schur RHS projection of
  Eq. regularize_schur; Alg. schur with a direct (lstsq) Schur solve.
* Shifted inverse iteration on S^T - sigma I for u_S (end of Sec. 2.4), used as
  a cross-check of the SVD null vector.
* ``StripSchur``: the assembled form the paper multiplies with (Sec. 3.1:
  blocks of S stored and applied as a sparse matrix), built strip by strip
  from a sparse LU of each strip's A_i.  Used for grids too large for dense S.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .smpm import Grid, assemble_L, rhs, split, gauge, left_null_dense


def _fix_sign(v):
    return -v if v[np.argmax(np.abs(v))] < 0 else v


def schur_dense(g: Grid, L):
    """Dense S = I + B A^-1 E for tiny grids; returns (S, A, E, B)."""
    A, E, B = split(g, L)
    AinvE = np.linalg.solve(A.toarray(), E.toarray())
    S = np.eye(g.k) + B.toarray() @ AinvE
    return S, A, E, B


def shifted_inverse_iteration(M, sigma, steps=3, seed=0):
    """Left null vector of a dense square M: a few steps of inverse iteration
    with (M^T - sigma I), as proposed for u_S at the end of Sec. 2.4."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(M.shape[0])
    v /= np.linalg.norm(v)
    T = M.T - sigma * np.eye(M.shape[0])
    for _ in range(steps):
        v = np.linalg.solve(T, v)
        v /= np.linalg.norm(v)
    return _fix_sign(v)


def left_null_sparse(L, steps=4, rel_shift=1e-12, seed=0):
    """Unit left null vector of a large sparse singular L: the shifted inverse
    iteration of Sec. 2.4 (a few solves with a sparse LU of M^T - sigma I),
    run on the row-equilibrated operator M = D L, D = diag(1 / max_j |L_ij|).

    The rows of the SMPM operator span many orders of magnitude (the penalty
    rows carry tau (u + n.grad u) with tau ~ (N (N+1) / h)^2, the interior rows
    only the Laplacian), so a shift that is "small" against max |L| can exceed
    the smallest nonzero eigenvalue of L on long or finely stretched meshes,
    and the iteration then converges to a mixture of eigenvectors.  On M every
    row has unit size, sigma = rel_shift stays far below M's smallest nonzero
    eigenvalue, and the left null vector of L is D times that of M
    (w^T M = 0  <=>  (D w)^T L = 0)."""
    d = 1.0 / abs(L).max(axis=1).toarray().ravel()
    M = (sp.diags(d) @ L).tocsr()
    T = (M.T - rel_shift * sp.identity(L.shape[0])).tocsc()
    lu = spla.splu(T)
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(L.shape[0])
    v /= np.linalg.norm(v)
    for _ in range(steps):
        v = lu.solve(v)
        v /= np.linalg.norm(v)
    u = d * v
    return _fix_sign(u / np.linalg.norm(u))


def alg_schur_direct(g: Grid, f, gb=None, k2=0.0):
    """Alg. schur on a tiny grid with dense S and an lstsq Schur solve.

    Returns (u, parts) with u gauge-fixed (k2 == 0) and parts holding the
    intermediate quantities for the invariant tests.
    """
    L = assemble_L(g, k2)
    S, A, E, B = schur_dense(g, L)
    b = rhs(g, f, gb)
    Ad = A.toarray()
    parts = {"L": L, "S": S, "A": A, "E": E, "B": B}
    if k2 == 0.0:
        uL, sL = left_null_dense(L.toarray())
        uS = E.T @ uL
        uS = _fix_sign(uS / np.linalg.norm(uS))
        b = b - uL * np.dot(uL, b)                         # Alg. schur step 1
        bS = B @ np.linalg.solve(Ad, b)                    # step 2
        bS_raw = bS.copy()
        bS = bS - uS * np.dot(uS, bS)                      # step 3
        xS = np.linalg.lstsq(S, bS, rcond=None)[0]         # step 4
        u = np.linalg.solve(Ad, b - E @ xS)                # step 5
        parts.update(uL=uL, uS=uS, sL=sL, bS_raw=bS_raw)
        u = gauge(g, u)
    else:
        bS = B @ np.linalg.solve(Ad, b)
        xS = np.linalg.solve(S, bS)
        u = np.linalg.solve(Ad, b - E @ xS)
    parts.update(b=b, bS=bS, xS=xS)
    return u, parts


def _refined(lu, A, rhs, steps=2):
    """A^-1 rhs from a sparse LU of A, with `steps` iterative-refinement steps."""
    x = lu.solve(rhs)
    for _ in range(steps):
        x = x + lu.solve(rhs - A @ x)
    return x


class StripSchur:
    """Assembled Schur matrix S = I + sum_i E_i-blocks, built strip by strip.

    For every strip i, the columns of A_i^-1 at the strip's own interface
    nodes are found with a sparse LU of A_i, and B's rows that read strip i
    turn them into the strip's block of B A^-1 E.  The blocks are stored in a
    sparse S (the paper's assembled form, Sec. 3.1).  A sparse LU of the whole
    block-diagonal A serves b_S = B A^-1 b and the recovery step.

    Every strip solve takes two steps of iterative refinement on its LU
    (x += LU^-1 (rhs - A x)): the strip operators are ill-conditioned, and an
    unrefined S is off by ~2.5e-13 relative, which on long domains (Schur
    condition ~1e4) moves the solution by ~4e-9.
    """

    def __init__(self, g: Grid, k2=0.0):
        self.g, self.k2 = g, k2
        self.L = assemble_L(g, k2)
        self.A, self.E, self.B = split(g, self.L)
        self.A_lu = spla.splu(self.A.tocsc())
        per = g.n * g.fz
        gam = g.gamma_nodes()
        strip_of_gam = g.strip_of(gam)
        Bc = self.B.tocsc()
        rows, cols, vals = [], [], []
        for i in range(g.mx):
            lo, hi = i * per, (i + 1) * per
            own = np.nonzero(strip_of_gam == i)[0]          # interface unknowns on strip i
            Ai = self.A[lo:hi, lo:hi].tocsc()
            rhs_cols = np.zeros((per, len(own)))
            rhs_cols[gam[own] - lo, np.arange(len(own))] = 1.0
            lu = spla.splu(Ai)
            H = _refined(lu, Ai, rhs_cols)                  # A_i^-1 E_i
            Bi = Bc[:, lo:hi]                               # B restricted to strip-i columns
            Gi = (Bi @ H)                                   # k x |own|
            nzr = np.nonzero(np.any(Gi != 0.0, axis=1))[0]
            rr, cc = np.meshgrid(nzr, own, indexing="ij")
            rows.append(rr.ravel())
            cols.append(cc.ravel())
            vals.append(Gi[nzr, :].ravel())
        rows.append(np.arange(g.k))
        cols.append(np.arange(g.k))
        vals.append(np.ones(g.k))
        self.S = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                               shape=(g.k, g.k)).tocsr()
        self.S.sum_duplicates()

    def Ainv(self, v):
        return _refined(self.A_lu, self.A, v)

    def null_vectors(self):
        """u_L by inverse iteration on L^T; u_S = E^T u_L normalised (Claim 1)."""
        uL = left_null_sparse(self.L)
        uS = self.E.T @ uL
        uS = _fix_sign(uS / np.linalg.norm(uS))
        return uL, uS
