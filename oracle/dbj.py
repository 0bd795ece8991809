"""Block-Jacobi + deflation GMRES on the Schur system (Sec. 3, Alg. seq).

Test infrastructure only (see ``oracle/__init__.py``).

* ``householder_gmres``: GMRES with Householder-reflector Arnoldi (Sec. 3.1,
  after Walker), zero initial guess, residual tracked through Givens rotations
  of the Hessenberg matrix, unrestarted.
* ``BlockJacobi``: the non-overlapping block-Jacobi preconditioner M of
  Sec. 3.2: diagonal blocks of S over pairs of consecutive interfaces
  (Gamma_{2p}, Gamma_{2p+1}), dimension 4 n m_z, the last block a single
  interface when m_x - 1 is odd; each block LU-factored.
* ``Deflation``: interface indicator vectors Z (Sec. 3.3), coarse matrix
  C = Z^T S Z, the regularised coarse division C \\ (Z^T - u_C u_C^T Z^T) with
  u_C = Z^T u_S normalised, the projections P and Q.  "C \\" on the singular
  coarse matrix is read as the minimum-norm least-squares solve.  Optional
  finer groups: one indicator per interface and element row.
* ``RangeProjected``: for k^2 = 0 the Krylov operator is (I - u_S u_S^T) S,
  the range-projected Schur matrix (equal to S in exact arithmetic).
* ``solve``: Alg. seq (method "dbj") and the comparison methods of
  Table table_methods ("schur", "bj", "2las"), with P applied literally
  (a second S product per iteration, as the paper does).
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .smpm import Grid, rhs, gauge
from .schur import StripSchur


class RangeProjected:
    """S_reg = (I - u_S u_S^T) S, the singular Schur matrix with its range
    projected out of the left null vector u_S.

    Eq. regularize_schur makes the system consistent by projecting b_S out of
    u_S, which presumes u_S^T S = 0.  The assembled S (from rounded strip
    solves) satisfies that only to rounding, ~1e-13 |S|, so S x_S keeps a u_S
    component of that relative size times |x_S| that no iterate removes; when
    |x_S| >> |b_S| (right-hand sides dominated by long x-waves) GMRES then
    stops on that floor with an error of ~1e-9 in u.  Projecting the range the
    same way keeps the system consistent in floating point; in exact
    arithmetic S_reg = S.  Vectors only (the coarse matrix is corrected in
    ``Deflation``)."""

    def __init__(self, S, uS):
        self.S = S
        self.uS = uS
        self.shape = S.shape

    def __matmul__(self, v):
        y = self.S @ v
        return y - self.uS * np.dot(self.uS, y)


def householder_gmres(apply, b, tol, maxiter):
    """Solve apply(x) = b from x0 = 0.  Returns (x, iterations, residual history
    relative to ||b||).  Stops when the Givens residual estimate <= tol ||b||."""
    n = b.shape[0]
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return np.zeros_like(b), 0, [0.0]
    refl = []                       # (start index j, tail of unit Householder vector)

    def house(z, j):
        x = z[j:]
        s = np.linalg.norm(x)
        if s == 0.0:
            return None, 0.0
        alpha = -s if x[0] >= 0.0 else s
        u = x.copy()
        u[0] -= alpha
        return u / np.linalg.norm(u), alpha

    def reflect(v, k):
        j, w = refl[k]
        if w is not None:
            v[j:] -= 2.0 * w * np.dot(w, v[j:])

    w0, beta = house(b.copy(), 0)
    refl.append((0, w0))
    g = [beta]                      # rotated right-hand side beta e_1
    cs, sn, R = [], [], []
    hist = [1.0]
    m = 0
    for j in range(min(maxiter, n)):
        v = np.zeros(n)
        v[j] = 1.0
        for k in range(j, -1, -1):  # v_j = P_0 P_1 ... P_j e_j
            reflect(v, k)
        z = apply(v)
        for k in range(j + 1):      # P_j ... P_0 A v_j
            reflect(z, k)
        if j + 1 < n:
            wn, alpha = house(z, j + 1)
            refl.append((j + 1, wn))
        else:
            alpha = 0.0
        h = np.concatenate([z[:j + 1], [alpha]])
        for k in range(j):          # earlier Givens rotations
            t = cs[k] * h[k] + sn[k] * h[k + 1]
            h[k + 1] = -sn[k] * h[k] + cs[k] * h[k + 1]
            h[k] = t
        rho = np.hypot(h[j], h[j + 1])
        c, s = (1.0, 0.0) if rho == 0.0 else (h[j] / rho, h[j + 1] / rho)
        cs.append(c)
        sn.append(s)
        h[j] = rho
        h[j + 1] = 0.0
        R.append(h[:j + 1].copy())
        g.append(-s * g[j])
        g[j] = c * g[j]
        m = j + 1
        res = abs(g[j + 1]) / bnorm
        hist.append(res)
        if res <= tol:
            break
    Rm = np.zeros((m, m))
    for col, hc in enumerate(R):
        Rm[:col + 1, col] = hc
    y = sla.solve_triangular(Rm, np.array(g[:m]))
    x = np.zeros(n)
    for k in range(m - 1, -1, -1):  # x = sum_k y_k v_k = P_0 (y_0 e_0 + P_1 (y_1 e_1 + ...))
        x[k] += y[k]
        reflect(x, k)
    return x, m, hist


class BlockJacobi:
    """Pairs of interfaces -> dense diagonal blocks of S, LU-factored (Sec. 3.2).

    With m_x <= 3 the single block is all of S; for the singular Poisson-Neumann
    S (singular=True) that block is replaced by the identity (reading: the
    paper's blocks are proper principal submatrices, which it notes are
    invertible)."""

    def __init__(self, g: Grid, S, singular=False):
        fz2 = 2 * g.fz
        nif = g.mx - 1
        self.ranges = []
        p = 0
        while 2 * p < nif:
            lo = 2 * p * fz2
            hi = min((2 * p + 2) * fz2, nif * fz2)
            self.ranges.append((lo, hi))
            p += 1
        Sc = S.tocsr()
        self.identity = singular and len(self.ranges) == 1
        self.lus = [] if self.identity else [sla.lu_factor(Sc[lo:hi, lo:hi].toarray()) for lo, hi in self.ranges]

    def solve(self, v):
        if self.identity:
            return v.copy()
        out = np.empty_like(v)
        for (lo, hi), lu in zip(self.ranges, self.lus):
            out[lo:hi] = sla.lu_solve(lu, v[lo:hi])
        return out


class Deflation:
    """Interface-indicator deflation with the regularised coarse division (Sec. 3.3)."""

    def __init__(self, g: Grid, S, uS=None, groups="interface", coarse="lstsq"):
        self.coarse_mode = coarse
        nif = g.mx - 1
        fz2 = 2 * g.fz
        rows, cols = [], []
        if groups == "interface":
            self.d = nif
            for j in range(nif):
                rows.append(np.arange(j * fz2, (j + 1) * fz2))
                cols.append(np.full(fz2, j))
        elif groups == "element_row":
            self.d = nif * g.mz
            for j in range(nif):
                for ez in range(g.mz):
                    zs = np.arange(ez * g.n, (ez + 1) * g.n)
                    idx = np.concatenate([j * fz2 + zs, j * fz2 + g.fz + zs])
                    rows.append(idx)
                    cols.append(np.full(idx.size, j * g.mz + ez))
        else:
            raise ValueError(groups)
        r = np.concatenate(rows)
        c = np.concatenate(cols)
        self.group_size = g.fz if groups == "interface" else g.n
        self.Z = sp.coo_matrix((np.ones(r.size), (r, c)), shape=(g.k, self.d)).tocsr()
        self.S = S
        if isinstance(S, RangeProjected):
            # C = Z^T (I - u_S u_S^T) S Z = Z^T S Z - (Z^T u_S)(u_S^T S Z)
            SZ = (S.S @ self.Z).tocsr()
            self.C = (self.Z.T @ SZ).toarray() - np.outer(self.Z.T @ S.uS, SZ.T @ S.uS)
        else:
            SZ = (S @ self.Z).tocsr()
            self.C = (self.Z.T @ SZ).toarray()
        if uS is not None:
            uC = self.Z.T @ uS
            self.uC = uC / np.linalg.norm(uC)
        else:
            self.uC = None

    def coarse(self, q):
        """C \\ (q - u_C u_C^T q) for singular C: minimum-norm least squares
        ("lstsq"), the solution with its last coarse unknown set to zero
        ("pinned": the leading (d-1) x (d-1) system is solved), or the
        zero-mean solution through C + a u_C 1^T / sqrt(d) ("rank1")."""
        if self.uC is not None:
            q = q - self.uC * np.dot(self.uC, q)
            if self.coarse_mode == "pinned":
                c = np.zeros_like(q)
                if self.d > 1:
                    c[:-1] = np.linalg.solve(self.C[:-1, :-1], q[:-1])
                return c
            if self.coarse_mode == "rank1":
                # zero-mean solution of the consistent system through the
                # nonsingular C + a u_C 1^T / sqrt(d)
                a = (np.abs(self.C).max() + 2.0 * self.group_size) / np.sqrt(self.d)
                return np.linalg.solve(self.C + a * np.outer(self.uC, np.ones(self.d)), q)
            return np.linalg.lstsq(self.C, q, rcond=None)[0]
        return np.linalg.solve(self.C, q)

    def P(self, v):
        """P v = v - S Z C\\(Z^T v - u_C u_C^T Z^T v), S applied again (Sec. 3.3)."""
        return v - self.S @ (self.Z @ self.coarse(self.Z.T @ v))

    def Q(self, v):
        """Q v = v - Z C\\(Z^T S v - u_C u_C^T Z^T S v)."""
        return v - self.Z @ self.coarse(self.Z.T @ (self.S @ v))

    def coarse_part(self, b):
        """Z C \\ (Z^T b - u_C u_C^T Z^T b), Alg. seq steps 6-7."""
        return self.Z @ self.coarse(self.Z.T @ b)


def solve(g: Grid, f, gb=None, k2=0.0, method="dbj", tol=1e-13, maxiter=2000,
          groups="interface", schur=None, coarse="lstsq"):
    """Iterative oracle: Alg. seq (method 'dbj') or a comparison method.

    Returns (u, info).  u is gauge-fixed for k2 == 0.  info holds the GMRES
    iteration count, its residual history and the true Schur residual
    ||S x_S - b_S|| / ||b_S|| of the assembled solution.
    """
    sch = schur if schur is not None else StripSchur(g, k2)
    S = sch.S
    b = rhs(g, f, gb)
    uS = None
    if k2 == 0.0:
        uL, uS = sch.null_vectors()
        b = b - uL * np.dot(uL, b)                  # Alg. seq step 1
    bS = sch.B @ sch.Ainv(b)                         # step 2
    if k2 == 0.0:
        bS = bS - uS * np.dot(uS, bS)                # step 3
    info = {}
    Sraw = S
    if k2 == 0.0:
        S = RangeProjected(Sraw, uS)                 # consistent in floating point
    if method == "schur":
        xS, it, hist = householder_gmres(lambda v: S @ v, bS, tol, maxiter)
    elif method == "bj":
        M = BlockJacobi(g, Sraw, singular=(k2 == 0.0))
        y, it, hist = householder_gmres(lambda v: S @ M.solve(v), bS, tol, maxiter)
        xS = M.solve(y)
    elif method == "dbj":
        M = BlockJacobi(g, Sraw, singular=(k2 == 0.0))
        Df = Deflation(g, S, uS, groups, coarse)
        x1, it, hist = householder_gmres(lambda v: Df.P(S @ M.solve(v)), Df.P(bS), tol, maxiter)  # step 4
        x1 = Df.Q(M.solve(x1))                       # step 5
        x2 = Df.coarse_part(bS)                      # steps 6-7
        xS = x1 + x2                                 # step 8
        info["coarse_dim"] = Df.d
    elif method == "2las":
        M = BlockJacobi(g, Sraw, singular=(k2 == 0.0))
        Df = Deflation(g, S, uS, groups, coarse)
        prec = lambda v: M.solve(v) + Df.coarse_part(v)
        y, it, hist = householder_gmres(lambda v: S @ prec(v), bS, tol, maxiter)
        xS = prec(y)
    else:
        raise ValueError(method)
    u = sch.Ainv(b - sch.E @ xS)                     # step 9
    if k2 == 0.0:
        u = gauge(g, u)
    nb = np.linalg.norm(bS)
    info.update(iterations=it, history=hist,
                schur_residual=np.linalg.norm(S @ xS - bS) / (nb if nb > 0 else 1.0),
                b=b, bS=bS, xS=xS)
    return u, info
