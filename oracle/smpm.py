"""Explicit assembly of the SMPM operator and its strip split (Secs. 2.2-2.4).

Test infrastructure only (see ``oracle/__init__.py``).

What this module computes
-------------------------
* ``Grid``: an m_x x m_z element mesh of [0, l_x] x [0, l_z] with n = order + 1
  GLL points per direction per element (Sec. 2.2: r = n^2 m_x m_z nodes, face
  nodes duplicated).  Elements are uniform in x and uniform or geometrically
  stretched in z.
* ``assemble_L``: the SMPM residual operator of Eq. smpm_poisson, written out
  node by node and edge by edge (no Kronecker shortcut): the Laplacian through
  the scaled second-derivative matrix, for every element edge a node lies on
  the Robin mismatch tau [(u + n.grad u)_own - (u + n.grad u)_neighbour]
  (R_ij = I + n_i . grad, n_i the own outward normal) or, on the physical
  boundary, the Neumann penalty tau n.grad u.  For the Fourier-mode Helmholtz
  problems (Sec. 5, Eq. fourier_poisson) k^2 is subtracted on the diagonal.
* ``rhs``: f + tau g on the physical boundary rows (right side of
  Eq. smpm_poisson).
* ``split``: A (entries coupling nodes of the same vertical strip), the
  inclusion E of the interface nodes (Sec. 2.3) and B := E^T (L - A).

Readings of the paper used here (where Sec. 2.2 leaves a choice open):
* n GLL points means polynomial order N = n - 1.
* tau is not given (Sec. 2.2 leaves it to stability criteria and a
  heuristic): tau = tau_scale * (N (N + 1) / h_perp)^2 on every edge, h_perp
  the own element's length normal to that edge, tau_scale = -0.1 by default.
  In the sign convention of Eq. smpm_poisson a positive tau anti-damps the
  modes that jump across an interface (the operator then has eigenvalues with
  positive real part, an unstable discretisation, and the Helmholtz problems
  of Sec. 5 become indefinite), so the stable sign is negative.  With the
  literal Robin operator R = I + n.grad the smallest stable |tau| grows as
  N^4 / h^2: in this parameterisation it is ~0.028 at every order from 8 to
  20 and every element length from 1/128 to 2 (0.010 at order 4), so -0.1
  keeps a margin of 3.6 everywhere.  The earlier form tau_scale N (N + 1) / h
  has no such constant: at a fixed tau_scale it turns unstable as h shrinks
  (order 16 needed |tau_scale| >= 119 at h = 1/16).  tau does not depend on
  k^2 (Sec. 5).
* A corner node receives the terms of both edges it lies on.
* Neumann data g is given per physical boundary side (west/east: one value per
  z-node, south/north: one value per x-node), so a corner node sees the g of
  each of its two sides.

Node ordering (shared convention with the library API, not code): node
index = X * f_z + Z with X = e_x n + a the global x-node index and
Z = e_z n + b the global z-node index, f_z = n m_z.  Interface ordering (the
Schur grid Gamma): index = (2 j + s) f_z + Z for interface j = 0..m_x-2 between
strips j and j+1, side s = 0 for strip j's east face, s = 1 for strip j+1's
west face.
"""
import numpy as np
import scipy.sparse as sp

from .lgl import lgl_nodes_weights, diff_matrix


class Grid:
    def __init__(self, mx, mz, order, lx, lz, z_ratio=1.0, tau_scale=-0.1):
        if mx < 2 or mz < 1 or order < 1:
            raise ValueError("need mx >= 2, mz >= 1, order >= 1")
        self.mx, self.mz, self.order = int(mx), int(mz), int(order)
        self.lx, self.lz = float(lx), float(lz)
        self.z_ratio, self.tau_scale = float(z_ratio), float(tau_scale)
        n = self.n = self.order + 1
        N = self.N = self.order
        self.xi, self.w = lgl_nodes_weights(n)
        self.D = diff_matrix(self.xi)
        self.D2 = self.D @ self.D
        self.hx = self.lx / self.mx
        if self.z_ratio == 1.0:
            self.hz = np.full(self.mz, self.lz / self.mz)
        else:
            h0 = self.lz * (self.z_ratio - 1.0) / (self.z_ratio ** self.mz - 1.0)
            self.hz = h0 * self.z_ratio ** np.arange(self.mz)
        self.zb = np.concatenate([[0.0], np.cumsum(self.hz)])
        self.zb[-1] = self.lz
        self.fz = n * self.mz
        self.nx = n * self.mx
        self.r = self.nx * self.fz
        self.k = 2 * self.fz * (self.mx - 1)
        self.tau_x = self.tau_scale * (N * (N + 1) / self.hx) ** 2
        self.tau_z = self.tau_scale * (N * (N + 1) / self.hz) ** 2

    # ----- indexing -------------------------------------------------------
    def node(self, ex, a, ez, b):
        return (ex * self.n + a) * self.fz + ez * self.n + b

    def elem_nodes(self, ex, ez):
        a = np.arange(self.n)[:, None]
        b = np.arange(self.n)[None, :]
        return self.node(ex, a, ez, b)          # [a, b]

    def strip_of(self, idx):
        return np.asarray(idx) // (self.n * self.fz)

    def x_nodes(self):
        ex = np.repeat(np.arange(self.mx), self.n)
        a = np.tile(np.arange(self.n), self.mx)
        return ex * self.hx + (self.xi[a] + 1.0) * self.hx / 2.0

    def z_nodes(self):
        ez = np.repeat(np.arange(self.mz), self.n)
        b = np.tile(np.arange(self.n), self.mz)
        return self.zb[ez] + (self.xi[b] + 1.0) * self.hz[ez] / 2.0

    def coords(self):
        """(x, z) of every node, each an array of length r in node order."""
        X, Z = np.meshgrid(self.x_nodes(), self.z_nodes(), indexing="ij")
        return X.ravel(), Z.ravel()

    def quad_weights(self):
        """Per-node GLL quadrature weight w_a w_b h_x h_z / 4 (node order)."""
        wx = np.tile(self.w, self.mx) * self.hx / 2.0
        wz = (self.w[None, :] * self.hz[:, None] / 2.0).ravel()
        return np.outer(wx, wz).ravel()

    def gamma_nodes(self):
        """Node index of every interface unknown, in Gamma order."""
        out = np.empty(self.k, dtype=np.int64)
        Zs = np.arange(self.fz)
        for j in range(self.mx - 1):
            out[(2 * j) * self.fz:(2 * j + 1) * self.fz] = (j * self.n + self.N) * self.fz + Zs
            out[(2 * j + 1) * self.fz:(2 * j + 2) * self.fz] = ((j + 1) * self.n) * self.fz + Zs
        return out


def assemble_L(g: Grid, k2=0.0):
    """Sparse SMPM operator L - k^2 I (CSR), assembled node by node, edge by edge."""
    n, N, D, D2 = g.n, g.N, g.D, g.D2
    rows, cols, vals = [], [], []

    def put(r, c, v):
        r, c, v = np.broadcast_arrays(r, c, v)
        rows.append(r.ravel())
        cols.append(c.ravel())
        vals.append(v.ravel())

    sx = 2.0 / g.hx
    for ex in range(g.mx):
        for ez in range(g.mz):
            idx = g.elem_nodes(ex, ez)                 # [a, b]
            sz = 2.0 / g.hz[ez]
            tx, tz = g.tau_x, g.tau_z[ez]
            # Laplacian: d2/dx2 along each x-line, d2/dz2 along each z-line
            put(idx[:, None, :], idx[None, :, :], (sx * sx) * D2[:, :, None])
            put(idx[:, :, None], idx[:, None, :], (sz * sz) * D2[None, :, :])
            # west edge (a = 0), outward normal -x
            rw = idx[0, :]                               # rows, one per b
            if ex == 0:
                put(rw[:, None], idx[:, :].T, -tx * sx * D[0, :][None, :])
            else:
                nb = g.elem_nodes(ex - 1, ez)
                put(rw, rw, tx)
                put(rw[:, None], idx.T, -tx * sx * D[0, :][None, :])
                put(rw, nb[N, :], -tx)
                put(rw[:, None], nb.T, tx * sx * D[N, :][None, :])
            # east edge (a = N), outward normal +x
            re = idx[N, :]
            if ex == g.mx - 1:
                put(re[:, None], idx.T, tx * sx * D[N, :][None, :])
            else:
                nb = g.elem_nodes(ex + 1, ez)
                put(re, re, tx)
                put(re[:, None], idx.T, tx * sx * D[N, :][None, :])
                put(re, nb[0, :], -tx)
                put(re[:, None], nb.T, -tx * sx * D[0, :][None, :])
            # south edge (b = 0), outward normal -z
            rs = idx[:, 0]
            if ez == 0:
                put(rs[:, None], idx, -tz * sz * D[0, :][None, :])
            else:
                nb = g.elem_nodes(ex, ez - 1)
                szn = 2.0 / g.hz[ez - 1]
                put(rs, rs, tz)
                put(rs[:, None], idx, -tz * sz * D[0, :][None, :])
                put(rs, nb[:, N], -tz)
                put(rs[:, None], nb, tz * szn * D[N, :][None, :])
            # north edge (b = N), outward normal +z
            rn = idx[:, N]
            if ez == g.mz - 1:
                put(rn[:, None], idx, tz * sz * D[N, :][None, :])
            else:
                nb = g.elem_nodes(ex, ez + 1)
                szn = 2.0 / g.hz[ez + 1]
                put(rn, rn, tz)
                put(rn[:, None], idx, tz * sz * D[N, :][None, :])
                put(rn, nb[:, 0], -tz)
                put(rn[:, None], nb, -tz * szn * D[0, :][None, :])
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    v = np.concatenate(vals)
    L = sp.coo_matrix((v, (r, c)), shape=(g.r, g.r)).tocsr()
    L.sum_duplicates()
    if k2 != 0.0:
        L = (L - k2 * sp.identity(g.r, format="csr")).tocsr()
    return L


def zero_g(g: Grid):
    return {"west": np.zeros(g.fz), "east": np.zeros(g.fz),
            "south": np.zeros(g.nx), "north": np.zeros(g.nx)}


def rhs(g: Grid, f, gb=None):
    """b = f + tau g on the physical boundary rows (Eq. smpm_poisson)."""
    b = np.array(f, dtype=np.float64, copy=True)
    if gb is None:
        return b
    U = b.reshape(g.nx, g.fz)
    U[0, :] += g.tau_x * np.asarray(gb["west"])
    U[g.nx - 1, :] += g.tau_x * np.asarray(gb["east"])
    U[:, 0] += g.tau_z[0] * np.asarray(gb["south"])
    U[:, g.fz - 1] += g.tau_z[g.mz - 1] * np.asarray(gb["north"])
    return U.ravel()


def split(g: Grid, L):
    """Return (A, E, B): strip-local part, interface inclusion and B = E^T (L - A)."""
    Lc = L.tocoo()
    same = g.strip_of(Lc.row) == g.strip_of(Lc.col)
    A = sp.coo_matrix((Lc.data[same], (Lc.row[same], Lc.col[same])), shape=L.shape).tocsr()
    gam = g.gamma_nodes()
    E = sp.coo_matrix((np.ones(g.k), (gam, np.arange(g.k))), shape=(g.r, g.k)).tocsr()
    B = (E.T @ (L - A)).tocsr()
    return A, E, B


def gauge(g: Grid, u):
    """Remove the GLL-quadrature mean (fixes the additive constant of the Neumann problem)."""
    W = g.quad_weights()
    return u - np.dot(W, u) / (g.lx * g.lz)


def left_null_dense(M, polish=2):
    """Unit left null vector of a dense singular M and M's singular values.

    The left singular vector of the smallest singular value is polished by a
    few steps of inverse iteration with (M^T - sigma I), sigma a tiny multiple
    of max|M| (the SVD vector alone leaves ||v^T M|| near 1e-10 ||M||, which
    the Neumann problem amplifies into ~1e-8 solution differences).  Sign
    fixed so that the entry of largest magnitude is positive.
    """
    U, s, Vt = np.linalg.svd(M)
    v = U[:, -1]
    if polish:
        sigma = 1e-12 * np.abs(M).max()
        T = M.T - sigma * np.eye(M.shape[0])
        for _ in range(polish):
            v = np.linalg.solve(T, v)
            v /= np.linalg.norm(v)
    if v[np.argmax(np.abs(v))] < 0:
        v = -v
    return v, s


def direct_solve(g: Grid, f, gb=None, k2=0.0):
    """Plain-definition solve on tiny grids: dense L, SVD null vector, lstsq.

    Returns (u, info): for k2 == 0 the RHS is projected out of the left null
    space of L (Eq. regularize_poisson) and u is gauge-fixed to zero mean.
    """
    L = assemble_L(g, k2).toarray()
    b = rhs(g, f, gb)
    info = {}
    if k2 == 0.0:
        uL, s = left_null_dense(L)
        info["sv"] = s
        info["uL"] = uL
        b = b - uL * np.dot(uL, b)
        u = np.linalg.lstsq(L, b, rcond=None)[0]
        u = gauge(g, u)
    else:
        u = np.linalg.solve(L, b)
    info["b"] = b
    return u, info
