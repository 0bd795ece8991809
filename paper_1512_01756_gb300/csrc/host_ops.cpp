// Host-side FP64 builders of libsmpm: GLL data, the 1-D factors of the SMPM
// operator, a banded LU for the null vectors and the deflation coarse operator.
//
// Sec. 2.2 (Eq. smpm_poisson): on every element the residual is the Laplacian
// plus, on each edge, tau * [(u + n.grad u)_own - (u + n.grad u)_neighbour]
// (interior edge, n the own outward normal) or tau * n.grad u (physical edge).
// With tau constant along each edge direction and a corner node taking the
// terms of both its edges, L is exactly the Kronecker sum L_x (+) L_z of a 1-D
// x-operator and a 1-D z-operator; the strip-local part A of Sec. 2.3 is
// A_i = Ax_{c(i)} (+) L_z with Ax_c the x-operator of one strip (own parts of
// the x-face terms only).  These builders produce those 1-D factors.
#include "smpm_internal.h"

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <functional>

namespace smpm {

// --- GLL nodes, weights, differentiation (Sec. 2.2) --------------------------

static void legendre_pn(int N, double x, double& p, double& pm1) {
    double a = 1.0, b = x;
    if (N == 0) { p = 1.0; pm1 = 0.0; return; }
    for (int m = 2; m <= N; ++m) {
        double c = ((2.0 * m - 1.0) * x * b - (m - 1.0) * a) / m;
        a = b;
        b = c;
    }
    p = b;
    pm1 = a;
}

void gll(int n, std::vector<double>& x, std::vector<double>& w) {
    const int N = n - 1;
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < n; ++i) x[i] = -std::cos(pi * i / N);
    // interior nodes: roots of P_N' by Newton; P_N' = N (x P_N - P_{N-1}) / (x^2 - 1),
    // P_N'' from (1 - x^2) P'' = 2 x P' - N (N + 1) P.
    for (int i = 1; i < N; ++i) {
        double xi = x[i];
        for (int it = 0; it < 200; ++it) {
            double p, q;
            legendre_pn(N, xi, p, q);
            double d1 = N * (xi * p - q) / (xi * xi - 1.0);
            double d2 = (2.0 * xi * d1 - N * (N + 1.0) * p) / (1.0 - xi * xi);
            double step = d1 / d2;
            xi -= step;
            if (std::fabs(step) < 1e-16) break;
        }
        x[i] = xi;
    }
    x[0] = -1.0;
    x[N] = 1.0;
    if (n % 2 == 1) x[N / 2] = 0.0;
    for (int i = 0; i < n; ++i) {  // symmetrise the node set exactly
        if (i < n - 1 - i) {
            double s = 0.5 * (x[n - 1 - i] - x[i]);
            x[i] = -s;
            x[n - 1 - i] = s;
        }
    }
    for (int i = 0; i < n; ++i) {
        double p, q;
        legendre_pn(N, x[i], p, q);
        w[i] = 2.0 / (N * (N + 1.0) * p * p);
    }
}

void gll_diff(const std::vector<double>& x, std::vector<double>& D) {
    const int n = (int)x.size(), N = n - 1;
    std::vector<double> p(n);
    for (int i = 0; i < n; ++i) {
        double q;
        legendre_pn(N, x[i], p[i], q);
    }
    D.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int j = 0; j < n; ++j) {
            if (i == j) continue;
            double v = p[i] / (p[j] * (x[i] - x[j]));
            D[(size_t)i * n + j] = v;
            s += v;
        }
        D[(size_t)i * n + i] = -s;  // rows annihilate constants exactly
    }
}

bool make_geometry(int mx, int mz, int order, double lx, double lz, double z_ratio,
                   double tau_scale, int groups, Geometry& g, std::string& msg) {
    if (mx < 2 || mz < 1 || order < 1 || order > 32) {
        msg = "need mx >= 2, mz >= 1, 1 <= order <= 32";
        return false;
    }
    if (!(lx > 0) || !(lz > 0)) { msg = "domain lengths must be positive"; return false; }
    if (z_ratio == 0.0) z_ratio = 1.0;
    if (tau_scale == 0.0) tau_scale = -0.1;
    if (!(z_ratio > 0)) { msg = "z_ratio must be positive"; return false; }
    if (!std::isfinite(tau_scale)) { msg = "tau_scale must be finite"; return false; }
    if (groups != 0 && groups != 1) { msg = "deflation_groups must be 0 or 1"; return false; }
    g.mx = mx; g.mz = mz; g.order = order; g.n = order + 1; g.N = order;
    g.lx = lx; g.lz = lz; g.z_ratio = z_ratio; g.tau_scale = tau_scale;
    g.fz = g.n * mz;
    g.nx = g.n * mx;
    g.r = (long long)g.nx * g.fz;
    g.k = 2LL * g.fz * (mx - 1);
    g.hx = lx / mx;
    g.hz.assign(mz, lz / mz);
    if (z_ratio != 1.0) {
        double h0 = lz * (z_ratio - 1.0) / (std::pow(z_ratio, mz) - 1.0);
        for (int e = 0; e < mz; ++e) g.hz[e] = h0 * std::pow(z_ratio, e);
    }
    g.zb.assign(mz + 1, 0.0);
    for (int e = 0; e < mz; ++e) g.zb[e + 1] = g.zb[e] + g.hz[e];
    g.zb[mz] = lz;
    // tau = tau_scale (N (N+1) / h_perp)^2 per edge, h_perp the own element's
    // length normal to the edge: the smallest |tau| without anti-damped jump
    // modes grows as N^4 / h^2 and is ~0.028 (N (N+1) / h)^2 at every order
    const double NN = (double)g.N * (g.N + 1.0);
    g.tau_x = tau_scale * (NN / g.hx) * (NN / g.hx);
    g.tau_z.resize(mz);
    for (int e = 0; e < mz; ++e) g.tau_z[e] = tau_scale * (NN / g.hz[e]) * (NN / g.hz[e]);
    gll(g.n, g.xi, g.w);
    gll_diff(g.xi, g.D);
    const int n = g.n;
    g.D2.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double s = 0.0;
            for (int l = 0; l < n; ++l) s += g.D[(size_t)i * n + l] * g.D[(size_t)l * n + j];
            g.D2[(size_t)i * n + j] = s;
        }
    g.ng = groups == 1 ? mz : 1;
    g.d = (mx - 1) * g.ng;
    if (g.d > 4096) { msg = "coarse dimension above 4096"; return false; }
    return true;
}

// --- 1-D operators ------------------------------------------------------------

using Adder = std::function<void(int, int, double)>;

// x-operator rows of element ex placed at offset off (off = ex*n for the full
// operator, 0 for a single strip); neighbours are coupled only if `full`.
static void x_element_rows(const Geometry& g, int ex, int off, bool full, const Adder& add) {
    const int n = g.n, N = g.N;
    const double sx = 2.0 / g.hx, t = g.tau_x;
    const double* D = g.D.data();
    const double* D2 = g.D2.data();
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b) add(off + a, off + b, sx * sx * D2[a * n + b]);
    // west face, outward normal -x
    if (ex == 0) {
        for (int b = 0; b < n; ++b) add(off, off + b, -t * sx * D[0 * n + b]);
    } else {
        add(off, off, t);
        for (int b = 0; b < n; ++b) add(off, off + b, -t * sx * D[0 * n + b]);
        if (full) {
            int nb = off - n;
            add(off, nb + N, -t);
            for (int b = 0; b < n; ++b) add(off, nb + b, t * sx * D[N * n + b]);
        }
    }
    // east face, outward normal +x
    if (ex == g.mx - 1) {
        for (int b = 0; b < n; ++b) add(off + N, off + b, t * sx * D[N * n + b]);
    } else {
        add(off + N, off + N, t);
        for (int b = 0; b < n; ++b) add(off + N, off + b, t * sx * D[N * n + b]);
        if (full) {
            int nb = off + n;
            add(off + N, nb, -t);
            for (int b = 0; b < n; ++b) add(off + N, nb + b, -t * sx * D[0 * n + b]);
        }
    }
}

static void z_rows(const Geometry& g, const Adder& add) {
    const int n = g.n, N = g.N;
    const double* D = g.D.data();
    const double* D2 = g.D2.data();
    for (int e = 0; e < g.mz; ++e) {
        const int off = e * n;
        const double s = 2.0 / g.hz[e], t = g.tau_z[e];
        for (int a = 0; a < n; ++a)
            for (int b = 0; b < n; ++b) add(off + a, off + b, s * s * D2[a * n + b]);
        if (e == 0) {
            for (int b = 0; b < n; ++b) add(off, off + b, -t * s * D[0 * n + b]);
        } else {
            const double sn = 2.0 / g.hz[e - 1];
            const int nb = off - n;
            add(off, off, t);
            for (int b = 0; b < n; ++b) add(off, off + b, -t * s * D[0 * n + b]);
            add(off, nb + N, -t);
            for (int b = 0; b < n; ++b) add(off, nb + b, t * sn * D[N * n + b]);
        }
        if (e == g.mz - 1) {
            for (int b = 0; b < n; ++b) add(off + N, off + b, t * s * D[N * n + b]);
        } else {
            const double sn = 2.0 / g.hz[e + 1];
            const int nb = off + n;
            add(off + N, off + N, t);
            for (int b = 0; b < n; ++b) add(off + N, off + b, t * s * D[N * n + b]);
            add(off + N, nb, -t);
            for (int b = 0; b < n; ++b) add(off + N, nb + b, -t * sn * D[0 * n + b]);
        }
    }
}

void strip_x_operator(const Geometry& g, int cls, std::vector<double>& Ax) {
    const int n = g.n;
    Ax.assign((size_t)n * n, 0.0);
    int ex = cls == 0 ? 0 : (cls == 2 ? g.mx - 1 : 1);
    if (cls == 1 && g.mx < 3) ex = 1;  // unused class when mx == 2, still well formed
    Geometry gg = g;
    if (cls == 1 && g.mx < 3) gg.mx = 3;
    x_element_rows(gg, ex, 0, false, [&](int i, int j, double v) { Ax[(size_t)i * n + j] += v; });
}

void z_operator(const Geometry& g, std::vector<double>& Lz) {
    const int fz = g.fz;
    Lz.assign((size_t)fz * fz, 0.0);
    z_rows(g, [&](int i, int j, double v) { Lz[(size_t)i * fz + j] += v; });
}

void face_flux_rows(const Geometry& g, int cls, std::vector<double>& beta) {
    const int n = g.n, N = g.N;
    const double sx = 2.0 / g.hx, t = g.tau_x;
    beta.assign(2 * (size_t)n, 0.0);
    if (cls != 0)  // flux onto the west neighbour's east face: -tau (u + d/dx u) at a = 0
        for (int a = 0; a < n; ++a) beta[a] = -t * ((a == 0 ? 1.0 : 0.0) + sx * g.D[0 * n + a]);
    if (cls != 2)  // flux onto the east neighbour's west face: -tau (u - d/dx u) at a = N
        for (int a = 0; a < n; ++a) beta[n + a] = -t * ((a == N ? 1.0 : 0.0) - sx * g.D[N * n + a]);
}

// --- banded LU (column band storage; the LAPACK gbtf2/gbtrs scheme) -----------

void BandLU::init(int n_, int kl_, int ku_) {
    n = n_; kl = kl_; ku = ku_;
    ldab = 2 * kl + ku + 1;
    ab.assign((size_t)ldab * n, 0.0);
    piv.assign(n, 0);
}

bool BandLU::factor() {
    const int kv = kl + ku;
    int ju = 0;
    bool ok = true;
    for (int j = 0; j < n; ++j) {
        int km = std::min(kl, n - 1 - j);
        int p = 0;
        double best = std::fabs(at(j, j));
        for (int i = 1; i <= km; ++i)
            if (std::fabs(at(j + i, j)) > best) { best = std::fabs(at(j + i, j)); p = i; }
        piv[j] = j + p;
        if (best == 0.0) { ok = false; continue; }
        ju = std::max(ju, std::min(j + ku + p, n - 1));
        if (p != 0)
            for (int c = j; c <= ju; ++c) std::swap(at(j, c), at(j + p, c));
        if (km > 0) {
            double inv = 1.0 / at(j, j);
            for (int i = 1; i <= km; ++i) at(j + i, j) *= inv;
            for (int c = j + 1; c <= ju; ++c) {
                double t = at(j, c);
                if (t != 0.0)
                    for (int i = 1; i <= km; ++i) at(j + i, c) -= at(j + i, j) * t;
            }
        }
    }
    (void)kv;
    return ok;
}

void BandLU::solve(double* b) const {
    const int kv = kl + ku;
    for (int j = 0; j < n; ++j) {
        int p = piv[j];
        if (p != j) std::swap(b[j], b[p]);
        int km = std::min(kl, n - 1 - j);
        for (int i = 1; i <= km; ++i) b[j + i] -= at(j + i, j) * b[j];
    }
    for (int j = n - 1; j >= 0; --j) {
        b[j] /= at(j, j);
        int i0 = std::max(0, j - kv);
        for (int i = i0; i < j; ++i) b[i] -= at(i, j) * b[j];
    }
}

void BandLU::solve_T(double* b) const {
    const int kv = kl + ku;
    for (int j = 0; j < n; ++j) {
        double t = b[j];
        int i0 = std::max(0, j - kv);
        for (int i = i0; i < j; ++i) t -= at(i, j) * b[i];
        b[j] = t / at(j, j);
    }
    for (int j = n - 2; j >= 0; --j) {
        int km = std::min(kl, n - 1 - j);
        double t = b[j];
        for (int i = 1; i <= km; ++i) t -= at(j + i, j) * b[j + i];
        b[j] = t;
        int p = piv[j];
        if (p != j) std::swap(b[j], b[p]);
    }
}

// Left null vector by inverse iteration on a band built by `fill`, after
// scaling every row to unit maximum (D L: the penalty rows are ~1e6 times
// the Laplacian rows, and the LU's rounding then stays relative to each row
// instead of to the largest one).  w^T (D L) = 0 gives u = D w.  The shift
// sigma = 1e-15 must stay far below the smallest nonzero eigenvalue of D L;
// a larger one only if that factorisation meets an exact zero pivot.
static bool left_null_from(int n, int bw, const std::function<void(const Adder&)>& fill,
                           std::vector<double>& v, std::string& msg) {
    msg = "null-vector factorisation hit a zero pivot";
    for (double sigma : {1e-15, 1e-13, 1e-12}) {
        BandLU lu;
        lu.init(n, bw, bw);
        fill([&](int i, int j, double x) { lu.at(i, j) += x; });
        std::vector<double> d(n, 0.0);
        for (int i = 0; i < n; ++i) {
            for (int j = std::max(0, i - bw); j <= std::min(n - 1, i + bw); ++j)
                d[i] = std::max(d[i], std::fabs(lu.at(i, j)));
            d[i] = d[i] > 0.0 ? 1.0 / d[i] : 1.0;
            for (int j = std::max(0, i - bw); j <= std::min(n - 1, i + bw); ++j) lu.at(i, j) *= d[i];
        }
        for (int i = 0; i < n; ++i) lu.at(i, i) -= sigma;
        if (!lu.factor()) continue;
        std::vector<double> w(n);
        for (int i = 0; i < n; ++i) w[i] = 1.0 + 0.01 * std::sin(1.0 + 3.0 * i);
        bool ok = true;
        for (int it = 0; it < 6 && ok; ++it) {
            lu.solve_T(w.data());
            double s = 0.0;
            for (double x : w) s += x * x;
            s = std::sqrt(s);
            if (!(s > 0) || !std::isfinite(s)) {
                msg = "null-vector iteration diverged";
                ok = false;
                break;
            }
            for (double& x : w) x /= s;
        }
        if (!ok) continue;
        v.assign(n, 0.0);
        double s = 0.0;
        for (int i = 0; i < n; ++i) {
            v[i] = d[i] * w[i];
            s += v[i] * v[i];
        }
        s = std::sqrt(s);
        for (double& x : v) x /= s;
        return true;
    }
    return false;
}

bool left_null_banded(const std::vector<double>& M, int n, int bw, std::vector<double>& v,
                      std::string& msg) {
    return left_null_from(n, bw, [&](const Adder& add) {
        for (int i = 0; i < n; ++i)
            for (int j = std::max(0, i - bw); j <= std::min(n - 1, i + bw); ++j)
                if (M[(size_t)i * n + j] != 0.0) add(i, j, M[(size_t)i * n + j]);
    }, v, msg);
}

bool left_null_x(const Geometry& g, std::vector<double>& v, std::string& msg) {
    return left_null_from(g.nx, g.n, [&](const Adder& add) {
        for (int ex = 0; ex < g.mx; ++ex) x_element_rows(g, ex, ex * g.n, true, add);
    }, v, msg);
}

bool left_null_z(const Geometry& g, std::vector<double>& v, std::string& msg) {
    return left_null_from(g.fz, g.n, [&](const Adder& add) { z_rows(g, add); }, v, msg);
}

void full_x_operator(const Geometry& g, std::vector<double>& Lx) {
    const int nx = g.nx;
    Lx.assign((size_t)nx * nx, 0.0);
    for (int ex = 0; ex < g.mx; ++ex)
        x_element_rows(g, ex, ex * g.n, true, [&](int i, int j, double v) { Lx[(size_t)i * nx + j] += v; });
}

// --- deflation coarse operator (Sec. 3.3) ---------------------------------------

// Dense LU with partial pivoting of A (d x d row-major, overwritten), then
// X <- A^-1 X for the d x nb row-major right-hand sides X.
static bool dense_solve(std::vector<double>& A, int d, std::vector<double>& X, int nb) {
    std::vector<int> piv(d);
    for (int k = 0; k < d; ++k) {
        int p = k;
        double best = std::fabs(A[(size_t)k * d + k]);
        for (int i = k + 1; i < d; ++i)
            if (std::fabs(A[(size_t)i * d + k]) > best) { best = std::fabs(A[(size_t)i * d + k]); p = i; }
        if (best == 0.0) return false;
        piv[k] = p;
        if (p != k) {
            for (int j = 0; j < d; ++j) std::swap(A[(size_t)k * d + j], A[(size_t)p * d + j]);
            for (int j = 0; j < nb; ++j) std::swap(X[(size_t)k * nb + j], X[(size_t)p * nb + j]);
        }
        const double inv = 1.0 / A[(size_t)k * d + k];
        for (int i = k + 1; i < d; ++i) {
            const double l = A[(size_t)i * d + k] * inv;
            if (l == 0.0) continue;
            A[(size_t)i * d + k] = l;
            double* ai = &A[(size_t)i * d];
            const double* ak = &A[(size_t)k * d];
            for (int j = k + 1; j < d; ++j) ai[j] -= l * ak[j];
            double* xi = &X[(size_t)i * nb];
            const double* xk = &X[(size_t)k * nb];
            for (int j = 0; j < nb; ++j) xi[j] -= l * xk[j];
        }
    }
    for (int k = d - 1; k >= 0; --k) {
        const double inv = 1.0 / A[(size_t)k * d + k];
        double* xk = &X[(size_t)k * nb];
        for (int j = 0; j < nb; ++j) xk[j] *= inv;
        for (int i = 0; i < k; ++i) {
            const double a = A[(size_t)i * d + k];
            if (a == 0.0) continue;
            double* xi = &X[(size_t)i * nb];
            for (int j = 0; j < nb; ++j) xi[j] -= a * xk[j];
        }
    }
    return true;
}

void coarse_matrix(std::vector<double>& C, int d, int fz_over_ng, const double* uC) {
    // Singular C (k^2 = 0): C 1 = 0 and u_C^T C = 0.  The regularised division
    // C \ (I - u_C u_C^T) q is taken as the zero-mean solution of the consistent
    // system, obtained from the nonsingular C + alpha u_C 1^T / sqrt(d): for
    // q' = (I - u_C u_C^T) q it returns c with C c = q' and 1^T c = 0, and it
    // absorbs the rounding-level part of q' outside range(C) smoothly.  The
    // caller forms K = (C + alpha u_C 1^T / sqrt(d))^-1 (I - u_C u_C^T).
    // Nonsingular C (k^2 > 0): C is left as it is and K = C^-1.
    if (!uC) return;
    double amax = 0.0;
    for (double v : C) amax = std::max(amax, std::fabs(v));
    // scale of the rank-1 term: |C| plus the identity part of each coarse
    // entry (2 fz / ng), so that a ~0 1 x 1 coarse matrix (mx = 2) stays regular
    const double a = (amax + 2.0 * (double)fz_over_ng) / std::sqrt((double)d);
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) C[(size_t)i * d + j] += a * uC[i];
}

// LU factorisation with partial pivoting of a tridiagonal matrix (the coarse
// matrix with one deflation vector per interface couples each interface to its
// two neighbours only).  On entry dl[i] = T(i+1, i), dd[i] = T(i, i),
// du[i] = T(i, i+1); on exit dl holds the multipliers, dd the diagonal of U,
// du and du2 its first and second superdiagonals, and swap[i] = 1 where rows
// i and i+1 were interchanged at step i.  Row interchanges between neighbours
// are the only fill-in, into du2.  Returns false if a pivot is zero.
bool tridiag_lu(int d, std::vector<double>& dl, std::vector<double>& dd, std::vector<double>& du,
                std::vector<double>& du2, std::vector<int>& swap) {
    du2.assign((size_t)std::max(d - 2, 0), 0.0);
    swap.assign((size_t)std::max(d - 1, 0), 0);
    for (int i = 0; i + 1 < d; ++i) {
        if (std::fabs(dd[i]) >= std::fabs(dl[i])) {
            if (dd[i] == 0.0) return false;
            const double l = dl[i] / dd[i];
            dl[i] = l;
            dd[i + 1] -= l * du[i];
        } else {
            // rows i and i+1 trade places: the new row i is the old row i+1
            // (dl[i], dd[i+1], du[i+1]), the eliminated one the old row i
            const double l = dd[i] / dl[i];
            dd[i] = dl[i];
            dl[i] = l;
            const double u1 = du[i];
            du[i] = dd[i + 1];
            dd[i + 1] = u1 - l * dd[i + 1];
            if (i + 2 < d) {
                du2[i] = du[i + 1];
                du[i + 1] = -l * du[i + 1];
            }
            swap[i] = 1;
        }
    }
    return d == 0 || dd[d - 1] != 0.0;
}

// --- real block diagonalisation of a small nonsymmetric matrix ----------------
//
// Ax = Q B Q^-1 with B block diagonal: a 1 x 1 block per real eigenvalue and a
// 2 x 2 block [[alpha, beta], [-beta, alpha]] per complex pair alpha +- i beta,
// whose columns in Q are (Re v, Im v) of the eigenvector of alpha + i beta.
// Eigenvalues by the shifted QR iteration (Wilkinson shift, complex arithmetic,
// deflation from the bottom), eigenvectors by inverse iteration.  Intended for
// the n x n (n <= 33) strip x-factors; the caller checks ||Q B Q^-1 - Ax||.

using cplx = std::complex<double>;

static void qr_step(std::vector<cplx>& H, int n, int m, cplx mu) {
    // one shifted QR step on the leading m x m block of the n x n row-major H
    std::vector<cplx> A((size_t)m * m), Qm((size_t)m * m, 0.0);
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) A[(size_t)i * m + j] = H[(size_t)i * n + j] - (i == j ? mu : 0.0);
    // Householder QR: A = Q R, accumulate Q
    for (int i = 0; i < m; ++i) Qm[(size_t)i * m + i] = 1.0;
    for (int k = 0; k < m - 1; ++k) {
        double nx = 0.0;
        for (int i = k; i < m; ++i) nx += std::norm(A[(size_t)i * m + k]);
        nx = std::sqrt(nx);
        if (nx == 0.0) continue;
        cplx a0 = A[(size_t)k * m + k];
        cplx ph = std::abs(a0) > 0 ? a0 / std::abs(a0) : cplx(1.0, 0.0);
        std::vector<cplx> v(m, 0.0);
        v[k] = a0 + ph * nx;
        for (int i = k + 1; i < m; ++i) v[i] = A[(size_t)i * m + k];
        double vn = 0.0;
        for (int i = k; i < m; ++i) vn += std::norm(v[i]);
        if (vn == 0.0) continue;
        for (int j = 0; j < m; ++j) {             // A <- (I - 2 v v^H / |v|^2) A
            cplx s = 0.0;
            for (int i = k; i < m; ++i) s += std::conj(v[i]) * A[(size_t)i * m + j];
            s *= 2.0 / vn;
            for (int i = k; i < m; ++i) A[(size_t)i * m + j] -= v[i] * s;
        }
        for (int i = 0; i < m; ++i) {             // Q <- Q (I - 2 v v^H / |v|^2)
            cplx s = 0.0;
            for (int j = k; j < m; ++j) s += Qm[(size_t)i * m + j] * v[j];
            s *= 2.0 / vn;
            for (int j = k; j < m; ++j) Qm[(size_t)i * m + j] -= s * std::conj(v[j]);
        }
    }
    // H_m <- R Q + mu I
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) {
            cplx s = 0.0;
            for (int l = i; l < m; ++l) s += A[(size_t)i * m + l] * Qm[(size_t)l * m + j];
            H[(size_t)i * n + j] = s + (i == j ? mu : 0.0);
        }
}

static bool eigenvalues(const std::vector<double>& Ax, int n, std::vector<cplx>& lam) {
    std::vector<cplx> H((size_t)n * n);
    double scale = 0.0;
    for (int i = 0; i < n * n; ++i) {
        H[i] = Ax[i];
        scale = std::max(scale, std::fabs(Ax[i]));
    }
    lam.assign(n, 0.0);
    int m = n, iters = 0;
    while (m > 1) {
        const cplx sub = H[(size_t)(m - 1) * n + (m - 2)];
        double offrow = 0.0;
        for (int j = 0; j < m - 1; ++j) offrow = std::max(offrow, std::abs(H[(size_t)(m - 1) * n + j]));
        if (offrow <= 1e-15 * scale) {
            lam[m - 1] = H[(size_t)(m - 1) * n + (m - 1)];
            --m;
            iters = 0;
            continue;
        }
        (void)sub;
        if (++iters > 200) return false;
        // Wilkinson shift: eigenvalue of the trailing 2 x 2 closer to the corner
        const cplx a = H[(size_t)(m - 2) * n + (m - 2)], b = H[(size_t)(m - 2) * n + (m - 1)];
        const cplx c = H[(size_t)(m - 1) * n + (m - 2)], d = H[(size_t)(m - 1) * n + (m - 1)];
        const cplx tr = a + d, det = a * d - b * c;
        const cplx disc = std::sqrt(tr * tr - 4.0 * det);
        const cplx l1 = 0.5 * (tr + disc), l2 = 0.5 * (tr - disc);
        cplx mu = std::abs(l1 - d) < std::abs(l2 - d) ? l1 : l2;
        if (iters % 11 == 10) mu += cplx(0.0, 1e-3 * scale * 1e-6);  // exceptional shift
        qr_step(H, n, m, mu);
    }
    lam[0] = H[0];
    return true;
}

// complex LU solve (A - mu I) x = b in place, A real n x n
static bool shifted_solve(const std::vector<double>& Ax, int n, cplx mu, std::vector<cplx>& x) {
    std::vector<cplx> A((size_t)n * n);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) A[(size_t)i * n + j] = Ax[(size_t)i * n + j] - (i == j ? mu : 0.0);
    for (int k = 0; k < n; ++k) {
        int p = k;
        for (int i = k + 1; i < n; ++i)
            if (std::abs(A[(size_t)i * n + k]) > std::abs(A[(size_t)p * n + k])) p = i;
        if (std::abs(A[(size_t)p * n + k]) == 0.0) return false;
        if (p != k) {
            for (int j = 0; j < n; ++j) std::swap(A[(size_t)k * n + j], A[(size_t)p * n + j]);
            std::swap(x[k], x[p]);
        }
        for (int i = k + 1; i < n; ++i) {
            const cplx l = A[(size_t)i * n + k] / A[(size_t)k * n + k];
            for (int j = k + 1; j < n; ++j) A[(size_t)i * n + j] -= l * A[(size_t)k * n + j];
            x[i] -= l * x[k];
        }
    }
    for (int k = n - 1; k >= 0; --k) {
        cplx s = x[k];
        for (int j = k + 1; j < n; ++j) s -= A[(size_t)k * n + j] * x[j];
        x[k] = s / A[(size_t)k * n + k];
    }
    return true;
}

bool real_block_diagonalise(const std::vector<double>& Ax, int n, std::vector<double>& Q, std::vector<double>& Qinv,
                            std::vector<int>& slot_start, std::vector<int>& slot_size, std::vector<double>& alpha,
                            std::vector<double>& beta, std::string& msg) {
    std::vector<cplx> lam;
    if (!eigenvalues(Ax, n, lam)) { msg = "x-factor eigenvalue iteration did not converge"; return false; }
    double scale = 0.0;
    for (double v : Ax) scale = std::max(scale, std::fabs(v));
    // order: real eigenvalues and one representative (Im > 0) per complex pair
    std::vector<cplx> reps;
    std::vector<bool> used(n, false);
    for (int i = 0; i < n; ++i) {
        if (used[i]) continue;
        used[i] = true;
        if (std::fabs(lam[i].imag()) <= 1e-10 * std::abs(lam[i]) + 1e-14 * scale) {
            reps.push_back(cplx(lam[i].real(), 0.0));
            continue;
        }
        int best = -1;
        double bd = 1e300;
        for (int j = 0; j < n; ++j)
            if (!used[j] && std::abs(lam[j] - std::conj(lam[i])) < bd) { bd = std::abs(lam[j] - std::conj(lam[i])); best = j; }
        if (best < 0 || bd > 1e-6 * std::abs(lam[i])) { msg = "unpaired complex eigenvalue"; return false; }
        used[best] = true;
        reps.push_back(lam[i].imag() > 0 ? lam[i] : std::conj(lam[i]));
    }
    Q.assign((size_t)n * n, 0.0);
    slot_start.clear(); slot_size.clear(); alpha.clear(); beta.clear();
    int col = 0;
    for (const cplx& l : reps) {
        std::vector<cplx> v(n);
        for (int i = 0; i < n; ++i) v[i] = cplx(1.0 + 0.1 * std::sin(1.0 + 7.0 * i), 0.3 * std::cos(2.0 + 5.0 * i));
        const cplx mu = l + cplx(1e-12 * scale, 1e-12 * scale);
        for (int it = 0; it < 3; ++it) {
            if (!shifted_solve(Ax, n, mu, v)) { msg = "eigenvector solve failed"; return false; }
            double nv = 0.0;
            for (const cplx& x : v) nv += std::norm(x);
            nv = std::sqrt(nv);
            for (cplx& x : v) x /= nv;
        }
        // rotate the phase so the largest entry is real
        int im = 0;
        for (int i = 1; i < n; ++i) if (std::abs(v[i]) > std::abs(v[im])) im = i;
        const cplx ph = std::conj(v[im]) / std::abs(v[im]);
        for (cplx& x : v) x *= ph;
        if (l.imag() == 0.0) {
            if (col >= n) { msg = "too many eigenvectors"; return false; }
            double nr = 0.0;
            for (int i = 0; i < n; ++i) nr += v[i].real() * v[i].real();
            nr = std::sqrt(nr);
            for (int i = 0; i < n; ++i) Q[(size_t)i * n + col] = v[i].real() / nr;
            slot_start.push_back(col); slot_size.push_back(1); alpha.push_back(l.real()); beta.push_back(0.0);
            col += 1;
        } else {
            if (col + 1 >= n) { msg = "too many eigenvectors"; return false; }
            for (int i = 0; i < n; ++i) {
                Q[(size_t)i * n + col] = v[i].real();
                Q[(size_t)i * n + col + 1] = v[i].imag();
            }
            slot_start.push_back(col); slot_size.push_back(2); alpha.push_back(l.real()); beta.push_back(l.imag());
            col += 2;
        }
    }
    if (col != n) { msg = "eigenvector count mismatch"; return false; }
    std::vector<double> A = Q;
    Qinv.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) Qinv[(size_t)i * n + i] = 1.0;
    if (!dense_solve(A, n, Qinv, n)) { msg = "eigenvector matrix singular"; return false; }
    // check Q B Q^-1 = Ax
    double err = 0.0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double s = 0.0;
            for (size_t t = 0; t < slot_start.size(); ++t) {
                const int c0 = slot_start[t];
                if (slot_size[t] == 1) {
                    s += Q[(size_t)i * n + c0] * alpha[t] * Qinv[(size_t)c0 * n + j];
                } else {
                    const double a = alpha[t], b = beta[t];
                    const double q0 = Q[(size_t)i * n + c0], q1 = Q[(size_t)i * n + c0 + 1];
                    const double r0 = Qinv[(size_t)c0 * n + j], r1 = Qinv[(size_t)(c0 + 1) * n + j];
                    s += q0 * (a * r0 + b * r1) + q1 * (-b * r0 + a * r1);
                }
            }
            err = std::max(err, std::fabs(s - Ax[(size_t)i * n + j]));
        }
    if (!(err <= 1e-10 * scale)) { msg = "x-factor block diagonalisation check failed: " + std::to_string(err / scale); return false; }
    { char buf[32]; snprintf(buf, sizeof buf, "%.2e", err / scale); msg = buf; }
    return true;
}

}  // namespace smpm
