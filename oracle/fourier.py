"""3-D y-periodic extension through Fourier modes (Sec. 5, Eqs. poisson3d,
fourier_poisson, transverse_schur, Alg. 3d).

Test infrastructure only (see ``oracle/__init__.py``).

u(x, y, z) = sum_j u_j(x, z) exp(i k_j y) turns the 3-D Poisson-Neumann problem
into one 2-D problem per wavenumber: (L - k_j^2 I) u_j = f_j.  The oracle takes
the plain route: a real DFT along y (numpy rfft), one independent 2-D solve per
mode for the real and imaginary parts (L is real), and the inverse DFT.

Reading (Sec. 5 prints h_y in the wavenumber): k_j = 2 pi j / l_y for j = 0 .. m_y/2 (the
printed h_y in the wavenumber is read as l_y; the Nyquist mode is kept).  Mode 0
is the singular Poisson-Neumann problem and gets the null-space projection and
the zero-mean gauge; the other modes are regular Helmholtz problems.
"""
import numpy as np

from .smpm import Grid, direct_solve, rhs, gauge
from . import dbj
from .schur import StripSchur


def wavenumbers(my, ly):
    return 2.0 * np.pi * np.arange(my // 2 + 1) / ly


def forward(f3):
    """f3[r, m_y] -> complex modes [r, m_y/2+1] with u = sum_j u_j e^{i k_j y}."""
    my = f3.shape[1]
    return np.fft.rfft(f3, axis=1) / my


def inverse(fh, my):
    return np.fft.irfft(fh * my, n=my, axis=1)


def solve_modes(g: Grid, fh, ly, method="direct", tol=1e-13, schurs=None):
    """Solve every mode's 2-D Helmholtz problem for the real and imaginary parts.

    fh: complex [r, n_modes].  Returns complex [r, n_modes] mode solutions."""
    nm = fh.shape[1]
    my = 2 * (nm - 1)
    ks = wavenumbers(my, ly)
    out = np.zeros_like(fh)
    for j in range(nm):
        k2 = float(ks[j] ** 2)
        parts = []
        for comp in (fh[:, j].real, fh[:, j].imag):
            if not np.any(comp):
                parts.append(np.zeros(g.r))
                continue
            if method == "direct":
                u, _ = direct_solve(g, comp, None, k2)
            else:
                sch = schurs[j] if schurs is not None else None
                u, _ = dbj.solve(g, comp, None, k2, method=method, tol=tol, schur=sch)
            parts.append(u)
        out[:, j] = parts[0] + 1j * parts[1]
    return out


def solve_3d(g: Grid, f3, ly, method="direct", tol=1e-13):
    """Alg. 3d with independent per-mode solves: rfft in y, 2-D Helmholtz per
    mode, irfft.  f3 is real [r, m_y] sampled at y_l = l l_y / m_y."""
    my = f3.shape[1]
    uh = solve_modes(g, forward(f3), ly, method=method, tol=tol)
    return inverse(uh, my)


def build_schurs(g: Grid, my, ly):
    return [StripSchur(g, float(k * k)) for k in wavenumbers(my, ly)]


def solve_3d_concatenated(g: Grid, f3, ly, tol=1e-13, maxiter=2000):
    """Alg. 3d as printed: every mode's deflated, preconditioned Schur system
    (Sec. 5, Eq. 3d_deflated_schur: P(k_j) S(k_j) M(k_j)^-1 applied to the
    mode's real and imaginary parts) stacked into one vector, and one GMRES
    on the block-diagonal operator (line 7), so every inner product and norm
    is the sum over the modes and the stopping test is the one of the stacked
    residual.  Before it, each part's right-hand side is prepared as in
    Alg. seq steps 1-3 (mode 0 with its null-space projections, Sec. 2.4);
    after it, each part is completed as in steps 5-9.  Returns (u3, info)
    with the GMRES iteration count and the stacked true Schur residual
    ||[S_j x_j - b_j]|| / ||[b_j]||.  The concatenated stopping test is the
    reading of the paper's single GMRES; where the paper is silent on it, the
    stacked residual is the natural norm of the stacked system."""
    my = f3.shape[1]
    fh = forward(f3)
    ks = wavenumbers(my, ly)
    parts = []                      # (mode, component, pieces of Alg. seq for that 2-D problem)
    for j, kj in enumerate(ks):
        k2 = float(kj * kj)
        sch = None
        for comp, vals in ((0, fh[:, j].real), (1, fh[:, j].imag)):
            if not np.any(vals):
                continue
            if sch is None:
                sch = StripSchur(g, k2)
            b = rhs(g, vals)
            uS = None
            if k2 == 0.0:
                uL, uS = sch.null_vectors()
                b = b - uL * np.dot(uL, b)                   # step 1
            bS = sch.B @ sch.Ainv(b)                          # step 2
            if k2 == 0.0:
                bS = bS - uS * np.dot(uS, bS)                 # step 3
            S = dbj.RangeProjected(sch.S, uS) if k2 == 0.0 else sch.S
            M = dbj.BlockJacobi(g, sch.S, singular=(k2 == 0.0))
            Df = dbj.Deflation(g, S, uS)
            parts.append(dict(j=j, comp=comp, k2=k2, sch=sch, b=b, bS=bS, S=S, M=M, Df=Df))
    sizes = [len(p["bS"]) for p in parts]
    offs = np.concatenate([[0], np.cumsum(sizes)])

    def apply(v):                   # line 7: the block-diagonal operator on the stacked vector
        out = np.empty_like(v)
        for i, p in enumerate(parts):
            x = v[offs[i]:offs[i + 1]]
            out[offs[i]:offs[i + 1]] = p["Df"].P(p["S"] @ p["M"].solve(x))
        return out

    rhs_stack = np.concatenate([p["Df"].P(p["bS"]) for p in parts]) if parts else np.zeros(0)
    y, it, hist = dbj.householder_gmres(apply, rhs_stack, tol, maxiter)
    uh = np.zeros((g.r, len(ks)), dtype=complex)
    r2, b2 = 0.0, 0.0
    for i, p in enumerate(parts):
        x1 = p["Df"].Q(p["M"].solve(y[offs[i]:offs[i + 1]]))    # step 5
        xS = x1 + p["Df"].coarse_part(p["bS"])                   # steps 6-8
        u = p["sch"].Ainv(p["b"] - p["sch"].E @ xS)              # step 9
        if p["k2"] == 0.0:
            u = gauge(g, u)
        r2 += float(np.sum((p["S"] @ xS - p["bS"]) ** 2))
        b2 += float(np.sum(p["bS"] ** 2))
        uh[:, p["j"]] += u if p["comp"] == 0 else 1j * u
    info = dict(iterations=it, history=hist, stacked_schur_residual=np.sqrt(r2 / b2) if b2 > 0 else 0.0)
    return inverse(uh, my), info
