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

from .smpm import Grid, direct_solve
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
