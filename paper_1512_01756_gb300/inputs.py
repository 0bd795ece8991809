"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no arithmetic of the solver: it only evaluates closed-form
right-hand sides at caller-supplied node coordinates and draws seeded random
numbers.  Both the CUDA path (through its node coordinates) and the CPU oracle
(through its own) call it, so each side gets the same input arrays.

Recipes
-------
* ``manufactured_cos``: f for u = cos(pi x / l_x) cos(pi z / l_z) scaled to the
  domain (the 4 x 1 manufactured case: u = cos(pi x/4) cos(pi z)), g = 0.
* ``cos_modes``: f = sum_m c_m cos(a_m pi x / l_x) cos(b_m pi z / l_z) with
  c_m ~ N(0, 1) and distinct (a_m, b_m) drawn from {0..a_max} x {0..b_max}
  without the (0, 0) mode, so the continuous mean is zero and g = 0 is
  compatible.  Returns the modes too, so a test can form the exact solution.
* ``uniform``: the paper's random right-hand side, U[0, 1] per node.
* ``seed_for``: the seed policy, 20151205 + workload index.
"""
import numpy as np

SEED_BASE = 20151205


def seed_for(index):
    return SEED_BASE + int(index)


def rng(seed):
    return np.random.Generator(np.random.PCG64(int(seed)))


def manufactured_cos(x, z, lx, lz):
    ax, bz = np.pi / lx, np.pi / lz
    u = np.cos(ax * x) * np.cos(bz * z)
    return -(ax * ax + bz * bz) * u, u


def cos_modes_spec(seed, n_modes=32, a_max=31, b_max=3):
    """Draw (c_m, a_m, b_m) for the cos-cos sum."""
    r = rng(seed)
    pairs = [(a, b) for a in range(a_max + 1) for b in range(b_max + 1) if (a, b) != (0, 0)]
    if n_modes > len(pairs):
        raise ValueError("not enough distinct modes")
    pick = r.choice(len(pairs), size=n_modes, replace=False)
    ab = np.array([pairs[i] for i in pick], dtype=np.int64)
    c = r.standard_normal(n_modes)
    return c, ab[:, 0], ab[:, 1]


def cos_modes(x, z, lx, lz, spec):
    """Evaluate f and the analytic solution u of lap u = f, n.grad u = 0 at (x, z)."""
    c, a, b = spec
    f = np.zeros_like(np.asarray(x, dtype=np.float64))
    u = np.zeros_like(f)
    for cm, am, bm in zip(c, a, b):
        kx, kz = am * np.pi / lx, bm * np.pi / lz
        phi = np.cos(kx * x) * np.cos(kz * z)
        f += cm * phi
        u += cm * phi / (-(kx * kx + kz * kz))
    return f, u


def uniform(shape, seed):
    return rng(seed).uniform(0.0, 1.0, size=shape)
