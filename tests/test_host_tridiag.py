"""The host tridiagonal LU with partial pivoting behind the coarse division
(one deflation vector per interface, Sec. 3.3: C = Z^T S Z is tridiagonal)
against numpy's dense inverse, on random matrices that force row
interchanges, on diagonally dominant ones (no interchange), at d = 1, 2, 3
and larger, and a singular matrix.  The library's C++ source is compiled
with a small driver (tests/native) on the host; no GPU is used."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    cuda_inc = None
    for cand in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        if cand and os.path.exists(os.path.join(cand, "include", "cuda_runtime.h")):
            cuda_inc = os.path.join(cand, "include")
            break
    if cuda_inc is None:
        pytest.skip("CUDA headers not found")
    exe = tmp_path_factory.mktemp("tri") / "tridiag_driver"
    csrc = os.path.join(ROOT, "paper_1512_01756_gb300", "csrc")
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", csrc, "-I", cuda_inc, "-o", str(exe),
                    os.path.join(ROOT, "tests", "native", "tridiag_driver.cpp"), os.path.join(csrc, "host_ops.cpp")],
                   check=True)
    return str(exe)


def _run(driver, lo, di, up):
    d = len(di)
    text = "%d\n" % d + " ".join("%.17g" % v for v in list(lo) + list(di) + list(up)) + "\n"
    out = subprocess.run([driver], input=text, capture_output=True, text=True, check=True).stdout.split()
    if out[0] == "singular":
        return None, None
    return int(out[1]), np.array([float(v) for v in out[2:]]).reshape(d, d)


def _dense(lo, di, up):
    d = len(di)
    T = np.diag(np.asarray(di, dtype=float))
    if d > 1:
        T += np.diag(lo, -1) + np.diag(up, 1)
    return T


@pytest.mark.parametrize("d", [1, 2, 3, 7, 64, 255])
@pytest.mark.parametrize("kind", ["pivoting", "dominant"])
def test_tridiagonal_inverse_matches_dense(driver, d, kind):
    for seed in range(1000 + d, 1100 + d):          # a draw of moderate condition (< 1e7)
        rng = np.random.default_rng(seed)
        lo, up = rng.standard_normal(d - 1), rng.standard_normal(d - 1)
        di = rng.standard_normal(d)
        if kind == "pivoting":
            lo *= 1.5                  # many subdiagonal entries above the diagonal: interchanges
        else:
            di = 4.0 + np.abs(di)
        if np.linalg.cond(_dense(lo, di, up)) < 1e7:
            break
    swaps, K = _run(driver, lo, di, up)
    T = _dense(lo, di, up)
    ref = np.linalg.inv(T)
    cond = np.linalg.cond(T)
    assert np.abs(K - ref).max() <= 1e-13 * cond * np.abs(ref).max()
    assert np.abs(T @ K - np.eye(d)).max() <= 1e-13 * cond
    if kind == "dominant":
        assert swaps == 0
    elif d >= 7:
        assert swaps > 0


def test_singular_tridiagonal_is_reported(driver):
    # the shape of the coarse matrix for k^2 = 0: rows summing to zero, null vector 1
    lo, di, up = [-1.0, -1.0, -1.0], [1.0, 2.0, 2.0, 1.0], [-1.0, -1.0, -1.0]
    assert np.linalg.matrix_rank(_dense(lo, di, up)) < 4
    swaps, K = _run(driver, lo, di, up)
    assert K is None
