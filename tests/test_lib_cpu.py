"""CPU-side checks of the C-ABI library (no GPU needed): it builds, loads, and
exports every entry point include/smpm.h declares; the binding's struct
layout matches the header."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z_0-9 \*]*?\b(smpm_[a-z0-9_]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1512_01756_gb300 import smpm
    return smpm.load()


def test_exports_every_declared_symbol(lib):
    names = _declared_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name
    from paper_1512_01756_gb300 import smpm
    assert sorted(smpm.EXPORTS) == names


def test_struct_layout_matches_header(tmp_path):
    """The ctypes mirrors of smpm_grid and smpm_stats have the size and field
    offsets the C compiler gives the structs of include/smpm.h."""
    import shutil
    import subprocess
    from paper_1512_01756_gb300 import smpm
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "smpm.h"', "int main(void) {"]
    for cname, cls in (("smpm_grid", smpm.Grid), ("smpm_stats", smpm.Stats)):
        lines.append(f'printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(root, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, cls in (("smpm_grid", smpm.Grid), ("smpm_stats", smpm.Stats)):
        assert got[(cname, "sizeof")] == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)


def test_last_error_without_gpu_call(lib):
    assert lib.smpm_last_error() in (b"",)


def test_grid_coords_match_oracle(lib):
    """smpm_grid_coords is host logic: it needs no GPU and must give the oracle's
    node positions (LGL nodes mapped to each element, Sec. 2.1)."""
    import numpy as np
    from paper_1512_01756_gb300 import smpm
    from oracle.smpm import Grid
    x, z = smpm.grid_coords(smpm.make_grid(5, 3, 6, 2.5, 1.0, z_ratio=1.2))
    X, Z = Grid(5, 3, 6, 2.5, 1.0, z_ratio=1.2).coords()
    assert np.abs(x - X).max() < 1e-14 and np.abs(z - Z).max() < 1e-14
    with pytest.raises(smpm.SmpmError):
        smpm.grid_coords(smpm.make_grid(1, 1, 6, 2.5, 1.0))


def test_request_footprint_is_host_arithmetic(lib):
    """smpm_request_footprint needs no GPU: it grows with the operators and
    the right-hand sides of a batch and with the grid, and rejects bad
    arguments with SMPM_EINVAL."""
    from paper_1512_01756_gb300 import smpm
    small = smpm.make_grid(64, 2, 6, 32.0, 1.0)
    big = smpm.make_grid(1024, 16, 16, 64.0, 1.0)
    f11 = smpm.request_footprint(small, 1, 1)
    assert f11 > 0
    assert smpm.request_footprint(small, 4, 1) > f11
    assert smpm.request_footprint(small, 1, 4) > f11
    assert smpm.request_footprint(big, 1, 1) > 100 * (f11 - (64 << 20))
    with pytest.raises(smpm.SmpmError) as e:
        smpm.request_footprint(small, 0, 1)
    assert e.value.code == smpm.SMPM_EINVAL


def test_residual_history_rejects_a_null_handle(lib):
    import ctypes
    from paper_1512_01756_gb300 import smpm
    cnt = ctypes.c_int(-1)
    rc = lib.smpm_residual_history(None, 0, 0, 0, None, ctypes.byref(cnt))
    assert rc == smpm.SMPM_EINVAL
    assert b"null" in lib.smpm_last_error()
