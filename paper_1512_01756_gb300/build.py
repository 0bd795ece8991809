"""Build libsmpm.so in-tree: nvcc for sm_103a, one object per translation unit
compiled in parallel, linked against cuSOLVER (used by the operator setup only).

    python -m paper_1512_01756_gb300.build          # incremental
    python -m paper_1512_01756_gb300.build --force  # rebuild everything
"""
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OBJ = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libsmpm.so")
INCLUDE = os.path.join(ROOT, "include")

SOURCES = ["kernels.cu", "api.cu", "host_ops.cpp", "noalloc.cu", "server.cu", "ozaki.cu"]
HEADERS = ["kernels.h", "smpm_internal.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _newest(paths):
    return max(os.path.getmtime(p) for p in paths)


def build(force=False, verbose=False):
    """Compile libsmpm.so if any source is newer than it.  Returns its path."""
    os.makedirs(OBJ, exist_ok=True)
    nvcc = _nvcc()
    deps = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(INCLUDE, "smpm.h")]
    dep_time = _newest(deps)
    procs, objs = [], []
    for src in SOURCES:
        sp = os.path.join(CSRC, src)
        op = os.path.join(OBJ, src + ".o")
        objs.append(op)
        if not force and os.path.exists(op) and os.path.getmtime(op) >= max(os.path.getmtime(sp), dep_time):
            continue
        cmd = [nvcc] + NVCC_FLAGS + ["-c", sp, "-o", op]
        if src.endswith(".cpp"):
            cmd = [nvcc, "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-x", "c++", "-c", sp, "-o", op]
        if verbose:
            print(" ".join(cmd), flush=True)
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append((src, out.decode(errors="replace")))
        elif verbose and out:
            print(out.decode(errors="replace"))
    if failed:
        msg = "\n".join(f"--- {s} ---\n{o}" for s, o in failed)
        raise RuntimeError("libsmpm build failed:\n" + msg)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < _newest(objs):
        cmd = [nvcc] + ARCH + ["-shared", "-o", LIB] + objs + ["-lcusolver", "-lcublas", "-lcudart"]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
        if r.returncode != 0:
            raise RuntimeError("libsmpm link failed:\n" + r.stdout.decode(errors="replace"))
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
