"""ctypes binding of libsmpm.so (include/smpm.h): argument marshalling only.

Every step of the solve runs in the library's CUDA kernels; this module only
converts Python arguments (torch tensors on the GPU, or numpy arrays / host
tensors) into the pointers and sizes of the C ABI.  There is no fallback: if
the library cannot be loaded, ``load()`` raises.
"""
import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libsmpm.so")

SMPM_OK, SMPM_EINVAL, SMPM_ENOMEM, SMPM_ENOCONV, SMPM_EBREAKDOWN, SMPM_ECUDA, SMPM_EBUSY, SMPM_ETIMEOUT = \
    0, -1, -2, -3, -4, -5, -6, -7

# every entry point include/smpm.h declares
EXPORTS = ["smpm_setup", "smpm_solve", "smpm_solve_batch", "smpm_solve_guess", "smpm_setup_multi", "smpm_solve_multi",
           "smpm_setup_3d", "smpm_solve_3d", "smpm_solve_3d_physical",
           "smpm_sizes", "smpm_node_coords", "smpm_grid_coords", "smpm_null_vectors", "smpm_set_stream", "smpm_device_bytes", "smpm_release", "smpm_probe_fp64",
           "smpm_profile", "smpm_profile_read", "smpm_profile_split", "smpm_kernel_launches", "smpm_apply", "smpm_last_residuals", "smpm_apply_deflation_noalloc",
           "smpm_server_create", "smpm_submit", "smpm_poll", "smpm_server_destroy", "smpm_request_footprint",
           "smpm_residual_history", "smpm_last_error"]


class Grid(ctypes.Structure):
    _fields_ = [("mx", ctypes.c_int), ("mz", ctypes.c_int), ("order", ctypes.c_int),
                ("lx", ctypes.c_double), ("lz", ctypes.c_double), ("z_ratio", ctypes.c_double),
                ("tau_scale", ctypes.c_double), ("deflation_groups", ctypes.c_int),
                ("restart", ctypes.c_int), ("max_iter", ctypes.c_int), ("precision", ctypes.c_int),
                ("krylov", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("restarts", ctypes.c_int), ("status", ctypes.c_int),
                ("rel_resid_true", ctypes.c_double), ("setup_ms", ctypes.c_double),
                ("solve_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class SmpmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"smpm error {code}: {msg}")
        self.code = code


_lib = None


def load():
    """Load libsmpm.so from the package directory (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} not built: run __graft_entry__.build() (no CPU fallback exists)")
    lib = ctypes.CDLL(LIB_PATH)
    H = ctypes.c_void_p
    P = ctypes.c_void_p
    lib.smpm_setup.argtypes = [ctypes.POINTER(Grid), ctypes.c_double, P, ctypes.POINTER(H)]
    lib.smpm_setup_multi.argtypes = [ctypes.POINTER(Grid), ctypes.c_int, P, P, ctypes.POINTER(H)]
    lib.smpm_solve.argtypes = [H, P, P, ctypes.c_double, P, ctypes.POINTER(Stats)]
    lib.smpm_solve_batch.argtypes = [H, ctypes.c_int, P, P, ctypes.c_double, P, ctypes.POINTER(Stats)]
    lib.smpm_solve_guess.argtypes = [H, ctypes.c_int, P, P, P, ctypes.c_double, P, ctypes.POINTER(Stats)]
    lib.smpm_solve_multi.argtypes = [H, ctypes.c_int, P, P, P, ctypes.c_double, P, ctypes.POINTER(Stats)]
    lib.smpm_setup_3d.argtypes = [ctypes.POINTER(Grid), ctypes.c_int, ctypes.c_double, P, ctypes.POINTER(H)]
    lib.smpm_solve_3d.argtypes = [H, P, P, ctypes.c_double, P, ctypes.POINTER(Stats)]
    lib.smpm_solve_3d_physical.argtypes = [H, P, P, ctypes.c_double, P, ctypes.POINTER(Stats)]
    lib.smpm_sizes.argtypes = [H, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong),
                               ctypes.POINTER(ctypes.c_longlong)]
    lib.smpm_node_coords.argtypes = [H, P, P]
    lib.smpm_grid_coords.argtypes = [ctypes.POINTER(Grid), P, P]
    lib.smpm_null_vectors.argtypes = [H, P, P]
    lib.smpm_set_stream.argtypes = [H, P]
    lib.smpm_device_bytes.argtypes = [H]
    lib.smpm_device_bytes.restype = ctypes.c_longlong
    lib.smpm_release.argtypes = [H]
    lib.smpm_release.restype = None
    lib.smpm_probe_fp64.argtypes = [P, ctypes.POINTER(ctypes.c_double)]
    lib.smpm_last_error.restype = ctypes.c_char_p
    lib.smpm_profile.argtypes = [H, ctypes.c_int]
    lib.smpm_profile_read.argtypes = [H, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_double), ctypes.c_int]
    lib.smpm_profile_split.argtypes = [H, ctypes.c_int, ctypes.POINTER(ctypes.c_longlong),
                                       ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), ctypes.c_int]
    lib.smpm_apply.argtypes = [H, ctypes.c_int, ctypes.c_int, P, P]
    lib.smpm_last_residuals.argtypes = [H, ctypes.c_int, P]
    lib.smpm_apply_deflation_noalloc.argtypes = [H, ctypes.c_int, P, P]
    lib.smpm_server_create.argtypes = [ctypes.c_int, ctypes.c_longlong, ctypes.c_int, ctypes.POINTER(H)]
    lib.smpm_submit.argtypes = [H, ctypes.POINTER(Grid), ctypes.c_double, P, P, ctypes.c_double, P,
                                ctypes.POINTER(ctypes.c_ulonglong)]
    lib.smpm_poll.argtypes = [H, ctypes.c_ulonglong, ctypes.POINTER(Stats)]
    lib.smpm_server_destroy.argtypes = [H]
    lib.smpm_residual_history.argtypes = [H, ctypes.c_int, ctypes.c_int, ctypes.c_int, P, ctypes.POINTER(ctypes.c_int)]
    lib.smpm_request_footprint.argtypes = [ctypes.POINTER(Grid), ctypes.c_int, ctypes.c_int,
                                           ctypes.POINTER(ctypes.c_longlong)]
    lib.smpm_kernel_launches.argtypes = []
    lib.smpm_kernel_launches.restype = ctypes.c_longlong
    for name in EXPORTS:
        if not hasattr(lib, name):
            raise RuntimeError(f"libsmpm.so does not export {name}")
    for name in EXPORTS:
        if name not in ("smpm_device_bytes", "smpm_release", "smpm_last_error", "smpm_kernel_launches"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(code):
    if code != SMPM_OK and code != SMPM_ENOCONV:
        raise SmpmError(code, load().smpm_last_error().decode())
    return code


def _ptr(x):
    """Pointer of a torch tensor (any device) or a numpy array; None -> NULL."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        if str(x.dtype) != "torch.float64" and str(x.dtype) != "torch.int32":
            raise ValueError("tensor must be float64")
        return ctypes.c_void_p(x.data_ptr())
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data_as(ctypes.c_void_p)
    raise TypeError(f"unsupported buffer type {type(x)}")


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def make_grid(mx, mz, order, lx, lz, z_ratio=1.0, tau_scale=-0.1, deflation_groups=0, restart=64,
              max_iter=2000, precision=0, krylov=0):
    return Grid(mx, mz, order, lx, lz, z_ratio, tau_scale, deflation_groups, restart, max_iter, precision, krylov)


class Solver:
    """One smpm handle (operators for one or several k^2 values)."""

    def __init__(self, grid: Grid, k2=0.0, stream=None):
        lib = load()
        self._h = ctypes.c_void_p()
        self.grid = grid
        if np.ndim(k2) == 0:
            self.k2 = np.array([float(k2)])
            _check(lib.smpm_setup(ctypes.byref(grid), float(k2), _stream_ptr(stream), ctypes.byref(self._h)))
        else:
            self.k2 = np.ascontiguousarray(k2, dtype=np.float64)
            _check(lib.smpm_setup_multi(ctypes.byref(grid), len(self.k2), self.k2.ctypes.data_as(ctypes.c_void_p),
                                        _stream_ptr(stream), ctypes.byref(self._h)))
        r, nb, k = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong()
        _check(lib.smpm_sizes(self._h, ctypes.byref(r), ctypes.byref(nb), ctypes.byref(k)))
        self.r, self.nb, self.k = r.value, nb.value, k.value

    def coords(self):
        x = np.empty(self.r)
        z = np.empty(self.r)
        _check(load().smpm_node_coords(self._h, _ptr(x), _ptr(z)))
        return x, z

    def device_bytes(self):
        return load().smpm_device_bytes(self._h)

    def set_stream(self, stream):
        _check(load().smpm_set_stream(self._h, _stream_ptr(stream)))

    def null_vectors(self):
        """(u_L, u_S) of the k^2 = 0 operator set, as numpy arrays."""
        uL = np.empty(self.r)
        uS = np.empty(self.k)
        _check(load().smpm_null_vectors(self._h, _ptr(uL), _ptr(uS)))
        return uL, uS

    def solve(self, f, u, g=None, tol=1e-10, u0=None):
        """f, u: one r-vector or [nrhs, r]; g: [nrhs, nb] or None; u0: an initial
        guess shaped like u, or None.  Returns Stats."""
        st = Stats()
        nrhs = 1 if len(f.shape) == 1 else int(f.shape[0])
        if u0 is not None:
            code = load().smpm_solve_guess(self._h, nrhs, _ptr(f), _ptr(g), _ptr(u0), float(tol), _ptr(u),
                                           ctypes.byref(st))
        elif nrhs == 1:
            code = load().smpm_solve(self._h, _ptr(f), _ptr(g), float(tol), _ptr(u), ctypes.byref(st))
        else:
            code = load().smpm_solve_batch(self._h, nrhs, _ptr(f), _ptr(g), float(tol), _ptr(u), ctypes.byref(st))
        _check(code)
        return st

    def solve_multi(self, op_of_rhs, f, u, g=None, tol=1e-10):
        ops = np.ascontiguousarray(op_of_rhs, dtype=np.int32)
        st = Stats()
        _check(load().smpm_solve_multi(self._h, len(ops), ops.ctypes.data_as(ctypes.c_void_p), _ptr(f), _ptr(g),
                                       float(tol), _ptr(u), ctypes.byref(st)))
        return st

    def residual_history(self, rhs=0, kind=0):
        """Residual history of right-hand side rhs of the last solve: kind 0 the
        Givens estimate after every Arnoldi step, kind 1 the true residual at
        every restart-cycle start (relative to ||b_S||)."""
        cnt = ctypes.c_int()
        _check(load().smpm_residual_history(self._h, int(rhs), int(kind), 0, None, ctypes.byref(cnt)))
        out = np.empty(cnt.value)
        if cnt.value:
            _check(load().smpm_residual_history(self._h, int(rhs), int(kind), cnt.value, _ptr(out), ctypes.byref(cnt)))
        return out

    def last_residuals(self, n):
        out = np.empty(n)
        _check(load().smpm_last_residuals(self._h, int(n), _ptr(out)))
        return out

    APPLY = {"S": 0, "Minv": 1, "P": 2, "bS": 3, "Ainv": 4}

    def apply(self, kind, x, y):
        """y = op(x) for op in APPLY (x, y: [nrhs, len] or one vector)."""
        nrhs = 1 if len(x.shape) == 1 else int(x.shape[0])
        _check(load().smpm_apply(self._h, self.APPLY[kind], nrhs, _ptr(x), _ptr(y)))

    def apply_deflation_noalloc(self, x, y):
        """y = P x through the allocation-free entry point (device buffers only)."""
        nrhs = 1 if len(x.shape) == 1 else int(x.shape[0])
        _check(load().smpm_apply_deflation_noalloc(self._h, nrhs, _ptr(x), _ptr(y)))

    def profile(self, enable=True):
        _check(load().smpm_profile(self._h, 1 if enable else 0))

    def profile_read(self, reset=True):
        n, fl, ms = ctypes.c_longlong(), ctypes.c_double(), ctypes.c_double()
        _check(load().smpm_profile_read(self._h, ctypes.byref(n), ctypes.byref(fl), ctypes.byref(ms), int(reset)))
        return {"launches": n.value, "flops": fl.value, "ms": ms.value}

    def close(self):
        if self._h:
            load().smpm_release(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Solver3D(Solver):
    """Handle for the y-periodic 3-D problem in Fourier space (my/2+1 modes)."""

    def __init__(self, grid: Grid, my, ly, stream=None):
        lib = load()
        self._h = ctypes.c_void_p()
        self.grid = grid
        self.my, self.ly = int(my), float(ly)
        self.n_modes = self.my // 2 + 1
        _check(lib.smpm_setup_3d(ctypes.byref(grid), self.my, self.ly, _stream_ptr(stream), ctypes.byref(self._h)))
        r, nb, k = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong()
        _check(lib.smpm_sizes(self._h, ctypes.byref(r), ctypes.byref(nb), ctypes.byref(k)))
        self.r, self.nb, self.k = r.value, nb.value, k.value

    def solve_3d(self, fhat, uhat, ghat=None, tol=1e-10):
        """fhat, uhat: [n_modes, 2, r] float64 (real and imaginary parts)."""
        st = Stats()
        _check(load().smpm_solve_3d(self._h, _ptr(fhat), _ptr(ghat), float(tol), _ptr(uhat), ctypes.byref(st)))
        return st

    def solve_3d_physical(self, f3, u3, g3=None, tol=1e-10):
        """f3, u3: [my, r] float64 planes (y_t = t ly / my); g3: [my, nb] or None."""
        st = Stats()
        _check(load().smpm_solve_3d_physical(self._h, _ptr(f3), _ptr(g3), float(tol), _ptr(u3), ctypes.byref(st)))
        return st


def request_footprint(grid: Grid, nop=1, nrhs=1):
    """Device bytes the serving runtime's admission charges for a batch of
    nrhs requests with nop distinct k^2 on grid (host arithmetic)."""
    b = ctypes.c_longlong()
    _check(load().smpm_request_footprint(ctypes.byref(grid), int(nop), int(nrhs), ctypes.byref(b)))
    return b.value


def grid_coords(grid: Grid):
    """Node coordinates (x, z) of a grid in node order, without a handle."""
    r = (grid.order + 1) ** 2 * grid.mx * grid.mz
    x = np.empty(r)
    z = np.empty(r)
    _check(load().smpm_grid_coords(ctypes.byref(grid), _ptr(x), _ptr(z)))
    return x, z


class Server:
    """Serving runtime (smpm_server_*): submit solves, poll their tickets.

    The buffers of a submitted request are kept referenced here until its
    ticket has been polled to completion (the library reads f, g and writes u
    asynchronously)."""

    def __init__(self, nworkers=2, device_budget_bytes=0, max_batch=16):
        self._s = ctypes.c_void_p()
        _check(load().smpm_server_create(int(nworkers), int(device_budget_bytes), int(max_batch),
                                         ctypes.byref(self._s)))
        self._keep = {}

    def submit(self, grid: Grid, k2, f, u, g=None, tol=1e-10):
        t = ctypes.c_ulonglong()
        _check(load().smpm_submit(self._s, ctypes.byref(grid), float(k2), _ptr(f), _ptr(g), float(tol), _ptr(u),
                                  ctypes.byref(t)))
        self._keep[t.value] = (grid, f, g, u)
        return t.value

    def poll(self, ticket):
        """None while the request runs; else its Stats (raises on a failed solve)."""
        st = Stats()
        code = load().smpm_poll(self._s, ctypes.c_ulonglong(ticket), ctypes.byref(st))
        if code == SMPM_EBUSY:
            return None
        self._keep.pop(ticket, None)
        _check(code)
        return st

    def close(self):
        if self._s:
            _check(load().smpm_server_destroy(self._s))
            self._s = ctypes.c_void_p()
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def kernel_launches():
    return load().smpm_kernel_launches()


def profile_all(enable=True):
    """Profile the dense-product launches of every handle created from now on
    (the serving workers' included)."""
    _check(load().smpm_profile(None, 1 if enable else 0))


def profile_split(handle=None, reset=True):
    """Dense-product launch totals per kind of one handle (a Solver), or of
    every handle of the process for None: FP64 and FP32 CUDA-core launches,
    the FP64-accurate tensor-core launches with their algorithmic FLOPs
    ("tensor") and executed BF16 tensor FLOPs ("tensor_exec", same time)."""
    if handle is not None and hasattr(handle, "_h"):
        handle = handle._h
    out = {}
    for p, name in ((0, "fp64"), (1, "fp32"), (2, "tensor"), (3, "tensor_exec")):
        n, fl, ms = ctypes.c_longlong(), ctypes.c_double(), ctypes.c_double()
        _check(load().smpm_profile_split(handle, p, ctypes.byref(n), ctypes.byref(fl), ctypes.byref(ms), int(reset)))
        out[name] = {"launches": n.value, "flops": fl.value, "ms": ms.value}
    return out


def probe_fp64(stream=None):
    t = ctypes.c_double()
    _check(load().smpm_probe_fp64(_stream_ptr(stream), ctypes.byref(t)))
    return t.value
