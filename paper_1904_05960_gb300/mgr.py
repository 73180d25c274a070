"""Python binding of the GB300 MGR library (include/mgr_gb300.h).

Argument marshalling only: every step of setup, preconditioner application and
the Krylov solve runs in the CUDA kernels of ``libmgr_gb300.so``.  PyTorch
provides the device buffers and the stream handle.  There is no fallback: if
the compiled library is missing, loading it raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

MGR_MAX_LEVELS = 8
MGR_SUCCESS, MGR_NOT_CONVERGED = 0, 1
MGR_FRELAX_AMG_VCYCLE, MGR_FRELAX_JACOBI = 0, 1
MGR_FP64, MGR_MIXED = 0, 1
MGR_ORTHO_CGS2, MGR_ORTHO_MGS, MGR_ORTHO_AUTO = 0, 1, 2

# hierarchy inspection kinds (mgr_get_csr)
Q_MGR_A, Q_MGR_W, Q_MGR_COR, Q_MGR_CORKEPT, Q_MGR_S, Q_MGR_WR, Q_MGR_BD, Q_MGR_ILU = 0, 1, 2, 3, 4, 5, 6, 7
Q_AMG_A, Q_AMG_S, Q_AMG_P, Q_AMG_R = 10, 11, 12, 13

EXPORTED = ["mgr_options_default", "fgmres_options_default", "mgr_setup", "mgr_apply",
            "fgmres_solve", "mgr_destroy", "mgr_error_string", "mgr_get_csr",
            "mgr_amg_levels", "mgr_get_cf", "mgr_vcycle", "mgr_splitmix64_device",
            "mgr_launch_count", "mgr_trim_memory", "mgr_solve_host", "mgr_vcycle_noalloc", "mgr_setup_batched",
            "fgmres_solve_batched", "mgr_batch_info", "mgr_batch_handle", "mgr_destroy_batched",
            "mgr_get_block_colors", "mgr_build_id", "mgr_memory_usage", "mgr_spmv", "mgr_host_launch_count", "mgr_row_patterns",
            "mgr_jacobian_product"]


class MgrMatrix(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("row_ptr", C.c_void_p),
                ("col_idx", C.c_void_p), ("val", C.c_void_p), ("dof_label", C.c_void_p),
                ("dof_node", C.c_void_p), ("dof_comp", C.c_void_p)]


class MgrOptions(C.Structure):
    _fields_ = [("num_levels", C.c_int32),
                ("f_label_mask", C.c_uint32 * MGR_MAX_LEVELS),
                ("frelax", C.c_int32 * MGR_MAX_LEVELS),
                ("frelax_sweeps", C.c_int32 * MGR_MAX_LEVELS),
                ("nmax_drop", C.c_int32 * MGR_MAX_LEVELS),
                ("global_sweeps", C.c_int32 * MGR_MAX_LEVELS),
                ("amg_theta", C.c_double), ("amg_pmax", C.c_int32),
                ("amg_max_coarse", C.c_int32), ("amg_max_levels", C.c_int32),
                ("precision", C.c_int32), ("seed", C.c_uint64),
                ("restrict_jacobi", C.c_int32 * MGR_MAX_LEVELS),
                ("frelax_post", C.c_int32 * MGR_MAX_LEVELS),
                ("dff_block", C.c_int32 * MGR_MAX_LEVELS),
                ("global_smoother", C.c_int32 * MGR_MAX_LEVELS),
                ("agg_levels", C.c_int32 * MGR_MAX_LEVELS),
                ("ilu_solve_sweeps", C.c_int32),
                ("diag_bf16", C.c_int32), ("values_f16", C.c_int32)]


class FgmresOptions(C.Structure):
    _fields_ = [("restart", C.c_int32), ("max_iter", C.c_int32), ("rtol", C.c_double),
                ("ortho", C.c_int32)]


class FgmresInfo(C.Structure):
    _fields_ = [("iters", C.c_int32), ("restarts", C.c_int32), ("converged", C.c_int32),
                ("rel_res_true", C.c_double), ("setup_s", C.c_double), ("solve_s", C.c_double),
                ("res_hist", C.c_void_p), ("res_hist_cap", C.c_int32)]


_lock = threading.Lock()
_lib = None


def lib_path():
    return _build.LIB


def lib():
    """Load libmgr_gb300.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            path = lib_path()
            if not os.path.exists(path):
                raise RuntimeError(
                    f"{path} is missing: build the CUDA library first "
                    "(python -m paper_1904_05960_gb300.build); there is no CPU fallback")
            L = C.CDLL(path)
            P, I64 = C.c_void_p, C.c_int64
            L.mgr_options_default.argtypes = [C.POINTER(MgrOptions), C.c_int]
            L.mgr_options_default.restype = None
            L.fgmres_options_default.argtypes = [C.POINTER(FgmresOptions)]
            L.fgmres_options_default.restype = None
            L.mgr_setup.argtypes = [C.POINTER(MgrMatrix), C.POINTER(MgrOptions), P, C.POINTER(P)]
            L.mgr_apply.argtypes = [P, P, P, P]
            L.fgmres_solve.argtypes = [P, C.POINTER(MgrMatrix), P, P, C.POINTER(FgmresOptions),
                                       C.POINTER(FgmresInfo), P]
            L.mgr_destroy.argtypes = [P]
            L.mgr_error_string.argtypes = [C.c_int]
            L.mgr_error_string.restype = C.c_char_p
            L.mgr_get_csr.argtypes = [P, C.c_int, C.c_int, C.c_int, P, P, P, P]
            L.mgr_amg_levels.argtypes = [P, C.c_int]
            L.mgr_get_cf.argtypes = [P, C.c_int, C.c_int, P]
            L.mgr_row_patterns.argtypes = [P, C.c_int, C.c_int]
            L.mgr_get_cf.restype = I64
            L.mgr_vcycle.argtypes = [P, C.c_int, P, P, P]
            L.mgr_splitmix64_device.argtypes = [P, P, I64, P]
            L.mgr_spmv.argtypes = [C.POINTER(MgrMatrix), P, P, P]
            L.mgr_jacobian_product.argtypes = [P, C.POINTER(MgrMatrix), P, P, C.c_int, P]
            L.mgr_vcycle_noalloc.argtypes = [P, C.c_int, P, P, P]
            L.mgr_setup_batched.argtypes = [C.c_int, C.POINTER(MgrMatrix), C.POINTER(MgrOptions),
                                            C.c_int, P, C.POINTER(P)]
            L.fgmres_solve_batched.argtypes = [P, C.POINTER(MgrMatrix), C.POINTER(P), C.POINTER(P),
                                               C.POINTER(FgmresOptions), C.POINTER(FgmresInfo), P]
            L.mgr_batch_info.argtypes = [P, C.POINTER(C.c_int), C.POINTER(C.c_double),
                                         C.POINTER(C.c_int), C.POINTER(C.c_double)]
            L.mgr_batch_handle.argtypes = [P, C.c_int, C.POINTER(P)]
            L.mgr_destroy_batched.argtypes = [P]
            L.mgr_get_block_colors.argtypes = [P, C.c_int, P, P]
            L.mgr_get_block_colors.restype = I64
            L.mgr_launch_count.argtypes = []
            L.mgr_launch_count.restype = I64
            L.mgr_host_launch_count.argtypes = []
            L.mgr_host_launch_count.restype = I64
            L.mgr_trim_memory.argtypes = [C.c_size_t]
            L.mgr_build_id.argtypes = []
            L.mgr_build_id.restype = C.c_char_p
            L.mgr_memory_usage.argtypes = [C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)]
            L.mgr_solve_host.argtypes = [C.POINTER(MgrMatrix), P, P, C.POINTER(MgrOptions),
                                         C.POINTER(FgmresOptions), C.POINTER(FgmresInfo), P]
            _lib = L
    return _lib


class MgrError(RuntimeError):
    def __init__(self, code, what):
        msg = lib().mgr_error_string(code).decode()
        super().__init__(f"{what} failed: {msg} ({code})")
        self.code = code


def _check(code, what):
    if code < 0:
        raise MgrError(code, what)
    return code


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


# ---------------------------------------------------------------------------
def mgr_options_default(two_phase=True, **overrides):
    """The paper's configuration (Sec. 5.3 / Sec. 6); keyword overrides take
    lists for the per-level fields."""
    o = MgrOptions()
    lib().mgr_options_default(C.byref(o), 1 if two_phase else 0)
    for k, v in overrides.items():
        if isinstance(v, (list, tuple)):
            arr = getattr(o, k)
            for i, x in enumerate(v):
                arr[i] = x
        else:
            setattr(o, k, v)
    return o


def fgmres_options_default(**overrides):
    o = FgmresOptions()
    lib().fgmres_options_default(C.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


class DeviceMatrix:
    """A synth.Problem (or any CSR with labels) copied into device tensors."""

    def __init__(self, prob, device="cuda"):
        import torch
        self.n = int(prob.n)
        self.nnz = int(prob.row_ptr[-1])
        t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).to(device)
        self.row_ptr = t(prob.row_ptr, np.int64)
        self.col_idx = t(prob.col, np.int32)
        self.val = t(prob.val, np.float64)
        self.dof_label = t(prob.dof_label, np.int32)
        self.dof_node = t(prob.dof_node, np.int32)
        self.dof_comp = t(prob.dof_comp, np.int32) if prob.dof_comp is not None else None
        self._s = MgrMatrix(self.n, self.nnz, self.row_ptr.data_ptr(), self.col_idx.data_ptr(),
                            self.val.data_ptr(), self.dof_label.data_ptr(),
                            self.dof_node.data_ptr(),
                            self.dof_comp.data_ptr() if self.dof_comp is not None else None)

    @property
    def c(self):
        return self._s


class HostMatrix:
    """A problem's CSR and labels in host tensors (pinned by default), for
    mgr_solve_host."""

    def __init__(self, prob, pin=True):
        import torch
        self.n = int(prob.n)
        self.nnz = int(prob.row_ptr[-1])

        def t(a, dt):
            x = torch.from_numpy(np.ascontiguousarray(a, dtype=dt))
            return x.pin_memory() if pin else x
        self.row_ptr = t(prob.row_ptr, np.int64)
        self.col_idx = t(prob.col, np.int32)
        self.val = t(prob.val, np.float64)
        self.dof_label = t(prob.dof_label, np.int32)
        self.dof_node = t(prob.dof_node, np.int32)
        self.dof_comp = t(prob.dof_comp, np.int32) if prob.dof_comp is not None else None
        self._s = MgrMatrix(self.n, self.nnz, self.row_ptr.data_ptr(), self.col_idx.data_ptr(),
                            self.val.data_ptr(), self.dof_label.data_ptr(),
                            self.dof_node.data_ptr(),
                            self.dof_comp.data_ptr() if self.dof_comp is not None else None)

    @property
    def c(self):
        return self._s

    @property
    def nbytes(self):
        ts = [self.row_ptr, self.col_idx, self.val, self.dof_label, self.dof_node]
        if self.dof_comp is not None:
            ts.append(self.dof_comp)
        return sum(x.numel() * x.element_size() for x in ts)


def mgr_solve_host(A: HostMatrix, b, x, opts: MgrOptions, fo: FgmresOptions | None = None,
                   stream=None):
    """Setup + FGMRES + teardown from host buffers (b, x: host FP64 tensors)."""
    info = FgmresInfo()
    st = _check(lib().mgr_solve_host(C.byref(A.c), _ptr(b), _ptr(x), C.byref(opts),
                                     C.byref(fo) if fo is not None else None, C.byref(info),
                                     _stream_ptr(stream)), "mgr_solve_host")
    return dict(status=st, iters=info.iters, restarts=info.restarts,
                converged=bool(info.converged), relres=info.rel_res_true,
                setup_s=info.setup_s, solve_s=info.solve_s)


def mgr_setup(A: DeviceMatrix, opts: MgrOptions, stream=None):
    h = C.c_void_p()
    _check(lib().mgr_setup(C.byref(A.c), C.byref(opts), _stream_ptr(stream), C.byref(h)),
           "mgr_setup")
    return h


def mgr_apply(h, v, z, stream=None):
    """z = M^-1 v (device FP64 tensors)."""
    return _check(lib().mgr_apply(h, _ptr(v), _ptr(z), _stream_ptr(stream)), "mgr_apply")


def fgmres_solve(h, A: DeviceMatrix, b, x, opts: FgmresOptions | None = None, stream=None,
                 hist_cap=0):
    info = FgmresInfo()
    hist = np.zeros(max(hist_cap, 1))
    if hist_cap:
        info.res_hist = hist.ctypes.data
        info.res_hist_cap = hist_cap
    o = opts if opts is not None else fgmres_options_default()
    st = _check(lib().fgmres_solve(h, C.byref(A.c), _ptr(b), _ptr(x), C.byref(o),
                                   C.byref(info), _stream_ptr(stream)), "fgmres_solve")
    return dict(status=st, iters=info.iters, restarts=info.restarts,
                converged=bool(info.converged), relres=info.rel_res_true,
                setup_s=info.setup_s, solve_s=info.solve_s,
                hist=hist[:min(hist_cap, info.iters + 1)] if hist_cap else None)


def mgr_destroy(h):
    if h:
        lib().mgr_destroy(h)


def _matrix_array(As):
    arr = (MgrMatrix * len(As))()
    for i, A in enumerate(As):
        arr[i] = A.c
    return arr


def mgr_setup_batched(As, opts: MgrOptions, workers=0, stream=None):
    """Set up every system of the list As (DeviceMatrix); workers = 0 lets the
    library's autotuner pick the number of concurrent workers."""
    h = C.c_void_p()
    _check(lib().mgr_setup_batched(len(As), _matrix_array(As), C.byref(opts), int(workers),
                                   _stream_ptr(stream), C.byref(h)), "mgr_setup_batched")
    return h


def fgmres_solve_batched(bh, As, bs, xs, opts: FgmresOptions | None = None, stream=None):
    """Solve As[i] xs[i] = bs[i] for all systems; returns (status, [info dicts])."""
    n = len(As)
    infos = (FgmresInfo * n)()
    bp = (C.c_void_p * n)(*[b.data_ptr() for b in bs])
    xp = (C.c_void_p * n)(*[x.data_ptr() for x in xs])
    o = opts if opts is not None else fgmres_options_default()
    st = _check(lib().fgmres_solve_batched(bh, _matrix_array(As), bp, xp, C.byref(o), infos,
                                           _stream_ptr(stream)), "fgmres_solve_batched")
    return st, [dict(iters=i.iters, restarts=i.restarts, converged=bool(i.converged),
                     relres=i.rel_res_true, setup_s=i.setup_s, solve_s=i.solve_s) for i in infos]


def mgr_batch_info(bh):
    w = C.c_int(0)
    s = C.c_double(0.0)
    tw = (C.c_int * 6)()
    t = (C.c_double * 6)()
    _check(lib().mgr_batch_info(bh, C.byref(w), C.byref(s), tw, t), "mgr_batch_info")
    return dict(workers=w.value, setup_s=s.value,
                tune_ms={k: v for k, v in zip(list(tw), list(t)) if k != 0})


def mgr_batch_handle(bh, i):
    h = C.c_void_p()
    _check(lib().mgr_batch_handle(bh, int(i), C.byref(h)), "mgr_batch_handle")
    return h


def mgr_destroy_batched(bh):
    if bh:
        lib().mgr_destroy_batched(bh)


def mgr_get_csr(h, kind, slot=0, lvl=0):
    """(rows, cols, row_ptr, col, val) of a hierarchy matrix (host numpy), or None."""
    dims = np.zeros(3, dtype=np.int64)
    if lib().mgr_get_csr(h, kind, slot, lvl, dims.ctypes.data, None, None, None) != 0:
        return None
    nr, nc, nnz = (int(x) for x in dims)
    rp = np.zeros(nr + 1, dtype=np.int64)
    ci = np.zeros(max(nnz, 1), dtype=np.int32)
    v = np.zeros(max(nnz, 1))
    _check(lib().mgr_get_csr(h, kind, slot, lvl, dims.ctypes.data, rp.ctypes.data,
                             ci.ctypes.data, v.ctypes.data), "mgr_get_csr")
    return nr, nc, rp, ci[:nnz], v[:nnz]


def mgr_get_csr_dims(h, kind, slot=0, lvl=0):
    """(rows, cols, nnz) of a hierarchy matrix, or None."""
    dims = np.zeros(3, dtype=np.int64)
    if lib().mgr_get_csr(h, kind, slot, lvl, dims.ctypes.data, None, None, None) != 0:
        return None
    return tuple(int(x) for x in dims)


def mgr_get_scipy(h, kind, slot=0, lvl=0):
    import scipy.sparse as sp
    r = mgr_get_csr(h, kind, slot, lvl)
    if r is None:
        return None
    nr, nc, rp, ci, v = r
    return sp.csr_matrix((v, ci, rp), shape=(nr, nc))


def mgr_amg_levels(h, slot):
    return int(lib().mgr_amg_levels(h, slot))


def mgr_row_patterns(h, slot, lvl):
    """Shared row patterns of an AMG operator (0: applied as plain CSR)."""
    return _check(lib().mgr_row_patterns(h, slot, lvl), "mgr_row_patterns")


def mgr_get_cf(h, slot, lvl):
    n = lib().mgr_get_cf(h, slot, lvl, None)
    if n < 0:
        return None
    out = np.zeros(n, dtype=np.int8)
    lib().mgr_get_cf(h, slot, lvl, out.ctypes.data)
    return out


def mgr_vcycle(h, slot, b, x, stream=None):
    return _check(lib().mgr_vcycle(h, slot, _ptr(b), _ptr(x), _stream_ptr(stream)), "mgr_vcycle")


def mgr_vcycle_noalloc(h, slot, b, x, stream=None):
    """One V-cycle like mgr_vcycle, with its workspace in the library's fixed
    8 MiB device buffer instead of memory of the handle (for callers that
    cannot allocate device memory where they run)."""
    return _check(lib().mgr_vcycle_noalloc(h, slot, _ptr(b), _ptr(x), _stream_ptr(stream)),
                  "mgr_vcycle_noalloc")


def mgr_spmv(A: DeviceMatrix, x, y, stream=None):
    """y = A x (device FP64 tensors) with FGMRES's Jacobian product."""
    return _check(lib().mgr_spmv(C.byref(A.c), _ptr(x), _ptr(y), _stream_ptr(stream)), "mgr_spmv")


def mgr_jacobian_product(h, A: DeviceMatrix, x, y, refresh=True, stream=None):
    """y = A x as fgmres_solve forms it; True when a sliced copy of A was read.
    refresh=False reuses the last copy (asynchronous; A must be unchanged)."""
    return _check(lib().mgr_jacobian_product(h, C.byref(A.c), _ptr(x), _ptr(y),
                                             int(bool(refresh)), _stream_ptr(stream)),
                  "mgr_jacobian_product") == 1


def mgr_splitmix64_device(inp, out, stream=None):
    return _check(lib().mgr_splitmix64_device(_ptr(inp), _ptr(out), inp.numel(),
                                              _stream_ptr(stream)), "mgr_splitmix64_device")


def mgr_get_block_colors(h, level):
    """(colours of the level's point blocks, colour count) or None."""
    nc = C.c_int32(0)
    n = lib().mgr_get_block_colors(h, int(level), None, C.byref(nc))
    if n < 0:
        return None
    out = np.zeros(n, dtype=np.int32)
    _check(lib().mgr_get_block_colors(h, int(level), out.ctypes.data, C.byref(nc)),
           "mgr_get_block_colors")
    return out, nc.value


def mgr_launch_count():
    """Kernel launches issued by the library so far in this process."""
    return int(lib().mgr_launch_count())


def mgr_build_id():
    """Source hash the loaded library was compiled from."""
    return lib().mgr_build_id().decode()


def mgr_memory_usage():
    """(used, reserved) bytes of the library's device memory pool."""
    u, r = C.c_size_t(0), C.c_size_t(0)
    _check(lib().mgr_memory_usage(C.byref(u), C.byref(r)), "mgr_memory_usage")
    return u.value, r.value


def mgr_host_launch_count():
    """Launch calls issued by the library's host code (a graph launch counts once)."""
    return int(lib().mgr_host_launch_count())


def mgr_trim_memory(keep_bytes=0):
    """Return the library pool's unused device memory to the driver."""
    return _check(lib().mgr_trim_memory(int(keep_bytes)), "mgr_trim_memory")


class Solver:
    """Convenience wrapper: device copy of a problem + MGR handle."""

    def __init__(self, prob, precision=MGR_FP64, stream=None, **opt_overrides):
        two_phase = bool(prob.meta.get("two_phase", True))
        self.A = DeviceMatrix(prob)
        self.opts = mgr_options_default(two_phase, precision=precision, **opt_overrides)
        self.stream = stream
        self.h = mgr_setup(self.A, self.opts, stream)

    def solve(self, b, restart=50, max_iter=1000, rtol=1e-8, hist_cap=0, ortho=MGR_ORTHO_AUTO):
        import torch
        x = torch.zeros_like(b)
        r = fgmres_solve(self.h, self.A, b, x,
                         fgmres_options_default(restart=restart, max_iter=max_iter, rtol=rtol,
                                                ortho=ortho),
                         self.stream, hist_cap=hist_cap)
        r["x"] = x
        return r

    def apply(self, v):
        import torch
        z = torch.empty_like(v)
        mgr_apply(self.h, v, z, self.stream)
        return z

    def close(self):
        if getattr(self, "h", None):
            mgr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
