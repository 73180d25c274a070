"""CPU FP64 oracle of MGR-preconditioned FGMRES (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline may import this package.  The product path (the CUDA library and its
binding) never does, and the two share no code: the oracle is the plain C file
``mgr_oracle.c`` in this directory, compiled with ``-ffp-contract=off`` so that
every setup multiply and add is rounded on its own, in the order the paper's
definitions give (ascending inner index).

Functions and what pins them are listed in the test files under ``tests/``;
``mgr_oracle.c`` cites the paper's section, equation or algorithm for each step.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mgr_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libmgr_oracle.so")
_lock = threading.Lock()
_lib = None

MAXL = 8

Q_MGR_A, Q_MGR_W, Q_MGR_COR, Q_MGR_CORKEPT, Q_MGR_S, Q_MGR_WR, Q_MGR_BD = 0, 1, 2, 3, 4, 5, 6
Q_MGR_ILU = 7
Q_AMG_A, Q_AMG_S, Q_AMG_P, Q_AMG_R = 10, 11, 12, 13

FRELAX_AMG, FRELAX_JACOBI = 0, 1


class OrcOpts(C.Structure):
    _fields_ = [
        ("num_levels", C.c_int32),
        ("f_label_mask", C.c_uint32 * MAXL),
        ("frelax", C.c_int32 * MAXL),
        ("frelax_sweeps", C.c_int32 * MAXL),
        ("nmax_drop", C.c_int32 * MAXL),
        ("global_sweeps", C.c_int32 * MAXL),
        ("amg_theta", C.c_double),
        ("amg_pmax", C.c_int32),
        ("amg_max_coarse", C.c_int32),
        ("amg_max_levels", C.c_int32),
        ("seed", C.c_uint64),
        ("restrict_jacobi", C.c_int32 * MAXL),
        ("frelax_post", C.c_int32 * MAXL),
        ("dff_block", C.c_int32 * MAXL),
        ("global_smoother", C.c_int32 * MAXL),
        ("agg_levels", C.c_int32 * MAXL),
        ("ilu_solve_sweeps", C.c_int32),
    ]


def _hash():
    import hashlib
    with open(_SRC, "rb") as f:
        return hashlib.sha256(f.read() + " ".join(_CFLAGS).encode()).hexdigest()[:16]


_CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


def build(force=False):
    """Compile the oracle into oracle/_build (plain gcc, no GPU needed); a
    build is reused only when the source hash recorded beside it matches."""
    os.makedirs(_BUILD, exist_ok=True)
    stamp = _LIB + ".build_id"
    want = _hash()
    if not force and os.path.exists(_LIB) and os.path.exists(stamp):
        with open(stamp) as f:
            if f.read().strip() == want:
                return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc"] + _CFLAGS + ["-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    with open(stamp + ".tmp", "w") as f:
        f.write(want + "\n")
    os.replace(stamp + ".tmp", stamp)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            P = C.c_void_p
            L.orc_setup.restype = P
            L.orc_setup.argtypes = [C.c_int64, P, P, P, P, P, P, C.POINTER(OrcOpts),
                                    C.POINTER(C.c_int)]
            L.orc_free.argtypes = [P]
            L.orc_apply.argtypes = [P, P, P]
            L.orc_vcycle.argtypes = [P, C.c_int, P, P]
            L.orc_fgmres.argtypes = [P, P, P, C.c_int, C.c_int, C.c_double,
                                     C.POINTER(C.c_int), C.POINTER(C.c_double), P, C.c_int]
            L.orc_get_csr.argtypes = [P, C.c_int, C.c_int, C.c_int, P, P, P, P]
            L.orc_amg_levels.argtypes = [P, C.c_int]
            L.orc_get_cf.restype = C.c_int64
            L.orc_get_cf.argtypes = [P, C.c_int, C.c_int, P]
            L.orc_get_l1.restype = C.c_int64
            L.orc_get_l1.argtypes = [P, C.c_int, C.c_int, P]
            L.orc_global_relax.argtypes = [P, C.c_int, P, P]
            L.orc_get_block_colors.restype = C.c_int64
            L.orc_get_block_colors.argtypes = [P, C.c_int, P, P]
            L.orc_pmis.argtypes = [C.c_int64, P, P, C.c_uint64, C.c_int, C.c_int, P]
            L.orc_interp.argtypes = [C.c_int64, P, P, P, P, P, P, P, C.c_int, P,
                                     C.POINTER(C.POINTER(C.c_int64)),
                                     C.POINTER(C.POINTER(C.c_int32)),
                                     C.POINTER(C.POINTER(C.c_double))]
            L.orc_free_buffer.argtypes = [P]
            L.orc_matvec.argtypes = [P, P, P]
            L.orc_csr_spmv.argtypes = [C.c_int64, P, P, P, P, P]
            L.orc_splitmix64.restype = C.c_uint64
            L.orc_splitmix64.argtypes = [C.c_uint64]
            _lib = L
    return _lib


def default_options(two_phase=True, **kw):
    """The solver configuration of Sec. 5.3 / Sec. 6.

    two-phase: level 0 F = {u} (F-relaxation: one AMG V-cycle, N_max = 4),
               level 1 F = {s} (one Jacobi sweep, no dropping, 3 sweeps of
               cell-block Jacobi as global smoother), coarsest = {p} by AMG.
    single-phase: level 0 F = {u}, coarsest = {p}.
    Operator variants of Sec. 5.1, per level, all off by default:
    restrict_jacobi (W_r = -A_CF D_FF^-1), frelax_post (Eq. MGR-post),
    dff_block (D_FF = point-block diagonal of A_FF); global_smoother 1 =
    multicolour point-block Gauss-Seidel, 2 = ILU(1) (ilu_solve_sweeps Jacobi
    iterations per triangular solve), instead of point-block Jacobi;
    agg_levels[s] = leading levels of AMG slot s coarsened aggressively.
    """
    d = dict(num_levels=2 if two_phase else 1,
             f_label_mask=[1 << 0, 1 << 1] if two_phase else [1 << 0],
             frelax=[FRELAX_AMG, FRELAX_JACOBI] if two_phase else [FRELAX_AMG],
             frelax_sweeps=[1, 1] if two_phase else [1],
             nmax_drop=[4, -1] if two_phase else [4],
             global_sweeps=[0, 3] if two_phase else [0],
             amg_theta=0.25, amg_pmax=4, amg_max_coarse=160, amg_max_levels=25, seed=0,
             restrict_jacobi=[0] * MAXL, frelax_post=[0] * MAXL, dff_block=[0] * MAXL,
             global_smoother=[0] * MAXL, agg_levels=[0] * MAXL,
             ilu_solve_sweeps=3)
    d.update(kw)
    return d


def _opts_struct(d):
    o = OrcOpts()
    o.num_levels = d["num_levels"]
    for name in ("f_label_mask", "frelax", "frelax_sweeps", "nmax_drop", "global_sweeps",
                 "restrict_jacobi", "frelax_post", "dff_block", "global_smoother",
                 "agg_levels"):
        arr = getattr(o, name)
        for i, v in enumerate(d[name]):
            arr[i] = v
    o.amg_theta = d["amg_theta"]
    o.amg_pmax = d["amg_pmax"]
    o.amg_max_coarse = d["amg_max_coarse"]
    o.amg_max_levels = d["amg_max_levels"]
    o.seed = d["seed"]
    o.ilu_solve_sweeps = d["ilu_solve_sweeps"]
    return o


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


class Oracle:
    """Hierarchy built by the oracle for one matrix (see mgr_oracle.c)."""

    def __init__(self, prob=None, *, n=None, row_ptr=None, col=None, val=None, label=None,
                 node=None, comp=None, **opts):
        if prob is not None:
            n, row_ptr, col, val = prob.n, prob.row_ptr, prob.col, prob.val
            label, node, comp = prob.dof_label, prob.dof_node, prob.dof_comp
            opts.setdefault("two_phase", bool(prob.meta.get("two_phase", True)))
        two_phase = opts.pop("two_phase", True)
        self.opts = default_options(two_phase, **opts)
        self._keep = [np.ascontiguousarray(row_ptr, dtype=np.int64),
                      np.ascontiguousarray(col, dtype=np.int32),
                      np.ascontiguousarray(val, dtype=np.float64),
                      np.ascontiguousarray(label, dtype=np.int32),
                      np.ascontiguousarray(node, dtype=np.int32),
                      np.ascontiguousarray(comp if comp is not None else np.zeros(n),
                                           dtype=np.int32)]
        self.n = int(n)
        self._o = _opts_struct(self.opts)
        st = C.c_int(0)
        self.h = lib().orc_setup(self.n, *[_p(a) for a in self._keep], C.byref(self._o),
                                 C.byref(st))
        self.status = st.value
        if not self.h:
            raise RuntimeError(f"oracle setup failed with status {st.value}")

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            lib().orc_free(h)
            self.h = None

    @property
    def num_levels(self):
        return self.opts["num_levels"]

    def apply(self, v):
        v = np.ascontiguousarray(v, dtype=np.float64)
        z = np.zeros(self.n)
        lib().orc_apply(self.h, _p(v), _p(z))
        return z

    def matvec(self, x):
        """y = A x with the input matrix."""
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.zeros(self.n)
        lib().orc_matvec(self.h, _p(x), _p(y))
        return y

    def vcycle(self, slot, b):
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros_like(b)
        if lib().orc_vcycle(self.h, slot, _p(b), _p(x)) != 0:
            raise ValueError("no AMG in that slot")
        return x

    def fgmres(self, b, restart=50, maxit=1000, rtol=1e-8, hist_cap=0):
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros(self.n)
        it = C.c_int(0)
        rr = C.c_double(0)
        hist = np.zeros(max(hist_cap, 1))
        st = lib().orc_fgmres(self.h, _p(b), _p(x), restart, maxit, rtol, C.byref(it),
                              C.byref(rr), _p(hist), hist_cap)
        return dict(x=x, iters=it.value, relres=rr.value, status=st,
                    hist=hist[:min(hist_cap, it.value + 1)])

    def csr(self, kind, slot=0, lvl=0):
        """(rows, cols, row_ptr, col, val) of a hierarchy matrix, or None."""
        dims = np.zeros(3, dtype=np.int64)
        if lib().orc_get_csr(self.h, kind, slot, lvl, _p(dims), None, None, None) != 0:
            return None
        nr, nc, nnz = (int(x) for x in dims)
        rp = np.zeros(nr + 1, dtype=np.int64)
        ci = np.zeros(nnz, dtype=np.int32)
        v = np.zeros(nnz)
        lib().orc_get_csr(self.h, kind, slot, lvl, _p(dims), _p(rp), _p(ci), _p(v))
        return nr, nc, rp, ci, v

    def scipy(self, kind, slot=0, lvl=0):
        import scipy.sparse as sp
        r = self.csr(kind, slot, lvl)
        if r is None:
            return None
        nr, nc, rp, ci, v = r
        return sp.csr_matrix((v, ci, rp), shape=(nr, nc))

    def amg_levels(self, slot):
        return lib().orc_amg_levels(self.h, slot)

    def cf(self, slot, lvl):
        n = lib().orc_get_cf(self.h, slot, lvl, None)
        if n < 0:
            return None
        out = np.zeros(n, dtype=np.int8)
        lib().orc_get_cf(self.h, slot, lvl, _p(out))
        return out

    def global_relax(self, l, v):
        """z = M_glo^-1 v of MGR level l alone."""
        v = np.ascontiguousarray(v, dtype=np.float64)
        z = np.zeros_like(v)
        if lib().orc_global_relax(self.h, l, _p(v), _p(z)) != 0:
            raise ValueError("no such level")
        return z

    def block_colors(self, l):
        """(colours of level l's point blocks, colour count), or None."""
        nc = C.c_int32(0)
        n = lib().orc_get_block_colors(self.h, l, None, C.byref(nc))
        if n < 0:
            return None
        out = np.zeros(n, dtype=np.int32)
        lib().orc_get_block_colors(self.h, l, _p(out), C.byref(nc))
        return out, nc.value

    def l1(self, slot, lvl):
        n = lib().orc_get_l1(self.h, slot, lvl, None)
        out = np.zeros(n)
        lib().orc_get_l1(self.h, slot, lvl, _p(out))
        return out


def csr_spmv(row_ptr, col, val, x):
    """y = A x for a CSR matrix given by its arrays (any size)."""
    n = len(row_ptr) - 1
    arrs = [np.ascontiguousarray(row_ptr, dtype=np.int64), np.ascontiguousarray(col, dtype=np.int32),
            np.ascontiguousarray(val, dtype=np.float64), np.ascontiguousarray(x, dtype=np.float64)]
    y = np.zeros(n)
    lib().orc_csr_spmv(n, *[_p(a) for a in arrs], _p(y))
    return y


def pmis(S, seed=0, slot=0, level=0):
    """PMIS C/F marks (+1/-1) of the strength graph S (scipy CSR, n x n)."""
    S = S.tocsr()
    S.sort_indices()
    rp = np.ascontiguousarray(S.indptr, dtype=np.int64)
    ci = np.ascontiguousarray(S.indices, dtype=np.int32)
    cf = np.zeros(S.shape[0], dtype=np.int8)
    if lib().orc_pmis(S.shape[0], _p(rp), _p(ci), seed, slot, level, _p(cf)) != 0:
        raise ValueError("orc_pmis failed")
    return cf


def interp(A, S, cf, comp=None, pmax=0):
    """Direct interpolation P (scipy CSR) of A with the given strength graph S,
    C/F marks and components."""
    import scipy.sparse as sp
    A = A.tocsr()
    A.sort_indices()
    S = S.tocsr()
    S.sort_indices()
    n = A.shape[0]
    arrs = [np.ascontiguousarray(A.indptr, dtype=np.int64),
            np.ascontiguousarray(A.indices, dtype=np.int32),
            np.ascontiguousarray(A.data, dtype=np.float64),
            np.ascontiguousarray(S.indptr, dtype=np.int64),
            np.ascontiguousarray(S.indices, dtype=np.int32),
            np.ascontiguousarray(np.zeros(n) if comp is None else comp, dtype=np.int32),
            np.ascontiguousarray(cf, dtype=np.int8)]
    dims = np.zeros(3, dtype=np.int64)
    prp, pci, pv = C.POINTER(C.c_int64)(), C.POINTER(C.c_int32)(), C.POINTER(C.c_double)()
    if lib().orc_interp(n, *[_p(a) for a in arrs], pmax, _p(dims), C.byref(prp), C.byref(pci),
                        C.byref(pv)) != 0:
        raise ValueError("orc_interp failed")
    nr, nc, nnz = (int(x) for x in dims)
    rp = np.ctypeslib.as_array(prp, shape=(nr + 1,)).copy()
    ci = np.ctypeslib.as_array(pci, shape=(max(nnz, 1),))[:nnz].copy()
    v = np.ctypeslib.as_array(pv, shape=(max(nnz, 1),))[:nnz].copy()
    for q in (prp, pci, pv):
        lib().orc_free_buffer(C.cast(q, C.c_void_p))
    return sp.csr_matrix((v, ci, rp), shape=(nr, nc))


def splitmix64(x):
    return int(lib().orc_splitmix64(C.c_uint64(x & 0xFFFFFFFFFFFFFFFF)))
