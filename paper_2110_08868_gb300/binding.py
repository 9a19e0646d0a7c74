"""Thin ctypes binding of libsdot (include/sdot.h): argument marshalling only.

Every function keeps the C name and returns the C status code; the buffers may be
numpy arrays (host memory) or torch tensors (host or CUDA memory). ``check``
turns a status into an exception carrying ``sdot_last_error()``. ``Solver`` owns one
context (one box), ``Server`` one reconstruction server (many boxes, queued and run
concurrently). The library must be built (``paper_2110_08868_gb300.build``); there is
no fallback path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsdot.so")

SDOT_OK = 0
ERRORS = {
    -1: "SDOT_ERR_ARG", -2: "SDOT_ERR_MASS", -3: "SDOT_ERR_DUPLICATE", -4: "SDOT_ERR_TOO_FEW",
    -5: "SDOT_ERR_OOM", -6: "SDOT_ERR_NO_DESCENT", -7: "SDOT_ERR_MAXIT",
    -8: "SDOT_ERR_EMPTY_CELL", -9: "SDOT_ERR_TIMEOUT", -10: "SDOT_ERR_CUDA",
    -11: "SDOT_ERR_CAPACITY", -12: "SDOT_ERR_NOT_READY",
}
for _v, _n in ERRORS.items():
    globals()[_n] = _v
SDOT_PREC_FP64 = 0
SDOT_PREC_MIXED = 1
SDOT_JOB_QUEUED, SDOT_JOB_RUNNING, SDOT_JOB_DONE, SDOT_JOB_FAILED = 0, 1, 2, 3


class sdot_options(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("precision", ctypes.c_int),
                ("seeds_per_leaf", ctypes.c_double), ("cg_rtol", ctypes.c_double),
                ("cg_maxit", ctypes.c_int), ("newton_maxit", ctypes.c_int),
                ("alpha_min", ctypes.c_double), ("verbose", ctypes.c_int),
                ("warm_alpha", ctypes.c_int), ("carry_certificates", ctypes.c_int)]


class sdot_csr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("row_ptr", ctypes.c_void_p),
                ("col", ctypes.c_void_p), ("val", ctypes.c_void_p)]


class sdot_stats(ctypes.Structure):
    _fields_ = [("newton_iters", ctypes.c_int), ("laguerre_evals", ctypes.c_int),
                ("cg_iters", ctypes.c_int64), ("max_rel_err", ctypes.c_double),
                ("l2_err", ctypes.c_double), ("min_vol", ctypes.c_double),
                ("last_alpha", ctypes.c_double), ("requeued", ctypes.c_int64),
                ("reclipped_fp64", ctypes.c_int64), ("ms_knn", ctypes.c_double),
                ("ms_clip", ctypes.c_double), ("ms_cg", ctypes.c_double),
                ("ms_total", ctypes.c_double), ("ms_pass", ctypes.c_double * 3),
                ("refined_fp64", ctypes.c_int), ("evals_fp32", ctypes.c_int),
                ("ms_pass1_fp32", ctypes.c_double), ("hess_slots", ctypes.c_int64),
                ("hess_offdiag", ctypes.c_int64)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_}
        d["ms_pass"] = list(self.ms_pass)
        return d


class sdot_eval_info(ctypes.Structure):
    _fields_ = [("ms_clip", ctypes.c_double), ("ms_pass", ctypes.c_double * 3),
                ("requeued", ctypes.c_int64), ("reclipped_fp64", ctypes.c_int64),
                ("n_empty", ctypes.c_int64), ("max_rel_err", ctypes.c_double),
                ("l2_err", ctypes.c_double), ("min_vol", ctypes.c_double),
                ("precision", ctypes.c_int), ("carried", ctypes.c_int64)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_}
        d["ms_pass"] = list(self.ms_pass)
        return d


class sdot_server_options(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_size_t), ("max_active", ctypes.c_int),
                ("device", ctypes.c_int), ("batch_clip", ctypes.c_int)]


class sdot_server_info(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_size_t), ("used_bytes", ctypes.c_size_t),
                ("peak_used_bytes", ctypes.c_size_t), ("max_active", ctypes.c_int),
                ("active", ctypes.c_int), ("peak_active", ctypes.c_int),
                ("queued", ctypes.c_int64), ("finished", ctypes.c_int64),
                ("submitted", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


# every symbol include/sdot.h declares
EXPORTS = ["sdot_default_options", "sdot_create", "sdot_set_stream", "sdot_set_allocator",
           "sdot_laguerre",
           "sdot_solve", "sdot_csr_copy", "sdot_get_psi", "sdot_displacement", "sdot_knn",
           "sdot_cell_status", "sdot_knn_static", "sdot_last_eval", "sdot_mesh", "sdot_size",
           "sdot_power_spectrum",
           "sdot_destroy",
           "sdot_kernel_launches", "sdot_last_error",
           "sdot_server_default_options", "sdot_server_footprint", "sdot_server_create",
           "sdot_server_submit", "sdot_server_poll", "sdot_server_wait", "sdot_server_result",
           "sdot_server_get_info", "sdot_server_destroy"]
_NO_STATUS = ("sdot_destroy", "sdot_last_error", "sdot_kernel_launches", "sdot_server_destroy")

_lib = None

# sdot_set_allocator callback types: alloc(bytes, user) -> ptr, free(ptr, user)
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)
_allocator_refs = None  # keeps the installed callbacks alive


class SdotError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


def load(path=LIB_PATH):
    """Load libsdot.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libsdot.so is not built ({path}); run paper_2110_08868_gb300.build")
    lib = ctypes.CDLL(path)
    P, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    lib.sdot_default_options.argtypes = [ctypes.POINTER(sdot_options)]
    lib.sdot_create.argtypes = [P, P, I64, P, ctypes.POINTER(sdot_options), ctypes.POINTER(P)]
    lib.sdot_set_stream.argtypes = [P, P]
    lib.sdot_set_allocator.argtypes = [ALLOC_FN, FREE_FN, P]
    lib.sdot_laguerre.argtypes = [P, P, P, P, ctypes.POINTER(sdot_csr)]
    lib.sdot_solve.argtypes = [P, D, P, ctypes.POINTER(sdot_stats)]
    lib.sdot_csr_copy.argtypes = [ctypes.POINTER(sdot_csr), P, P, P]
    lib.sdot_get_psi.argtypes = [P, P]
    lib.sdot_displacement.argtypes = [P, P]
    lib.sdot_knn.argtypes = [P, P]
    lib.sdot_cell_status.argtypes = [P, P]
    lib.sdot_knn_static.argtypes = [P, I64, P, I, P, P]
    lib.sdot_size.argtypes = [P, ctypes.POINTER(I64), ctypes.POINTER(I)]
    lib.sdot_last_eval.argtypes = [P, ctypes.POINTER(sdot_eval_info)]
    lib.sdot_mesh.argtypes = [P, D, I, P, P, P]
    lib.sdot_power_spectrum.argtypes = [P, I, D, I, P, P, P, P]
    lib.sdot_destroy.argtypes = [P]
    lib.sdot_destroy.restype = None
    lib.sdot_kernel_launches.argtypes = []
    lib.sdot_kernel_launches.restype = I64
    lib.sdot_last_error.argtypes = []
    lib.sdot_last_error.restype = ctypes.c_char_p
    lib.sdot_server_default_options.argtypes = [ctypes.POINTER(sdot_server_options)]
    lib.sdot_server_footprint.argtypes = [I64, P, ctypes.POINTER(sdot_options),
                                          ctypes.POINTER(ctypes.c_size_t)]
    lib.sdot_server_create.argtypes = [ctypes.POINTER(sdot_server_options), ctypes.POINTER(P)]
    lib.sdot_server_submit.argtypes = [P, P, P, I64, P, ctypes.POINTER(sdot_options), D,
                                       ctypes.POINTER(I64)]
    lib.sdot_server_poll.argtypes = [P, I64, ctypes.POINTER(I)]
    lib.sdot_server_wait.argtypes = [P, I64, D, ctypes.POINTER(I)]
    lib.sdot_server_result.argtypes = [P, I64, P, P, ctypes.POINTER(sdot_stats), P]
    lib.sdot_server_get_info.argtypes = [P, ctypes.POINTER(sdot_server_info)]
    lib.sdot_server_destroy.argtypes = [P]
    lib.sdot_server_destroy.restype = None
    for name in EXPORTS:
        if name not in _NO_STATUS:
            getattr(lib, name).restype = I
    _lib = lib
    return lib


def _ptr(x, dtype=np.float64):
    """Raw address of a numpy array or torch tensor (contiguous, right dtype)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):  # torch tensor
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        want = {np.float64: "torch.float64", np.int32: "torch.int32",
                np.int64: "torch.int64", np.uint8: "torch.uint8"}[dtype]
        if str(x.dtype) != want:
            raise TypeError(f"expected {want}, got {x.dtype}")
        return ctypes.c_void_p(x.data_ptr())
    if not isinstance(x, np.ndarray) or x.dtype != dtype or not x.flags.c_contiguous:
        raise TypeError(f"expected a C-contiguous numpy array of {np.dtype(dtype)}")
    return ctypes.c_void_p(x.ctypes.data)


def sdot_kernel_launches():
    return int(load().sdot_kernel_launches())


def sdot_last_error():
    return load().sdot_last_error().decode()


def check(rc):
    if rc != SDOT_OK:
        raise SdotError(rc, sdot_last_error())
    return rc


def sdot_default_options(**kw):
    o = sdot_options()
    load().sdot_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = {"fp64": SDOT_PREC_FP64, "mixed": SDOT_PREC_MIXED}[v]
        setattr(o, k, v)
    return o


def sdot_create(pos, mass, box, opt=None):
    """Returns (rc, ctx). pos: N x 3 float64; mass: N float64 or None; box: 3 floats."""
    lib = load()
    n = int(pos.shape[0])
    b = np.ascontiguousarray(np.broadcast_to(np.asarray(box, dtype=np.float64), (3,)))
    ctx = ctypes.c_void_p()
    rc = lib.sdot_create(_ptr(pos), _ptr(mass), n, ctypes.c_void_p(b.ctypes.data),
                         ctypes.byref(opt) if opt is not None else None, ctypes.byref(ctx))
    return rc, ctx


def sdot_set_allocator(alloc=None, free=None):
    """Install Python callables alloc(bytes) -> device address (0: failure) and
    free(ptr) for the contexts created later; no arguments restores cudaMalloc/cudaFree."""
    global _allocator_refs
    fa = ALLOC_FN(lambda n, u: alloc(n) or None) if alloc is not None else ALLOC_FN()
    ff = FREE_FN(lambda p, u: free(p)) if free is not None else FREE_FN()
    rc = load().sdot_set_allocator(fa, ff, None)
    if rc == SDOT_OK:
        _allocator_refs = (fa, ff) if alloc is not None else None
    return rc


def sdot_set_stream(ctx, stream):
    """stream: a torch.cuda.Stream, a raw cudaStream_t integer, or None."""
    h = getattr(stream, "cuda_stream", stream)
    return load().sdot_set_stream(ctx, ctypes.c_void_p(h) if h else None)


def sdot_laguerre(ctx, psi=None, volumes=None, centroids=None, hess=None):
    """hess: an sdot_csr() to receive borrowed device pointers, or None."""
    return load().sdot_laguerre(ctx, _ptr(psi), _ptr(volumes), _ptr(centroids),
                                ctypes.byref(hess) if hess is not None else None)


def sdot_solve(ctx, tol, psi0=None, stats=None):
    return load().sdot_solve(ctx, float(tol), _ptr(psi0),
                             ctypes.byref(stats) if stats is not None else None)


def sdot_get_psi(ctx, psi):
    return load().sdot_get_psi(ctx, _ptr(psi))


def sdot_displacement(ctx, disp):
    return load().sdot_displacement(ctx, _ptr(disp))


def sdot_knn(ctx, nbr):
    return load().sdot_knn(ctx, _ptr(nbr, np.int32))


def sdot_cell_status(ctx, status):
    return load().sdot_cell_status(ctx, _ptr(status, np.uint8))


SDOT_STATIC_MAX_N = 32768
SDOT_STATIC_MAX_K = 32


def _check_knn_static_args(pos, k, nbr):
    """Shapes and placement sdot_knn_static relies on: the C call cannot see buffer
    sizes, so a (N, 2) pos or a short nbr would make its kernels read or write past
    the caller's buffers. Raises ValueError."""
    for name, t in (("pos", pos), ("nbr", nbr)):
        if not hasattr(t, "is_cuda") or not t.is_cuda:
            raise ValueError(f"sdot_knn_static: {name} must be a CUDA tensor")
    if pos.dim() != 2 or pos.shape[1] != 3:
        raise ValueError(f"sdot_knn_static: pos must have shape (N, 3), got {tuple(pos.shape)}")
    n = int(pos.shape[0])
    if tuple(nbr.shape) != (n, int(k)):
        raise ValueError(f"sdot_knn_static: nbr must have shape ({n}, {int(k)}), "
                         f"got {tuple(nbr.shape)}")
    if pos.device != nbr.device:
        raise ValueError("sdot_knn_static: pos and nbr must be on the same device")


def sdot_knn_static(pos, box, k, nbr, stream=None):
    """kNN lists without device allocation (pos: (N, 3) float64, nbr: (N, k) int32, both
    CUDA tensors on the current device; see include/sdot.h)."""
    _check_knn_static_args(pos, k, nbr)
    b = np.ascontiguousarray(np.broadcast_to(np.asarray(box, dtype=np.float64), (3,)))
    h = getattr(stream, "cuda_stream", stream)
    return load().sdot_knn_static(_ptr(pos), int(pos.shape[0]), ctypes.c_void_p(b.ctypes.data),
                                  int(k), _ptr(nbr, np.int32), ctypes.c_void_p(h) if h else None)


def sdot_mesh(ctx, lam, mesh, rho=None, phi=None, owner=None):
    return load().sdot_mesh(ctx, float(lam), int(mesh), _ptr(rho), _ptr(phi),
                            _ptr(owner, np.int32))


def sdot_power_spectrum(rho, L, nbins=None, stream=None):
    """Power spectrum of an M^3 density mesh of a cubic box of side L (host array or
    CUDA tensor, indexed [z, y, x]; see include/sdot.h). Returns (P, kmean, nmodes) per
    bin."""
    M = int(rho.shape[0])
    if tuple(rho.shape) != (M, M, M):
        raise ValueError("rho must be an M x M x M mesh")
    if hasattr(rho, "is_contiguous"):
        if rho.dtype != __import__("torch").float64 or not rho.is_contiguous():
            raise ValueError("rho must be a contiguous float64 tensor")
    else:
        rho = np.ascontiguousarray(rho, dtype=np.float64)
    nb = M // 2 if nbins is None else int(nbins)
    P = np.zeros(nb)
    k = np.zeros(nb)
    n = np.zeros(nb, dtype=np.int64)
    h = getattr(stream, "cuda_stream", stream)
    check(load().sdot_power_spectrum(_ptr(rho), M, float(L), nb, _ptr(P), _ptr(k),
                                     _ptr(n, np.int64), ctypes.c_void_p(h) if h else None))
    return P, k, n


def sdot_last_eval(ctx, info):
    return load().sdot_last_eval(ctx, ctypes.byref(info))


def sdot_size(ctx):
    n = ctypes.c_int64()
    k = ctypes.c_int()
    rc = load().sdot_size(ctx, ctypes.byref(n), ctypes.byref(k))
    return rc, n.value, k.value


def sdot_destroy(ctx):
    if ctx:
        load().sdot_destroy(ctx)


class Solver:
    """Owning convenience wrapper over one context (raises on errors)."""

    def __init__(self, pos, box, mass=None, **opts):
        self.opt = sdot_default_options(**opts)
        rc, self.ctx = sdot_create(pos, mass, box, self.opt)
        check(rc)
        _, self.N, self.k = sdot_size(self.ctx)

    def close(self):
        if self.ctx:
            sdot_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def laguerre(self, psi=None, with_hessian=False, allow_empty=False):
        vol = np.empty(self.N)
        cen = np.empty((self.N, 3))
        h = sdot_csr() if with_hessian else None
        rc = sdot_laguerre(self.ctx, psi, vol, cen, h)
        if not (allow_empty and rc == SDOT_ERR_EMPTY_CELL):
            check(rc)
        out = dict(vol=vol, centroid=cen, rc=rc)
        if with_hessian:
            out["hess"] = csr_to_scipy(h)
        return out

    def solve(self, tol, psi0=None):
        st = sdot_stats()
        check(sdot_solve(self.ctx, tol, psi0, st))
        return st.as_dict()

    def psi(self):
        out = np.empty(self.N)
        check(sdot_get_psi(self.ctx, out))
        return out

    def displacement(self):
        out = np.empty((self.N, 3))
        check(sdot_displacement(self.ctx, out))
        return out

    def mesh(self, lam, M):
        """rho (moved-cell mass density), phi (phi_I) and owner on the M^3 mesh, each
        shaped (M, M, M) and indexed [z, y, x]."""
        rho = np.empty(M ** 3)
        phi = np.empty(M ** 3)
        owner = np.empty(M ** 3, dtype=np.int32)
        check(sdot_mesh(self.ctx, lam, M, rho, phi, owner))
        return {"rho": rho.reshape(M, M, M), "phi": phi.reshape(M, M, M),
                "owner": owner.reshape(M, M, M)}

    def status(self):
        out = np.empty(self.N, dtype=np.uint8)
        check(sdot_cell_status(self.ctx, out))
        return out

    def knn(self):
        out = np.empty((self.N, self.k), dtype=np.int32)
        check(sdot_knn(self.ctx, out))
        return out


def sdot_csr_copy(h, row_ptr, col, val):
    return load().sdot_csr_copy(ctypes.byref(h), _ptr(row_ptr, np.int64), _ptr(col, np.int32),
                                _ptr(val))


def csr_to_scipy(h):
    """Copy a borrowed device CSR (sdot_csr) to a scipy.sparse.csr_matrix."""
    import scipy.sparse as sp

    rp = np.empty(h.n + 1, dtype=np.int64)
    col = np.empty(h.nnz, dtype=np.int32)
    val = np.empty(h.nnz, dtype=np.float64)
    check(sdot_csr_copy(h, rp, col, val))
    return sp.csr_matrix((val, col, rp), shape=(h.n, h.n))


# ---------------------------------------------------------------------------
# reconstruction server
# ---------------------------------------------------------------------------
def _box3(box):
    return np.ascontiguousarray(np.broadcast_to(np.asarray(box, dtype=np.float64), (3,)))


def sdot_server_default_options(**kw):
    o = sdot_server_options()
    load().sdot_server_default_options(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def sdot_server_footprint(n, box, opt=None):
    """Returns (rc, bytes): device bytes a job of n seeds holds while admitted."""
    b = _box3(box)
    out = ctypes.c_size_t()
    rc = load().sdot_server_footprint(int(n), ctypes.c_void_p(b.ctypes.data),
                                      ctypes.byref(opt) if opt is not None else None,
                                      ctypes.byref(out))
    return rc, int(out.value)


def sdot_server_create(opt=None):
    """Returns (rc, srv)."""
    srv = ctypes.c_void_p()
    rc = load().sdot_server_create(ctypes.byref(opt) if opt is not None else None,
                                   ctypes.byref(srv))
    return rc, srv


def sdot_server_submit(srv, pos, mass, box, tol, opt=None):
    """Returns (rc, id). pos: N x 3 float64 numpy (host); mass: N float64 or None."""
    b = _box3(box)
    jid = ctypes.c_int64()
    rc = load().sdot_server_submit(srv, _ptr(pos), _ptr(mass), int(pos.shape[0]),
                                   ctypes.c_void_p(b.ctypes.data),
                                   ctypes.byref(opt) if opt is not None else None, float(tol),
                                   ctypes.byref(jid))
    return rc, int(jid.value)


def sdot_server_poll(srv, jid):
    st = ctypes.c_int()
    rc = load().sdot_server_poll(srv, int(jid), ctypes.byref(st))
    return rc, st.value


def sdot_server_wait(srv, jid, timeout_s=-1.0):
    st = ctypes.c_int(-1)
    rc = load().sdot_server_wait(srv, int(jid), float(timeout_s), ctypes.byref(st))
    return rc, st.value


def sdot_server_result(srv, jid, disp=None, psi=None, stats=None, times=None):
    """disp (N x 3), psi (N), times (3): float64 numpy arrays or None."""
    return load().sdot_server_result(srv, int(jid), _ptr(disp), _ptr(psi),
                                     ctypes.byref(stats) if stats is not None else None,
                                     _ptr(times))


def sdot_server_get_info(srv):
    info = sdot_server_info()
    rc = load().sdot_server_get_info(srv, ctypes.byref(info))
    return rc, info


def sdot_server_destroy(srv):
    if srv:
        load().sdot_server_destroy(srv)


class Server:
    """Owning wrapper over one reconstruction server (raises on errors)."""

    def __init__(self, hbm_budget=0, max_active=8, device=-1, batch_clip=True):
        rc, self.srv = sdot_server_create(sdot_server_default_options(
            hbm_budget=int(hbm_budget), max_active=int(max_active), device=int(device),
            batch_clip=int(bool(batch_clip))))
        check(rc)
        self._n = {}

    def submit(self, pos, box, tol, mass=None, **opts):
        pos = np.ascontiguousarray(pos, dtype=np.float64)
        rc, jid = sdot_server_submit(self.srv, pos, mass, box, tol, sdot_default_options(**opts))
        check(rc)
        self._n[jid] = int(pos.shape[0])
        return jid

    def state(self, jid):
        rc, st = sdot_server_poll(self.srv, jid)
        check(rc)
        return st

    def wait(self, jid, timeout_s=-1.0):
        """True when the job finished within timeout_s seconds."""
        rc, _ = sdot_server_wait(self.srv, jid, timeout_s)
        if rc == SDOT_ERR_TIMEOUT:
            return False
        check(rc)
        return True

    def result(self, jid):
        """dict(disp, psi, stats, times) of a finished job; raises on its error."""
        n = self._n[jid]
        disp = np.empty((n, 3))
        psi = np.empty(n)
        st = sdot_stats()
        times = np.empty(3)
        rc = sdot_server_result(self.srv, jid, disp, psi, st, times)
        if rc != SDOT_ERR_NOT_READY:
            self._n.pop(jid, None)
        check(rc)
        return dict(disp=disp, psi=psi, stats=st.as_dict(), times=times)

    def info(self):
        rc, info = sdot_server_get_info(self.srv)
        check(rc)
        return info.as_dict()

    def close(self):
        if self.srv:
            sdot_server_destroy(self.srv)
            self.srv = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
