"""Thin ctypes binding of libgmls (the C ABI in include/gmls.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  PyTorch provides device memory (the context arena and output
buffers) and streams.  If the library has not been built, ``load()`` raises;
there is no CPU fallback.

    ctx = Context(device=0)
    cid = ctx.cloud(x)                                   # gmls_cloud
    nid = ctx.neighbors(cid, k=12, eps_factor=1.5)       # gmls_neighbors
    sid = ctx.stencils(nid, basis=SCALAR, degree=2,
                       functionals=[LAPLACIAN, GRAD])   # gmls_stencils
    w = ctx.weights(sid, LAPLACIAN)                      # gmls_export
    row_ptr, col, val = ctx.assemble_csr(sid, LAPLACIAN) # gmls_csr_size + gmls_assemble_csr
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libgmls.so")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EBUSY, ENOTFOUND, ECANCELED = 0, -1, -2, -3, -4, -5, -6, -7
T_OK, T_RANK_DEFICIENT, T_ILL_CONDITIONED, T_REFINE_NOT_CONVERGED = 0, 1, 2, 4
T_TOO_FEW_NEIGHBOURS, T_FP64_FALLBACK, T_OVERFLOW = 8, 16, 32
KNN, RADIUS = 0, 1
SCALAR, DIVFREE, STAGGERED = 0, 1, 2
WEIGHT_POLY = 0
GRAD, LAPLACIAN, DIV, VEC_LAPLACIAN, CURLCURL = 0, 1, 2, 3, 4
FP64, FP32_REFINE = 0, 1
X_NBR_OFFSETS, X_NBR_INDEX, X_NBR_EPS, X_NBR_STATUS, X_WEIGHTS, X_BETA, X_STATUS, X_ITERS = range(8)

EXPORTED = [
    "gmls_create", "gmls_destroy", "gmls_set_stream", "gmls_cloud", "gmls_neighbors", "gmls_neighbors_prefix",
    "gmls_stencils",
    "gmls_stencil_info", "gmls_csr_size", "gmls_assemble_csr", "gmls_assemble_csr_at", "gmls_export", "gmls_export_size", "gmls_release",
    "gmls_sync", "gmls_arena_usage", "gmls_launch_count", "gmls_set_option", "gmls_knn_noalloc", "gmls_last_error",
    "gmls_version", "gmls_tune_info", "gmls_capture_begin", "gmls_capture_end", "gmls_graph_launch",
    "gmls_server_create", "gmls_server_submit", "gmls_server_wait", "gmls_server_result", "gmls_server_release",
    "gmls_server_cancel", "gmls_server_stats", "gmls_server_destroy", "gmls_stokes_size", "gmls_stokes_assemble", "gmls_stokes_rhs",
    "gmls_csr_spmv", "gmls_gmres",
]
NOALLOC_MAX_POINTS = 262144
OPT_FORCE_GENERIC, OPT_AUTOTUNE, OPT_CLEAR_TUNING, OPT_FORCE_VARIANT, OPT_POISON, OPT_FAIL_ALLOC = 0, 1, 2, 3, 4, 5
OPT_ORDER_KEY64 = 6
T_UNSUPPORTED = 64


class GmlsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"gmls error {code}: {msg}")
        self.code = code


class NbrParams(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("k", ctypes.c_int32), ("eps_factor", ctypes.c_double),
                ("cap", ctypes.c_int32), ("reserved", ctypes.c_int32), ("targets", ctypes.c_void_p),
                ("n_targets", ctypes.c_int64), ("halfspace", ctypes.c_void_p), ("k_per_target", ctypes.c_void_p)]


class StencilParams(ctypes.Structure):
    _fields_ = [("basis", ctypes.c_int32), ("degree", ctypes.c_int32), ("weight", ctypes.c_int32),
                ("weight_power", ctypes.c_int32), ("precision", ctypes.c_int32), ("n_functionals", ctypes.c_int32),
                ("functionals", ctypes.c_int32 * 5), ("neumann", ctypes.c_int32), ("max_refine", ctypes.c_int32),
                ("refine_tol", ctypes.c_double), ("degree_per_target", ctypes.c_void_p)]


class Request(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("n", ctypes.c_int64), ("xyz", ctypes.c_void_p), ("basis", ctypes.c_int32),
                ("degree", ctypes.c_int32), ("k", ctypes.c_int32), ("eps_factor", ctypes.c_double),
                ("precision", ctypes.c_int32), ("n_functionals", ctypes.c_int32), ("functionals", ctypes.c_int32 * 5)]


class StokesParams(ctypes.Structure):
    _fields_ = [("velocity", ctypes.c_int64), ("pressure", ctypes.c_int64), ("nu", ctypes.c_double),
                ("pressure_interior", ctypes.c_int64)]


class GmresParams(ctypes.Structure):
    _fields_ = [("restart", ctypes.c_int32), ("max_iter", ctypes.c_int32), ("rtol", ctypes.c_double),
                ("row_scaling", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class ServerStats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_int64), ("targets", ctypes.c_int64), ("pending", ctypes.c_int64),
                ("inflight", ctypes.c_int64), ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("mean_ms", ctypes.c_double), ("elapsed_s", ctypes.c_double), ("targets_per_s", ctypes.c_double)]


_lib = None


def load(path: str = LIB_PATH):
    """Load libgmls.so; raises if it is missing (build it with build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libgmls not built ({path} missing): run paper_2104_14447_gb300.build.build()")
    L = ctypes.CDLL(path)
    vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
    P64 = ctypes.POINTER(ctypes.c_int64)
    sig = {
        "gmls_create": [ctypes.POINTER(vp), ctypes.c_int, vp, vp, sz],
        "gmls_destroy": [vp],
        "gmls_set_stream": [vp, vp],
        "gmls_cloud": [vp, ctypes.c_int, i64, vp, vp, vp, P64],
        "gmls_neighbors": [vp, i64, ctypes.POINTER(NbrParams), P64],
        "gmls_neighbors_prefix": [vp, i64, i32, ctypes.c_double, P64],
        "gmls_stencils": [vp, i64, ctypes.POINTER(StencilParams), P64],
        "gmls_stencil_info": [vp, i64, i32, P64, ctypes.POINTER(i32), ctypes.POINTER(i32), P64],
        "gmls_csr_size": [vp, i64, i32, P64, P64, P64],
        "gmls_assemble_csr": [vp, i64, i32, vp, vp, vp],
        "gmls_assemble_csr_at": [vp, i64, i32, i64, vp, vp, vp],
        "gmls_export": [vp, i64, i32, i32, vp, sz],
        "gmls_export_size": [vp, i64, i32, i32, ctypes.POINTER(sz)],
        "gmls_release": [vp, i64],
        "gmls_sync": [vp],
        "gmls_arena_usage": [vp, ctypes.POINTER(sz), ctypes.POINTER(sz), ctypes.POINTER(sz)],
        "gmls_launch_count": [vp, P64],
        "gmls_set_option": [vp, i32, i64],
        "gmls_knn_noalloc": [ctypes.c_int, i64, vp, i32, ctypes.c_double, vp, vp, vp, vp],
        "gmls_tune_info": [vp, i32, ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_float)],
        "gmls_capture_begin": [vp],
        "gmls_capture_end": [vp, P64],
        "gmls_graph_launch": [vp, i64],
        "gmls_server_create": [ctypes.POINTER(vp), ctypes.c_int, vp, sz, i32, i32],
        "gmls_server_submit": [vp, ctypes.POINTER(Request), P64],
        "gmls_server_wait": [vp, i64, i32, ctypes.POINTER(i32)],
        "gmls_server_result": [vp, i64, i32, i32, vp, sz, ctypes.POINTER(sz)],
        "gmls_server_release": [vp, i64],
        "gmls_server_cancel": [vp, i64],
        "gmls_server_stats": [vp, ctypes.POINTER(ServerStats)],
        "gmls_server_destroy": [vp],
        "gmls_stokes_size": [vp, ctypes.POINTER(StokesParams), P64, P64],
        "gmls_stokes_assemble": [vp, ctypes.POINTER(StokesParams), vp, vp, vp],
        "gmls_stokes_rhs": [vp, ctypes.POINTER(StokesParams), vp, vp, vp, vp],
        "gmls_csr_spmv": [vp, i64, vp, vp, vp, vp, vp],
        "gmls_gmres": [vp, i64, vp, vp, vp, vp, vp, ctypes.POINTER(GmresParams), ctypes.POINTER(i32),
                       ctypes.POINTER(ctypes.c_double)],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int32
    L.gmls_last_error.argtypes = [vp]
    L.gmls_last_error.restype = ctypes.c_char_p
    L.gmls_version.argtypes = []
    L.gmls_version.restype = ctypes.c_char_p
    _lib = L
    return L


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        return ctypes.c_void_p(t.data_ptr())
    if isinstance(t, np.ndarray):
        return ctypes.c_void_p(t.ctypes.data)
    raise TypeError(type(t))


class Context:
    """One gmls context on one device and stream; owns a torch-allocated arena."""

    def __init__(self, device: int = 0, arena_bytes: int = 4 << 30, stream: torch.cuda.Stream | None = None):
        self.lib = load()
        self.device = torch.device("cuda", device)
        self.arena = torch.empty(arena_bytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        rc = self.lib.gmls_create(ctypes.byref(h), device, ctypes.c_void_p(self.stream.cuda_stream),
                                  _ptr(self.arena), arena_bytes)
        if rc != OK:
            raise GmlsError(rc, self.lib.gmls_last_error(None).decode())
        self.h = h
        self._keep = {}

    def _check(self, rc):
        if rc != OK:
            raise GmlsError(rc, self.lib.gmls_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.gmls_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --------------------------------------------------------------- calls
    def set_stream(self, stream: torch.cuda.Stream):
        self._check(self.lib.gmls_set_stream(self.h, ctypes.c_void_p(stream.cuda_stream)))
        self.stream = stream

    def cloud(self, x, normals=None, bflags=None) -> int:
        """x: (dim, n) float64 tensor/array (host or device), SoA."""
        x = _contig(x, torch.float64)
        dim, n = x.shape
        nr = _contig(normals, torch.float64) if normals is not None else None
        bf = _contig(bflags, torch.uint8) if bflags is not None else None
        out = ctypes.c_int64()
        self._check(self.lib.gmls_cloud(self.h, dim, n, _ptr(x), _ptr(nr), _ptr(bf), ctypes.byref(out)))
        self._keep[out.value] = (x, nr, bf)  # host buffers stay alive until the copy has run
        return out.value

    def neighbors(self, cloud: int, k: int, eps_factor: float, mode: int = KNN, cap: int | None = None,
                  targets=None, halfspace=None, k_per_target=None) -> int:
        tg = _contig(targets, torch.int32) if targets is not None else None
        hs = _contig(halfspace, torch.float64) if halfspace is not None else None
        kp = _contig(k_per_target, torch.int32) if k_per_target is not None else None
        nt = 0 if tg is None else tg.shape[0]
        if tg is not None and nt == 0:
            tg = torch.zeros(1, dtype=torch.int32)  # an empty list still needs a non-NULL pointer
        p = NbrParams(mode, k, eps_factor, cap if cap is not None else k, 0, _ptr(tg), nt, _ptr(hs), _ptr(kp))
        out = ctypes.c_int64()
        self._check(self.lib.gmls_neighbors(self.h, cloud, ctypes.byref(p), ctypes.byref(out)))
        self._keep[out.value] = (tg, hs, kp)
        return out.value

    def neighbors_prefix(self, nbrs: int, k: int, eps_factor: float) -> int:
        """k-nearest lists as prefixes of a longer k-nearest handle (gmls_neighbors_prefix)."""
        out = ctypes.c_int64()
        self._check(self.lib.gmls_neighbors_prefix(self.h, nbrs, k, eps_factor, ctypes.byref(out)))
        return out.value

    def stencils(self, nbrs: int, basis: int, degree: int, functionals, precision: int = FP64,
                 weight_power: int = 4, neumann: bool = False, max_refine: int = 0, refine_tol: float = 0.0,
                 degree_per_target=None) -> int:
        fs = (ctypes.c_int32 * 5)(*(list(functionals) + [0] * (5 - len(functionals))))
        dp = _contig(degree_per_target, torch.int8) if degree_per_target is not None else None
        p = StencilParams(basis, degree, WEIGHT_POLY, weight_power, precision, len(functionals), fs, int(neumann),
                          max_refine, refine_tol, _ptr(dp))
        out = ctypes.c_int64()
        self._check(self.lib.gmls_stencils(self.h, nbrs, ctypes.byref(p), ctypes.byref(out)))
        self._keep[out.value] = (dp,)
        return out.value

    def stencil_info(self, sid: int, functional: int):
        nt, vals = ctypes.c_int64(), ctypes.c_int64()
        rows, nc = ctypes.c_int32(), ctypes.c_int32()
        self._check(self.lib.gmls_stencil_info(self.h, sid, functional, ctypes.byref(nt), ctypes.byref(rows),
                                               ctypes.byref(nc), ctypes.byref(vals)))
        return nt.value, rows.value, nc.value, vals.value

    def export(self, hid: int, what: int, dtype, functional: int = 0, device=None):
        """Copy one array of a handle into a new tensor (device by default)."""
        nb = ctypes.c_size_t()
        self._check(self.lib.gmls_export_size(self.h, hid, what, functional, ctypes.byref(nb)))
        esz = torch.tensor([], dtype=dtype).element_size()
        dev = self.device if device is None else torch.device(device)
        out = torch.empty(nb.value // esz, dtype=dtype, device=dev, pin_memory=False)
        if nb.value:
            self._check(self.lib.gmls_export(self.h, hid, what, functional, _ptr(out), nb.value))
        return out

    def weights(self, sid: int, functional: int, device=None):
        return self.export(sid, X_WEIGHTS, torch.float64, functional, device)

    def csr_size(self, sid: int, functional: int):
        r, c, z = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        self._check(self.lib.gmls_csr_size(self.h, sid, functional, ctypes.byref(r), ctypes.byref(c),
                                           ctypes.byref(z)))
        return r.value, c.value, z.value

    def assemble_csr(self, sid: int, functional: int, out=None, nnz_offset: int = 0):
        """CSR of one operator into torch device tensors (row_ptr, col, val);
        with nnz_offset, the rows of a target range of a larger operator
        (gmls_assemble_csr_at: out = views at the range's first row / nonzero)."""
        if out is None:
            nr, _, nnz = self.csr_size(sid, functional)
            out = (torch.empty(nr + 1, dtype=torch.int64, device=self.device),
                   torch.empty(max(nnz, 1), dtype=torch.int32, device=self.device),
                   torch.empty(max(nnz, 1), dtype=torch.float64, device=self.device))
        rp, col, val = out
        self._check(self.lib.gmls_assemble_csr_at(self.h, sid, functional, nnz_offset, _ptr(rp), _ptr(col),
                                                  _ptr(val)))
        return out

    # ------------------------------------------------------- Stokes system
    def stokes_size(self, velocity: int, pressure: int, nu: float, pressure_interior: int = 0):
        """(n_rows, nnz) of the collocation system (gmls_stokes_size);
        pressure_interior: 0, or staggered Laplacian stencils for the interior
        pressure rows."""
        p = StokesParams(velocity, pressure, nu, pressure_interior)
        r, z = ctypes.c_int64(), ctypes.c_int64()
        self._check(self.lib.gmls_stokes_size(self.h, ctypes.byref(p), ctypes.byref(r), ctypes.byref(z)))
        return r.value, z.value

    def stokes_assemble(self, velocity: int, pressure: int, nu: float, pressure_interior: int = 0):
        """The collocation system as device CSR tensors (row_ptr, col, val)."""
        nr, nnz = self.stokes_size(velocity, pressure, nu, pressure_interior)
        rp = torch.empty(nr + 1, dtype=torch.int64, device=self.device)
        col = torch.empty(max(nnz, 1), dtype=torch.int32, device=self.device)
        val = torch.empty(max(nnz, 1), dtype=torch.float64, device=self.device)
        p = StokesParams(velocity, pressure, nu, pressure_interior)
        self._check(self.lib.gmls_stokes_assemble(self.h, ctypes.byref(p), _ptr(rp), _ptr(col), _ptr(val)))
        return rp, col, val

    def stokes_rhs(self, velocity: int, pressure: int, nu: float, f, w, div_f):
        """Right-hand side b (device) from f, w ([dim, n]) and div f ([n])."""
        f, w, div_f = (_contig(a, torch.float64).to(self.device) for a in (f, w, div_f))
        n = div_f.shape[0]
        b = torch.empty(f.shape[0] * n + n + 1, dtype=torch.float64, device=self.device)
        p = StokesParams(velocity, pressure, nu)
        self._check(self.lib.gmls_stokes_rhs(self.h, ctypes.byref(p), _ptr(f), _ptr(w), _ptr(div_f), _ptr(b)))
        for a in (f, w, div_f, b):
            a.record_stream(self.stream)  # in use on the context stream until its kernels have run
        return b

    def spmv(self, row_ptr, col, val, x):
        """y = A x (gmls_csr_spmv), device tensors."""
        x = _contig(x, torch.float64).to(self.device)
        n_rows = row_ptr.shape[0] - 1
        y = torch.empty(n_rows, dtype=torch.float64, device=self.device)
        self._check(self.lib.gmls_csr_spmv(self.h, n_rows, _ptr(row_ptr), _ptr(col), _ptr(val), _ptr(x), _ptr(y)))
        for a in (row_ptr, col, val, x, y):
            a.record_stream(self.stream)
        return y

    def gmres(self, row_ptr, col, val, b, x0=None, restart: int = 60, max_iter: int = 5000, rtol: float = 1e-10,
              row_scaling: bool = False):
        """Solve A x = b (gmls_gmres); returns (x, iterations, relative
        residual).  row_scaling: GMRES on the row-equilibrated system (the
        residual is then that of the scaled rows)."""
        b = _contig(b, torch.float64).to(self.device)
        n = row_ptr.shape[0] - 1
        x = (torch.zeros(n, dtype=torch.float64, device=self.device) if x0 is None
             else _contig(x0, torch.float64).to(self.device).clone())
        p = GmresParams(restart, max_iter, rtol, int(row_scaling))
        it, rel = ctypes.c_int32(), ctypes.c_double()
        self._check(self.lib.gmls_gmres(self.h, n, _ptr(row_ptr), _ptr(col), _ptr(val), _ptr(b), _ptr(x),
                                        ctypes.byref(p), ctypes.byref(it), ctypes.byref(rel)))
        return x, it.value, rel.value

    def release(self, hid: int):
        self._check(self.lib.gmls_release(self.h, hid))
        self._keep.pop(hid, None)

    def sync(self):
        self._check(self.lib.gmls_sync(self.h))

    def arena_usage(self):
        u, p, c = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_size_t()
        self._check(self.lib.gmls_arena_usage(self.h, ctypes.byref(u), ctypes.byref(p), ctypes.byref(c)))
        return u.value, p.value, c.value

    def set_option(self, option: int, value: int):
        self._check(self.lib.gmls_set_option(self.h, option, value))

    def tune_log(self):
        """The autotuner's timings: list of dicts (shape, variant, ms)."""
        out = []
        f = (ctypes.c_int32 * 9)()
        ms = ctypes.c_float()
        i = 0
        while self.lib.gmls_tune_info(self.h, i, f, ctypes.byref(ms)) == OK:
            keys = ["basis", "dim", "degree", "precision", "rows", "solve_rows", "neumann", "bucketed", "variant"]
            out.append(dict(zip(keys, list(f)), ms=ms.value))
            i += 1
        return out

    def capture_begin(self):
        self._check(self.lib.gmls_capture_begin(self.h))

    def capture_end(self) -> int:
        out = ctypes.c_int64()
        self._check(self.lib.gmls_capture_end(self.h, ctypes.byref(out)))
        return out.value

    def graph_launch(self, graph: int):
        self._check(self.lib.gmls_graph_launch(self.h, graph))

    def launch_count(self) -> int:
        v = ctypes.c_int64()
        self._check(self.lib.gmls_launch_count(self.h, ctypes.byref(v)))
        return v.value


def _contig(a, dtype):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        a = torch.from_numpy(np.ascontiguousarray(a))
    if a.dtype != dtype:
        a = a.to(dtype)
    return a.contiguous()


class Server:
    """Continuous-batching stencil server (gmls_server_*) over a torch-allocated arena."""

    def __init__(self, device: int = 0, arena_bytes: int = 16 << 30, streams: int = 4, max_inflight: int = 8):
        self.lib = load()
        self.arena = torch.empty(arena_bytes, dtype=torch.uint8, device=torch.device("cuda", device))
        h = ctypes.c_void_p()
        rc = self.lib.gmls_server_create(ctypes.byref(h), device, _ptr(self.arena), arena_bytes, streams, max_inflight)
        if rc != OK:
            raise GmlsError(rc, self.lib.gmls_last_error(None).decode())
        self.h = h

    def submit(self, x, basis: int, degree: int, k: int, functionals, precision: int = FP32_REFINE,
               eps_factor: float = 1.5) -> int:
        x = np.ascontiguousarray(x, dtype=np.float64)
        fs = (ctypes.c_int32 * 5)(*(list(functionals) + [0] * (5 - len(functionals))))
        r = Request(x.shape[0], x.shape[1], ctypes.c_void_p(x.ctypes.data), basis, degree, k, eps_factor, precision,
                    len(functionals), fs)
        t = ctypes.c_int64()
        rc = self.lib.gmls_server_submit(self.h, ctypes.byref(r), ctypes.byref(t))
        if rc != OK:
            raise GmlsError(rc, "gmls_server_submit rejected the request")
        return t.value

    def wait(self, ticket: int, timeout_ms: int = 60000) -> bool:
        done = ctypes.c_int32()
        rc = self.lib.gmls_server_wait(self.h, ticket, timeout_ms, ctypes.byref(done))
        if rc != OK:
            raise GmlsError(rc, f"request {ticket} failed")
        return bool(done.value)

    def result(self, ticket: int, what: int, dtype, functional: int = 0):
        need = ctypes.c_size_t()
        rc = self.lib.gmls_server_result(self.h, ticket, what, functional, None, 0, ctypes.byref(need))
        if rc != OK:
            raise GmlsError(rc, f"result of request {ticket}")
        esz = torch.tensor([], dtype=dtype).element_size()
        out = torch.empty(need.value // esz, dtype=dtype)
        rc = self.lib.gmls_server_result(self.h, ticket, what, functional, _ptr(out), need.value, None)
        if rc != OK:
            raise GmlsError(rc, f"result of request {ticket}")
        return out

    def cancel(self, ticket: int) -> int:
        """Cancel a request still waiting for admission: returns OK, or EBUSY
        once it was admitted or finished (no exception: both are normal)."""
        rc = self.lib.gmls_server_cancel(self.h, ticket)
        if rc not in (OK, EBUSY):
            raise GmlsError(rc, f"cancel of request {ticket}")
        return rc

    def release(self, ticket: int):
        rc = self.lib.gmls_server_release(self.h, ticket)
        if rc != OK:
            raise GmlsError(rc, f"release of request {ticket}")

    def stats(self) -> dict:
        st = ServerStats()
        self.lib.gmls_server_stats(self.h, ctypes.byref(st))
        return {f: getattr(st, f) for f, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "h", None):
            self.lib.gmls_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
