"""ctypes binding of the C ABI in ``include/sem.h``.

Argument marshalling only: every computation runs in the CUDA library
``_build/libsem.so``.  Device vectors are torch CUDA tensors (the binding
passes their data pointers); streams are torch CUDA streams (their raw
``cudaStream_t``).  Importing this module does not load the library; the first
call does, and raises if it was not built (there is no fallback path).
"""

from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsem.so")

SEM_OK, SEM_EINVAL, SEM_ENOMEM, SEM_ECUDA, SEM_ENOTCONV, SEM_ENUMERIC, SEM_EAGAIN, SEM_EBUSY, \
    SEM_ETIMEOUT = range(9)
STATUS_NAMES = ["SEM_OK", "SEM_EINVAL", "SEM_ENOMEM", "SEM_ECUDA", "SEM_ENOTCONV", "SEM_ENUMERIC",
                "SEM_EAGAIN", "SEM_EBUSY", "SEM_ETIMEOUT"]
SEM_F64, SEM_F32, SEM_F16, SEM_BF16 = range(4)
SEM_DIRICHLET, SEM_NEUMANN = 0, 1
SEM_GEOM_STORED, SEM_GEOM_TRILINEAR = 0, 1
SEM_ARITH_PAIR, SEM_ARITH_NATIVE = 0, 1
SEM_AX_LOCAL, SEM_AX_ASSEMBLED = 0, 1
SEM_FIELD_X, SEM_FIELD_Y, SEM_FIELD_Z, SEM_FIELD_MASS, SEM_FIELD_MULT, SEM_FIELD_MASK, \
    SEM_FIELD_DINV = range(7)
SEM_SOLVER_PCG, SEM_SOLVER_FLEXCG, SEM_SOLVER_FGMRES = 0, 1, 2
SEM_COARSE_JACOBI, SEM_COARSE_MG = 0, 1
SEM_RHS_HOST, SEM_RHS_MANUFACTURED = 0, 1
SEM_SMOOTH_JACOBI, SEM_SMOOTH_ASM, SEM_SMOOTH_ASM_TC, SEM_SMOOTH_ASM_TF32 = 0, 1, 2, 3
SEM_EAGAIN, SEM_EBUSY = 6, 7
SEM_MAX_ORDER = 11

EXPORTED = ["sem_mesh_create", "sem_mesh_destroy", "sem_mesh_info", "sem_mesh_field", "sem_ax",
            "sem_gs", "sem_dot", "sem_pmg_setup", "sem_pmg_destroy", "sem_pmg_info",
            "sem_pmg_vcycle", "sem_pmg_coarse_iters", "sem_solve", "sem_solve_host", "sem_trace_enable",
            "sem_trace_read", "sem_dot_noalloc", "sem_proj_create", "sem_proj_destroy",
            "sem_proj_info", "sem_solve_projected", "sem_server_create", "sem_server_destroy",
            "sem_submit", "sem_poll", "sem_server_stats_read", "sem_server_autotune",
            "sem_inject_wait_error", "sem_inject_alloc_failure", "sem_batch_create",
            "sem_batch_solve", "sem_batch_info", "sem_batch_pmg_desc", "sem_batch_x",
            "sem_batch_destroy", "sem_batch_autotune", "sem_pmg_coarse_solve",
            "sem_last_error"]


class SemError(RuntimeError):
    def __init__(self, status, msg):
        self.status = status
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 9 else status}: {msg}")


class sem_mesh_desc(C.Structure):
    _fields_ = [("ex", C.c_int32), ("ey", C.c_int32), ("ez", C.c_int32), ("N", C.c_int32),
                ("jitter", C.c_double), ("seed", C.c_uint64), ("bc", C.c_int32),
                ("geom", C.c_int32), ("verts", C.c_void_p), ("f64_arith", C.c_int32)]


class sem_pmg_desc(C.Structure):
    _fields_ = [("nlevels", C.c_int32), ("orders", C.c_int32 * 8), ("cheb_degree", C.c_int32),
                ("lanczos_steps", C.c_int32), ("seed", C.c_uint64), ("smoother_dtype", C.c_int32),
                ("coarse_tol", C.c_double), ("coarse_maxit", C.c_int32),
                ("coarse_mode", C.c_int32), ("smoother", C.c_int32), ("coarse_ctas", C.c_int32)]


class sem_solve_desc(C.Structure):
    _fields_ = [("solver", C.c_int32), ("tol", C.c_double), ("max_iter", C.c_int32),
                ("check_every", C.c_int32), ("restart", C.c_int32), ("use_graph", C.c_int32),
                ("zero_guess", C.c_int32)]


class sem_server_desc(C.Structure):
    _fields_ = [("workers", C.c_int32), ("hbm_budget", C.c_int64), ("cache_per_shape", C.c_int32),
                ("cheb_degree", C.c_int32), ("smoother_dtype", C.c_int32),
                ("coarse_tol", C.c_double), ("coarse_maxit", C.c_int32)]


class sem_request(C.Structure):
    _fields_ = [("ex", C.c_int32), ("ey", C.c_int32), ("ez", C.c_int32), ("N", C.c_int32),
                ("bc", C.c_int32), ("jitter", C.c_double), ("seed", C.c_uint64),
                ("rhs", C.c_int32), ("b", C.c_void_p), ("x", C.c_void_p),
                ("solve", sem_solve_desc)]


class sem_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64),
                ("setups_built", C.c_int64), ("setups_reused", C.c_int64),
                ("hbm_in_use", C.c_int64)]


class sem_batch_desc(C.Structure):
    _fields_ = [("cheb_degree", C.c_int32), ("smoother_dtype", C.c_int32),
                ("coarse_tol", C.c_double), ("coarse_maxit", C.c_int32),
                ("coarse_ctas", C.c_int32), ("ax_fill", C.c_float * (SEM_MAX_ORDER + 1)),
                ("arena_chunk", C.c_int64)]


class sem_trace_entry(C.Structure):
    _fields_ = [("name", C.c_char * 48), ("launches", C.c_int64), ("timed", C.c_int64),
                ("total_ms", C.c_double)]


class sem_solve_info(C.Structure):
    _fields_ = [("iters", C.c_int32), ("status", C.c_int32), ("res0", C.c_double),
                ("res", C.c_double), ("bnorm", C.c_double), ("time_ms", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib():
    """Load libsem.so (raises when it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                           "(run paper_2110_01716_gb300.build.build())")
    L = C.CDLL(LIB_PATH)
    vp, i32, i64, d = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    L.sem_last_error.restype = C.c_char_p
    L.sem_mesh_create.argtypes = [C.POINTER(sem_mesh_desc), vp, C.POINTER(vp)]
    L.sem_mesh_destroy.argtypes = [vp]
    L.sem_mesh_info.argtypes = [vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(C.c_size_t)]
    L.sem_mesh_field.argtypes = [vp, i32, vp, vp]
    L.sem_inject_wait_error.argtypes = [vp, vp]
    L.sem_inject_alloc_failure.argtypes = [i32]
    L.sem_ax.argtypes = [vp, i32, vp, vp, i32, vp]
    L.sem_gs.argtypes = [vp, i32, vp, vp]
    L.sem_dot.argtypes = [vp, vp, vp, C.POINTER(d), vp]
    L.sem_dot_noalloc.argtypes = [vp, vp, vp, vp, vp]
    L.sem_pmg_setup.argtypes = [vp, C.POINTER(sem_pmg_desc), vp, C.POINTER(vp)]
    L.sem_pmg_destroy.argtypes = [vp]
    L.sem_pmg_info.argtypes = [vp, i32, C.POINTER(d), C.POINTER(d)]
    L.sem_pmg_vcycle.argtypes = [vp, vp, vp, vp]
    L.sem_pmg_coarse_solve.argtypes = [vp, vp, vp, vp]
    L.sem_pmg_coarse_iters.argtypes = [vp, vp, C.POINTER(i32)]
    L.sem_solve.argtypes = [vp, vp, vp, vp, C.POINTER(sem_solve_desc), C.POINTER(sem_solve_info),
                            vp]
    L.sem_solve_host.argtypes = L.sem_solve.argtypes
    L.sem_proj_create.argtypes = [vp, i32, vp, C.POINTER(vp)]
    L.sem_proj_destroy.argtypes = [vp]
    L.sem_proj_info.argtypes = [vp, C.POINTER(i32)]
    L.sem_solve_projected.argtypes = [vp, vp, vp, vp, vp, C.POINTER(sem_solve_desc),
                                      C.POINTER(sem_solve_info), vp]
    L.sem_server_create.argtypes = [C.POINTER(sem_server_desc), C.POINTER(vp)]
    L.sem_server_destroy.argtypes = [vp]
    L.sem_submit.argtypes = [vp, C.POINTER(sem_request), C.POINTER(C.c_uint64)]
    L.sem_poll.argtypes = [vp, C.c_uint64, C.POINTER(sem_solve_info)]
    L.sem_server_stats_read.argtypes = [vp, C.POINTER(sem_server_stats)]
    L.sem_server_autotune.argtypes = [C.POINTER(sem_server_desc), C.POINTER(sem_request), i32, i32,
                                      C.POINTER(i32), C.POINTER(d)]
    L.sem_batch_create.argtypes = [C.POINTER(sem_batch_desc), C.POINTER(sem_request), i32, vp,
                                   C.POINTER(vp)]
    L.sem_batch_solve.argtypes = [vp, C.POINTER(sem_solve_info), vp]
    L.sem_batch_info.argtypes = [vp, C.POINTER(C.c_size_t), C.POINTER(i32), C.POINTER(d)]
    L.sem_batch_pmg_desc.argtypes = [vp, i32, C.POINTER(sem_pmg_desc)]
    L.sem_batch_x.argtypes = [vp, i32, C.POINTER(vp)]
    L.sem_batch_destroy.argtypes = [vp]
    L.sem_batch_autotune.argtypes = [vp, C.POINTER(C.c_float), i32, i32, vp,
                                     C.POINTER(C.c_float), C.POINTER(d)]
    L.sem_trace_enable.argtypes = [i32, C.c_char_p]
    L.sem_trace_read.argtypes = [C.POINTER(sem_trace_entry), i32, C.POINTER(i32), i32]
    for name in EXPORTED:
        if name != "sem_last_error":
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def last_error() -> str:
    return lib().sem_last_error().decode()


def check(status: int):
    if status != SEM_OK:
        raise SemError(status, last_error())
    return status


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        import torch

        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ---------------------------------------------------------------- handles
class Mesh:
    """Owning wrapper of a sem_mesh handle."""

    def __init__(self, ex, ey, ez, N, bc=SEM_DIRICHLET, geom=SEM_GEOM_STORED, verts=None,
                 jitter=0.1, seed=1, stream=None, f64_arith=SEM_ARITH_PAIR):
        import numpy as np

        self._verts = None
        vptr = None
        if verts is not None:
            self._verts = np.ascontiguousarray(verts, dtype=np.float64)
            vptr = self._verts.ctypes.data
        desc = sem_mesh_desc(ex, ey, ez, N, float(jitter), int(seed), bc, geom, vptr, f64_arith)
        h = C.c_void_p()
        check(lib().sem_mesh_create(C.byref(desc), _stream(stream), C.byref(h)))
        self.h = h
        self.ex, self.ey, self.ez, self.N, self.bc, self.geom = ex, ey, ez, N, bc, geom
        self.f64_arith = f64_arith
        nl, ng, nb = C.c_int64(), C.c_int64(), C.c_size_t()
        check(lib().sem_mesh_info(self.h, C.byref(nl), C.byref(ng), C.byref(nb)))
        self.n_local, self.n_global = nl.value, ng.value

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            lib().sem_mesh_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        nl, ng, nb = C.c_int64(), C.c_int64(), C.c_size_t()
        check(lib().sem_mesh_info(self.h, C.byref(nl), C.byref(ng), C.byref(nb)))
        return {"n_local": nl.value, "n_global": ng.value, "dev_bytes": nb.value}


def sem_mesh_field(mesh: Mesh, which: int, out, stream=None):
    check(lib().sem_mesh_field(mesh.h, which, _ptr(out), _stream(stream)))
    return out


def sem_inject_wait_error(mesh: Mesh, stream=None):
    """Test hook: set the fine level's wait-error flag from the host, so that
    the next solve on the mesh reports SEM_ETIMEOUT."""
    check(lib().sem_inject_wait_error(mesh.h, _stream(stream)))


def sem_inject_alloc_failure(after: int):
    """Test hook: make the after-th device allocation of the library from now
    on fail with SEM_ENOMEM (0 disarms)."""
    check(lib().sem_inject_alloc_failure(int(after)))


def sem_ax(mesh: Mesh, dtype: int, u, w, flags=SEM_AX_ASSEMBLED, stream=None):
    check(lib().sem_ax(mesh.h, dtype, _ptr(u), _ptr(w), flags, _stream(stream)))
    return w


def sem_gs(mesh: Mesh, dtype: int, u, stream=None):
    check(lib().sem_gs(mesh.h, dtype, _ptr(u), _stream(stream)))
    return u


def sem_dot(mesh: Mesh, u, v, stream=None) -> float:
    out = C.c_double()
    check(lib().sem_dot(mesh.h, _ptr(u), _ptr(v), C.byref(out), _stream(stream)))
    return out.value


def sem_dot_noalloc(mesh: Mesh, u, v, result, stream=None):
    """Unique-node inner product into ``result`` (a one-element device tensor)
    for callers that cannot have the library allocate; see include/sem.h."""
    for name, t in (("u", u), ("v", v)):
        if str(t.dtype) != "torch.float64" or not t.is_cuda or t.numel() < mesh.n_local:
            raise ValueError(f"{name} must be a float64 CUDA tensor of at least n_local "
                             f"= {mesh.n_local} values")
    if str(result.dtype) != "torch.float64" or not result.is_cuda or result.numel() < 1:
        raise ValueError("result must be a float64 CUDA tensor with at least one element")
    check(lib().sem_dot_noalloc(mesh.h, _ptr(u), _ptr(v), _ptr(result), _stream(stream)))
    return result


class Pmg:
    """Owning wrapper of a sem_pmg handle (keeps its mesh alive)."""

    def __init__(self, mesh: Mesh, orders=(7, 3, 1), cheb_degree=2, lanczos_steps=20, seed=0,
                 smoother_dtype=SEM_F32, coarse_tol=1e-2, coarse_maxit=50, stream=None,
                 coarse_mode=SEM_COARSE_JACOBI, smoother=SEM_SMOOTH_JACOBI, coarse_ctas=0):
        desc = sem_pmg_desc()
        desc.nlevels = len(orders)
        for i, o in enumerate(orders):
            desc.orders[i] = int(o)
        desc.cheb_degree = cheb_degree
        desc.lanczos_steps = lanczos_steps
        desc.seed = int(seed)
        desc.smoother_dtype = smoother_dtype
        desc.coarse_tol = float(coarse_tol)
        desc.coarse_maxit = int(coarse_maxit)
        desc.coarse_mode = int(coarse_mode)
        desc.smoother = int(smoother)
        desc.coarse_ctas = int(coarse_ctas)
        h = C.c_void_p()
        check(lib().sem_pmg_setup(mesh.h, C.byref(desc), _stream(stream), C.byref(h)))
        self.h = h
        self.mesh = mesh
        self.orders = tuple(orders)

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            lib().sem_pmg_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def coarse_iters(self, stream=None):
        """Iterations of the coarsest-level solver in the last V-cycle."""
        it = C.c_int32()
        check(lib().sem_pmg_coarse_iters(self.h, _stream(stream), C.byref(it)))
        return it.value

    def lam(self, level):
        lo, hi = C.c_double(), C.c_double()
        check(lib().sem_pmg_info(self.h, level, C.byref(lo), C.byref(hi)))
        return lo.value, hi.value


def sem_pmg_coarse_solve(pmg: Pmg, b, x, stream=None):
    """The coarsest level's solve alone (b, x: that level's E-layout vectors)."""
    check(lib().sem_pmg_coarse_solve(pmg.h, _ptr(b), _ptr(x), _stream(stream)))
    return x


def sem_pmg_vcycle(pmg: Pmg, r, z, stream=None):
    check(lib().sem_pmg_vcycle(pmg.h, _ptr(r), _ptr(z), _stream(stream)))
    return z


def sem_solve(mesh: Mesh, pmg, b, x, solver=SEM_SOLVER_PCG, tol=1e-8, max_iter=1000,
              check_every=1, stream=None, raise_on_notconv=False, restart=0, use_graph=False,
              zero_guess=False):
    """Solve in place (x: initial guess in, solution out; with zero_guess the
    guess is 0 and x is output only); returns the info dict."""
    desc = sem_solve_desc(solver, float(tol), int(max_iter), int(check_every), int(restart),
                          int(bool(use_graph)), int(bool(zero_guess)))
    info = sem_solve_info()
    st = lib().sem_solve(mesh.h, pmg.h if pmg is not None else None, _ptr(b), _ptr(x),
                         C.byref(desc), C.byref(info), _stream(stream))
    if st not in (SEM_OK, SEM_ENOTCONV) or (raise_on_notconv and st != SEM_OK):
        raise SemError(st, last_error())
    d = info.as_dict()
    d["status"] = st
    return d


def sem_solve_host(mesh: Mesh, pmg, b_host, x_host, solver=SEM_SOLVER_PCG, tol=1e-8,
                   max_iter=1000, check_every=1, stream=None, restart=0, use_graph=False,
                   zero_guess=False):
    """As sem_solve with host (CPU tensor or numpy) b and x; x is updated in place
    (with zero_guess its input is not read or copied)."""
    desc = sem_solve_desc(solver, float(tol), int(max_iter), int(check_every), int(restart),
                          int(bool(use_graph)), int(bool(zero_guess)))
    info = sem_solve_info()
    bp = b_host.ctypes.data if hasattr(b_host, "ctypes") else b_host.data_ptr()
    xp = x_host.ctypes.data if hasattr(x_host, "ctypes") else x_host.data_ptr()
    st = lib().sem_solve_host(mesh.h, pmg.h if pmg is not None else None, bp, xp, C.byref(desc),
                              C.byref(info), _stream(stream))
    if st not in (SEM_OK, SEM_ENOTCONV):
        raise SemError(st, last_error())
    d = info.as_dict()
    d["status"] = st
    return d


class Projection:
    """sem_proj handle: projection onto previous solutions (Lmax vectors)."""

    def __init__(self, mesh: "Mesh", Lmax: int, stream=None):
        self.mesh = mesh
        h = C.c_void_p()
        check(lib().sem_proj_create(mesh.h, int(Lmax), _stream(stream), C.byref(h)))
        self.h = h

    @property
    def nvec(self) -> int:
        n = C.c_int32()
        check(lib().sem_proj_info(self.h, C.byref(n)))
        return n.value

    def close(self):
        if getattr(self, "h", None):
            lib().sem_proj_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sem_solve_projected(mesh: Mesh, pmg, proj: Projection, b, x, solver=SEM_SOLVER_FLEXCG,
                        tol=1e-8, max_iter=1000, check_every=1, restart=0, stream=None,
                        use_graph=False):
    """Projected solve: x (output) = best fit in the kept space + correction;
    returns the info dict (res0 = residual after projection)."""
    desc = sem_solve_desc(solver, float(tol), int(max_iter), int(check_every), int(restart),
                          int(bool(use_graph)))
    info = sem_solve_info()
    st = lib().sem_solve_projected(mesh.h, pmg.h if pmg is not None else None, proj.h, _ptr(b),
                                   _ptr(x), C.byref(desc), C.byref(info), _stream(stream))
    if st not in (SEM_OK, SEM_ENOTCONV):
        raise SemError(st, last_error())
    d = info.as_dict()
    d["status"] = st
    return d


def make_request(ex, ey, ez, N, bc=SEM_DIRICHLET, jitter=0.1, seed=0, b=None, x=None,
                 solver=SEM_SOLVER_FLEXCG, tol=1e-8, max_iter=200, restart=0, use_graph=False):
    """A sem_request; b (host float64 array, n_local) selects SEM_RHS_HOST, else the
    manufactured right-hand side; x (host float64 array) receives the solution."""
    r = sem_request()
    r.ex, r.ey, r.ez, r.N, r.bc = ex, ey, ez, N, bc
    r.jitter, r.seed = float(jitter), int(seed)
    r.rhs = SEM_RHS_MANUFACTURED if b is None else SEM_RHS_HOST
    r.b = b.ctypes.data if b is not None else None
    r.x = x.ctypes.data if x is not None else None
    r.solve = sem_solve_desc(solver, float(tol), int(max_iter), 1, int(restart),
                             int(bool(use_graph)))
    return r


def server_desc(workers=4, hbm_budget=0, cache_per_shape=1, cheb_degree=3,
                smoother_dtype=SEM_F32, coarse_tol=1e-1, coarse_maxit=30):
    return sem_server_desc(int(workers), int(hbm_budget), int(cache_per_shape), int(cheb_degree),
                           int(smoother_dtype), float(coarse_tol), int(coarse_maxit))


class Server:
    """Continuous-batching server of independent solves (sem_server)."""

    def __init__(self, **kw):
        self.desc = server_desc(**kw)
        h = C.c_void_p()
        check(lib().sem_server_create(C.byref(self.desc), C.byref(h)))
        self.h = h
        self._keep = {}

    def submit(self, *args, **kw):
        """Arguments of make_request; returns the ticket.  Host arrays given as
        b and x are kept alive until the request is polled."""
        r = make_request(*args, **kw)
        t = C.c_uint64()
        check(lib().sem_submit(self.h, C.byref(r), C.byref(t)))
        self._keep[t.value] = (kw.get("b"), kw.get("x"))
        return t.value

    def poll(self, ticket):
        """The info dict when done (the ticket is then released), else None."""
        info = sem_solve_info()
        st = lib().sem_poll(self.h, C.c_uint64(ticket), C.byref(info))
        if st == SEM_EAGAIN:
            return None
        check(st)
        self._keep.pop(ticket, None)
        return info.as_dict()

    def wait(self, ticket, sleep=0.0005):
        import time as _time

        while True:
            d = self.poll(ticket)
            if d is not None:
                return d
            _time.sleep(sleep)

    def stats(self):
        s = sem_server_stats()
        check(lib().sem_server_stats_read(self.h, C.byref(s)))
        return {k: getattr(s, k) for k, _ in s._fields_}

    def close(self):
        if getattr(self, "h", None):
            lib().sem_server_destroy(self.h)
            self.h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def server_autotune(requests, max_workers=16, **desc_kw):
    """Fastest worker count for a sample batch: (workers, solves per second)."""
    arr = (sem_request * len(requests))(*requests)
    w, rate = C.c_int32(), C.c_double()
    check(lib().sem_server_autotune(C.byref(server_desc(**desc_kw)), arr, len(requests),
                                    int(max_workers), C.byref(w), C.byref(rate)))
    return w.value, rate.value


class Batch:
    """Many independent FlexCG solves in one graph launch (sem_batch).
    requests: sem_request structures (make_request); host arrays they point
    to are kept alive with the batch."""

    def __init__(self, requests, cheb_degree=3, smoother_dtype=SEM_F32, coarse_tol=0.2,
                 coarse_maxit=30, coarse_ctas=1, ax_fill=None, arena_chunk=0, keep=(),
                 stream=None):
        d = sem_batch_desc()
        d.cheb_degree, d.smoother_dtype = int(cheb_degree), int(smoother_dtype)
        d.coarse_tol, d.coarse_maxit = float(coarse_tol), int(coarse_maxit)
        d.coarse_ctas, d.arena_chunk = int(coarse_ctas), int(arena_chunk)
        for o, f in (ax_fill or {}).items():
            d.ax_fill[int(o)] = float(f)
        self.n = len(requests)
        self._reqs = (sem_request * self.n)(*requests)
        self._keep = list(keep)
        h = C.c_void_p()
        check(lib().sem_batch_create(C.byref(d), self._reqs, self.n, _stream(stream),
                                     C.byref(h)))
        self.h = h

    def solve(self, stream=None, raise_on_fail=True):
        """One launch of the batch's graph: the list of info dicts."""
        infos = (sem_solve_info * self.n)()
        st = lib().sem_batch_solve(self.h, infos, _stream(stream))
        if raise_on_fail:
            check(st)
        return [i.as_dict() for i in infos]

    def info(self):
        b, nodes, ms = C.c_size_t(), C.c_int32(), C.c_double()
        check(lib().sem_batch_info(self.h, C.byref(b), C.byref(nodes), C.byref(ms)))
        return {"dev_bytes": b.value, "graph_nodes": nodes.value, "setup_ms": ms.value}

    def pmg_desc(self, i):
        d = sem_pmg_desc()
        check(lib().sem_batch_pmg_desc(self.h, int(i), C.byref(d)))
        return d

    def autotune(self, candidates=(4.0, 2.0, 1.0, 0.5, 0.25, 0.125), reps=3, stream=None):
        """Per-order work split of the FP32 operator: ({order: fill}, ms per launch)."""
        c = (C.c_float * len(candidates))(*candidates)
        out = (C.c_float * (SEM_MAX_ORDER + 1))()
        ms = C.c_double()
        check(lib().sem_batch_autotune(self.h, c, len(candidates), int(reps), _stream(stream),
                                       out, C.byref(ms)))
        return {o: out[o] for o in range(SEM_MAX_ORDER + 1) if out[o] > 0}, ms.value

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            lib().sem_batch_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pmg_from_desc(mesh: "Mesh", desc: "sem_pmg_desc", stream=None):
    """A Pmg built from a full sem_pmg_desc (e.g. Batch.pmg_desc(i))."""
    p = Pmg.__new__(Pmg)
    h = C.c_void_p()
    check(lib().sem_pmg_setup(mesh.h, C.byref(desc), _stream(stream), C.byref(h)))
    p.h, p.mesh = h, mesh
    p.orders = tuple(desc.orders[i] for i in range(desc.nlevels))
    return p


def sem_trace_enable(enable: bool, timed_filter: str = ""):
    check(lib().sem_trace_enable(int(bool(enable)), timed_filter.encode()))


def sem_trace_read(reset: bool = True):
    """{class name: {"launches", "timed", "total_ms"}} of the launches traced so far."""
    n = C.c_int32()
    check(lib().sem_trace_read(None, 0, C.byref(n), 0))
    arr = (sem_trace_entry * max(n.value, 1))()
    check(lib().sem_trace_read(arr, n.value, C.byref(n), int(bool(reset))))
    return {e.name.decode(): {"launches": e.launches, "timed": e.timed, "total_ms": e.total_ms}
            for e in arr[:n.value]}
