"""Python access to the FP64 CPU oracle (``sem_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg, never by the library.  ``build()`` compiles the C
file with gcc (no FMA contraction, so x86 and Arm give the same bits) into
``oracle/_build``; the wrappers below only marshal numpy arrays.  With
``SEM_ORACLE_LIB`` set, ``lib()`` loads that already built library instead
(the planted-mistake tests load altered copies of the oracle this way).
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sem_oracle.c")
_OUT = os.path.join(_HERE, "_build", "libsemoracle.so")
_lib = None

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")


def compile_to(src: str, out: str) -> str:
    """Compile the C source src into the shared object out (OpenMP when
    available), with the oracle's flags."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    base = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off", src, "-o",
            out + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(out + ".tmp", out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle into a shared object (OpenMP when available)."""
    if not force and os.path.exists(_OUT) and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC):
        return _OUT
    return compile_to(_SRC, _OUT)


def lib():
    global _lib
    if _lib is not None:
        return _lib
    L = C.CDLL(os.environ.get("SEM_ORACLE_LIB") or build())
    L.orc_splitmix64.argtypes = [C.c_uint64, C.c_uint64]
    L.orc_splitmix64.restype = C.c_uint64
    L.orc_legendre.argtypes = [C.c_int, C.c_double]
    L.orc_legendre.restype = C.c_double
    L.orc_gll.argtypes = [C.c_int, _dp, _dp]
    L.orc_dhat.argtypes = [C.c_int, _dp, _dp]
    L.orc_interp.argtypes = [C.c_int, _dp, C.c_int, _dp, _dp]
    L.orc_geometry.argtypes = [C.c_int] * 4 + [_dp, C.c_void_p, C.c_void_p, C.c_void_p]
    L.orc_global_ids.argtypes = [C.c_int] * 4 + [_ip]
    L.orc_mask.argtypes = [C.c_int] * 5 + [_dp]
    L.orc_ax_local.argtypes = [C.c_int64, C.c_int, _dp, _dp, _dp, _dp]
    L.orc_gs.argtypes = [C.c_int64, _ip, C.c_int64, _dp]
    L.orc_level_create.argtypes = [C.c_int] * 5 + [_dp]
    L.orc_level_create.restype = C.c_void_p
    L.orc_level_destroy.argtypes = [C.c_void_p]
    L.orc_level_nl.argtypes = [C.c_void_p]
    L.orc_level_nl.restype = C.c_int64
    L.orc_level_ng.argtypes = [C.c_void_p]
    L.orc_level_ng.restype = C.c_int64
    L.orc_level_copy.argtypes = [C.c_void_p, C.c_int, _dp]
    L.orc_level_ids.argtypes = [C.c_void_p, _ip]
    L.orc_level_ax.argtypes = [C.c_void_p, _dp, _dp]
    L.orc_level_gs.argtypes = [C.c_void_p, _dp]
    L.orc_level_dot.argtypes = [C.c_void_p, _dp, _dp]
    L.orc_level_dot.restype = C.c_double
    L.orc_level_diag.argtypes = [C.c_void_p, _dp]
    L.orc_pcg.argtypes = [C.c_void_p, _dp, _dp, C.c_double, C.c_int, C.c_int,
                          C.POINTER(C.c_int), C.POINTER(C.c_double), C.POINTER(C.c_double)]
    L.orc_cheb.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, _dp, _dp, _dp, C.c_int,
                           C.c_double, C.c_double, C.c_int]
    L.orc_cheb_m.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, _dp,
                             _dp, C.c_int, C.c_double, C.c_double, C.c_int]
    L.orc_level_lanczos_max.argtypes = [C.c_void_p, C.c_int, C.c_uint64, C.POINTER(C.c_int)]
    L.orc_lanczos_start.argtypes = [C.c_void_p, C.c_uint64, _dp]
    L.orc_level_lanczos_max.restype = C.c_double
    L.orc_pmg_create.argtypes = [C.c_int] * 4 + [_i32p, C.c_int, _dp, C.c_int, C.c_int,
                                                 C.c_uint64, C.c_double, C.c_int]
    L.orc_pmg_create.restype = C.c_void_p
    L.orc_pmg_destroy.argtypes = [C.c_void_p]
    L.orc_pmg_lambda.argtypes = [C.c_void_p, C.c_int, C.c_int]
    L.orc_pmg_lambda.restype = C.c_double
    L.orc_pmg_level.argtypes = [C.c_void_p, C.c_int]
    L.orc_pmg_level.restype = C.c_void_p
    L.orc_pmg_vcycle.argtypes = [C.c_void_p, _dp, _dp]
    L.orc_pmg_coarse_iters.argtypes = [C.c_void_p]
    L.orc_interp3.argtypes = [C.c_int64, C.c_int, C.c_int, _dp, _dp, _dp, C.c_int]
    L.orc_flexpcg.argtypes = [C.c_void_p, C.c_int, _dp, _dp, C.c_double, C.c_int,
                              C.POINTER(C.c_int), C.POINTER(C.c_double), C.POINTER(C.c_double)]
    L.orc_proj_create.argtypes = [C.c_void_p, C.c_int]
    L.orc_proj_create.restype = C.c_void_p
    L.orc_proj_destroy.argtypes = [C.c_void_p]
    L.orc_proj_nvec.argtypes = [C.c_void_p]
    L.orc_proj_vector.argtypes = [C.c_void_p, C.c_int, _dp, _dp]
    L.orc_solve_projected.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_int, _dp, _dp,
                                      C.c_double, C.c_int, C.POINTER(C.c_int),
                                      C.POINTER(C.c_double), C.POINTER(C.c_double)]
    L.orc_pmg_create2.argtypes = [C.c_int] * 4 + [_i32p, C.c_int, _dp, C.c_int, C.c_int,
                                                  C.c_uint64, C.c_double, C.c_int, C.c_int]
    L.orc_pmg_create2.restype = C.c_void_p
    L.orc_asm_create.argtypes = [C.c_void_p]
    L.orc_asm_create.restype = C.c_void_p
    L.orc_asm_destroy.argtypes = [C.c_void_p]
    L.orc_asm_apply.argtypes = [C.c_void_p, _dp, _dp]
    L.orc_asm_local_matrix.argtypes = [C.c_void_p, C.c_int64, _dp]
    L.orc_fgmres.argtypes = [C.c_void_p, C.c_int, _dp, _dp, C.c_double, C.c_int, C.c_int,
                             C.POINTER(C.c_int), C.POINTER(C.c_double), C.POINTER(C.c_double),
                             C.c_void_p]
    _lib = L
    return L


APPLY_FN = C.CFUNCTYPE(None, C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double))


# ---------------------------------------------------------------- 1D basis
def set_threads(n: int) -> int:
    """OpenMP threads of the oracle's parallel loops (the elements of the
    local operator); returns the count in force (1 without OpenMP)."""
    lib()
    try:
        gomp = C.CDLL("libgomp.so.1")
    except OSError:
        return 1
    gomp.omp_set_num_threads(int(n))
    return int(gomp.omp_get_max_threads())


def gll(N: int):
    x = np.zeros(N + 1)
    w = np.zeros(N + 1)
    if lib().orc_gll(N, x, w) != 0:
        raise ValueError("N must be >= 1")
    return x, w


def dhat(N: int) -> np.ndarray:
    x, _ = gll(N)
    D = np.zeros((N + 1) * (N + 1))
    lib().orc_dhat(N, x, D)
    return D.reshape(N + 1, N + 1)


def interp(Nf: int, Nc: int) -> np.ndarray:
    xf, _ = gll(Nf)
    xc, _ = gll(Nc)
    J = np.zeros((Nf + 1) * (Nc + 1))
    lib().orc_interp(Nf, xf, Nc, xc, J)
    return J.reshape(Nf + 1, Nc + 1)


def legendre(n: int, x: float) -> float:
    return lib().orc_legendre(n, x)


# ---------------------------------------------------------------- mesh
def geometry(ex, ey, ez, N, verts):
    """(G [E,6,Np^3], B [E,Np^3], X [E,3,Np^3]); raises on a folded element."""
    E = ex * ey * ez
    Np3 = (N + 1) ** 3
    G = np.zeros(E * 6 * Np3)
    B = np.zeros(E * Np3)
    X = np.zeros(E * 3 * Np3)
    v = np.ascontiguousarray(verts, dtype=np.float64).ravel()
    rc = lib().orc_geometry(ex, ey, ez, N, v, G.ctypes.data, B.ctypes.data, X.ctypes.data)
    if rc != 0:
        raise ValueError("non-positive Jacobian")
    return G.reshape(E, 6, Np3), B.reshape(E, Np3), X.reshape(E, 3, Np3)


def global_ids(ex, ey, ez, N) -> np.ndarray:
    ids = np.zeros(ex * ey * ez * (N + 1) ** 3, dtype=np.int64)
    lib().orc_global_ids(ex, ey, ez, N, ids)
    return ids


def mask(ex, ey, ez, N, bc) -> np.ndarray:
    m = np.zeros(ex * ey * ez * (N + 1) ** 3)
    lib().orc_mask(ex, ey, ez, N, bc, m)
    return m


def ax_local(N, D, G, u) -> np.ndarray:
    G = np.ascontiguousarray(G, dtype=np.float64).ravel()
    u = np.ascontiguousarray(u, dtype=np.float64).ravel()
    E = u.size // (N + 1) ** 3
    w = np.zeros_like(u)
    lib().orc_ax_local(E, N, np.ascontiguousarray(D, dtype=np.float64).ravel(), G, u, w)
    return w


def gs(ids, ng, u) -> np.ndarray:
    v = np.array(u, dtype=np.float64, copy=True).ravel()
    lib().orc_gs(v.size, np.ascontiguousarray(ids, dtype=np.int64), ng, v)
    return v


def interp3(E, nf, nc, J, u, transpose=False) -> np.ndarray:
    n_out = E * (nc if transpose else nf) ** 3
    out = np.zeros(n_out)
    lib().orc_interp3(E, nf, nc, np.ascontiguousarray(J, dtype=np.float64).ravel(),
                      np.ascontiguousarray(u, dtype=np.float64).ravel(), out, int(transpose))
    return out


def cheb(n, apply, dinv, b, x, k, lmin, lmax, x_zero):
    """Chebyshev smoothing with a Python operator ``apply(in) -> out``."""

    def _cb(_ctx, pin, pout):
        vin = np.ctypeslib.as_array(pin, shape=(n,))
        vout = np.ctypeslib.as_array(pout, shape=(n,))
        vout[:] = apply(vin.copy())

    cb = APPLY_FN(_cb)
    x = np.ascontiguousarray(x, dtype=np.float64).copy()
    lib().orc_cheb(n, C.cast(cb, C.c_void_p), None, np.ascontiguousarray(dinv, dtype=np.float64),
                   np.ascontiguousarray(b, dtype=np.float64), x, k, lmin, lmax, int(x_zero))
    return x


def cheb_m(n, apply, prec, b, x, k, lmin, lmax, x_zero):
    """Chebyshev smoothing on M A with Python operators ``apply(in) -> out``
    (A) and ``prec(in) -> out`` (M), the form the Schwarz smoother uses."""

    def wrap(f):
        def _cb(_ctx, pin, pout):
            vin = np.ctypeslib.as_array(pin, shape=(n,))
            vout = np.ctypeslib.as_array(pout, shape=(n,))
            vout[:] = f(vin.copy())

        return APPLY_FN(_cb)

    ca, cm = wrap(apply), wrap(prec)
    x = np.ascontiguousarray(x, dtype=np.float64).copy()
    lib().orc_cheb_m(n, C.cast(ca, C.c_void_p), None, C.cast(cm, C.c_void_p), None,
                     np.ascontiguousarray(b, dtype=np.float64), x, k, lmin, lmax, int(x_zero))
    return x


# ---------------------------------------------------------------- levels
class Level:
    """One discretisation level (mesh, operator, unique-dof inner product)."""

    DIRICHLET, NEUMANN = 0, 1

    def __init__(self, ex, ey, ez, N, bc, verts, _ptr=None, _owner=None):
        self.ex, self.ey, self.ez, self.N, self.bc = ex, ey, ez, N, bc
        self._owner = _owner
        if _ptr is None:
            v = np.ascontiguousarray(verts, dtype=np.float64).ravel()
            _ptr = lib().orc_level_create(ex, ey, ez, N, bc, v)
            if not _ptr:
                raise ValueError("oracle level creation failed (bad sizes or folded element)")
        self.ptr = _ptr
        self.E = ex * ey * ez
        self.Np = N + 1
        self.nl = lib().orc_level_nl(self.ptr)
        self.ng = lib().orc_level_ng(self.ptr)

    def __del__(self):
        if getattr(self, "_owner", None) is None and getattr(self, "ptr", None):
            lib().orc_level_destroy(self.ptr)
            self.ptr = None

    def _get(self, what, size):
        out = np.zeros(size)
        lib().orc_level_copy(self.ptr, what, out)
        return out

    @property
    def mult(self):
        return self._get(0, self.nl)

    @property
    def mask(self):
        return self._get(1, self.nl)

    @property
    def dinv(self):
        return self._get(2, self.nl)

    @property
    def B(self):
        return self._get(3, self.nl)

    @property
    def X(self):
        return self._get(4, 3 * self.nl).reshape(self.E, 3, self.Np ** 3)

    @property
    def G(self):
        return self._get(5, 6 * self.nl).reshape(self.E, 6, self.Np ** 3)

    @property
    def D(self):
        return self._get(6, self.Np * self.Np).reshape(self.Np, self.Np)

    @property
    def ids(self):
        out = np.zeros(self.nl, dtype=np.int64)
        lib().orc_level_ids(self.ptr, out)
        return out

    def ax(self, u):
        w = np.zeros(self.nl)
        lib().orc_level_ax(self.ptr, np.ascontiguousarray(u, dtype=np.float64), w)
        return w

    def ax_local(self, u):
        return ax_local(self.N, self.D, self.G, u)

    def gs(self, u):
        v = np.array(u, dtype=np.float64, copy=True)
        lib().orc_level_gs(self.ptr, v)
        return v

    def dot(self, u, v):
        return lib().orc_level_dot(self.ptr, np.ascontiguousarray(u, dtype=np.float64),
                                   np.ascontiguousarray(v, dtype=np.float64))

    def diag(self):
        d = np.zeros(self.nl)
        lib().orc_level_diag(self.ptr, d)
        return d

    def pcg(self, b, x0=None, tol=1e-10, maxit=1000, precond=True):
        x = np.zeros(self.nl) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
        it, r0, r1 = C.c_int(), C.c_double(), C.c_double()
        st = lib().orc_pcg(self.ptr, np.ascontiguousarray(b, dtype=np.float64), x, tol, maxit,
                           int(precond), C.byref(it), C.byref(r0), C.byref(r1))
        return x, {"status": st, "iters": it.value, "res0": r0.value, "res": r1.value}

    def lanczos_start(self, seed=0):
        v = np.zeros(self.nl)
        lib().orc_lanczos_start(self.ptr, seed, v)
        return v

    def lanczos_max(self, m=20, seed=0):
        steps = C.c_int()
        lam = lib().orc_level_lanczos_max(self.ptr, m, seed, C.byref(steps))
        return lam, steps.value

    def assembled_rhs(self, f_values):
        """b = mask * gs(B f) for f given at the local points."""
        return self.gs(self.B * f_values) * self.mask


class PMG:
    """p-multigrid hierarchy with Chebyshev-Jacobi smoothing (all FP64)."""

    def __init__(self, ex, ey, ez, orders, bc, verts, cheb_degree=2, lanczos_steps=20, seed=0,
                 coarse_tol=1e-2, coarse_maxit=50, smoother="jacobi"):
        Ns = np.ascontiguousarray(orders, dtype=np.int32)
        v = np.ascontiguousarray(verts, dtype=np.float64).ravel()
        self.ptr = lib().orc_pmg_create2(ex, ey, ez, len(orders), Ns, bc, v, cheb_degree,
                                         lanczos_steps, seed, coarse_tol, coarse_maxit,
                                         {"jacobi": 0, "asm": 1}[smoother])
        if not self.ptr:
            raise ValueError("oracle pMG creation failed")
        self.orders = list(orders)
        self.levels = [Level(ex, ey, ez, N, bc, None, _ptr=lib().orc_pmg_level(self.ptr, l),
                             _owner=self) for l, N in enumerate(orders)]

    def __del__(self):
        if getattr(self, "ptr", None):
            lib().orc_pmg_destroy(self.ptr)
            self.ptr = None

    def lam(self, l):
        return lib().orc_pmg_lambda(self.ptr, l, 0), lib().orc_pmg_lambda(self.ptr, l, 1)

    def vcycle(self, r):
        z = np.zeros(self.levels[0].nl)
        lib().orc_pmg_vcycle(self.ptr, np.ascontiguousarray(r, dtype=np.float64), z)
        return z

    def coarse_iters(self):
        return lib().orc_pmg_coarse_iters(self.ptr)

    def fgmres(self, b, x0=None, tol=1e-8, restart=30, maxit=500, precond=True):
        """Flexible GMRES(restart); returns x and a dict with the residual
        history (||r0||, then the least-squares residual of every step)."""
        x = np.zeros(self.levels[0].nl) if x0 is None else np.array(x0, dtype=np.float64,
                                                                     copy=True)
        it, r0, r1 = C.c_int(), C.c_double(), C.c_double()
        hist = np.zeros(maxit + 1)
        st = lib().orc_fgmres(self.ptr, int(precond), np.ascontiguousarray(b, dtype=np.float64),
                              x, tol, restart, maxit, C.byref(it), C.byref(r0), C.byref(r1),
                              hist.ctypes.data_as(C.c_void_p))
        return x, {"status": st, "iters": it.value, "res0": r0.value, "res": r1.value,
                   "hist": hist[:it.value + 1]}

    def flexpcg(self, b, x0=None, tol=1e-8, maxit=500, precond=True):
        x = np.zeros(self.levels[0].nl) if x0 is None else np.array(x0, dtype=np.float64,
                                                                     copy=True)
        it, r0, r1 = C.c_int(), C.c_double(), C.c_double()
        st = lib().orc_flexpcg(self.ptr, int(precond), np.ascontiguousarray(b, dtype=np.float64),
                               x, tol, maxit, C.byref(it), C.byref(r0), C.byref(r1))
        return x, {"status": st, "iters": it.value, "res0": r0.value, "res": r1.value}


class Projection:
    """Projection onto previous solutions (orc_solve_projected) for a PMG."""

    def __init__(self, pmg, Lmax):
        self.pmg = pmg
        self.ptr = lib().orc_proj_create(pmg.ptr, Lmax)

    def __del__(self):
        if getattr(self, "ptr", None):
            lib().orc_proj_destroy(self.ptr)
            self.ptr = None

    @property
    def nvec(self):
        return lib().orc_proj_nvec(self.ptr)

    def vector(self, i):
        n = self.pmg.levels[0].nl
        p, ap = np.zeros(n), np.zeros(n)
        lib().orc_proj_vector(self.ptr, i, p, ap)
        return p, ap

    def solve(self, b, tol=1e-8, maxit=500, solver="flexcg", restart=20):
        x = np.zeros(self.pmg.levels[0].nl)
        it, rp, r1 = C.c_int(), C.c_double(), C.c_double()
        st = lib().orc_solve_projected(self.pmg.ptr, self.ptr, 1 if solver == "fgmres" else 0,
                                       restart, np.ascontiguousarray(b, dtype=np.float64), x,
                                       tol, maxit, C.byref(it), C.byref(rp), C.byref(r1))
        return x, {"status": st, "iters": it.value, "res_proj": rp.value, "res": r1.value}


class ASM:
    """Overlapping Schwarz preconditioner of a level (orc_asm): local
    separable problems on elements extended by one layer, solved densely."""

    def __init__(self, level):
        self.level = level
        self.ptr = lib().orc_asm_create(level.ptr)

    def __del__(self):
        if getattr(self, "ptr", None):
            lib().orc_asm_destroy(self.ptr)
            self.ptr = None

    def apply(self, r):
        z = np.zeros(self.level.nl)
        lib().orc_asm_apply(self.ptr, np.ascontiguousarray(r, dtype=np.float64), z)
        return z

    def local_matrix(self, e):
        n = self.level.N + 3
        K = np.zeros((n ** 3, n ** 3))
        lib().orc_asm_local_matrix(self.ptr, int(e), K)
        return K
