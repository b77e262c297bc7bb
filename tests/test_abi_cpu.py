"""The C ABI library builds, loads and exports what include/sem.h declares;
argument errors come back as status codes before any device work (CPU only)."""

import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libsem():
    from paper_2110_01716_gb300 import build, sem

    build.build()
    return sem


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "sem.h")).read()
    return sorted(set(re.findall(r"^\s*(?:sem_status|const char \*)\s*(sem_\w+)\(", text, re.M)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ["sem_mesh_create", "sem_ax", "sem_gs", "sem_pmg_setup", "sem_solve"]:
        assert required in names


def test_library_has_no_unresolved_symbols(libsem):
    """Load with immediate binding, as some loaders do: every symbol the
    library needs (internal template instantiations included) resolves."""
    C.CDLL(libsem.LIB_PATH, mode=os.RTLD_NOW | os.RTLD_LOCAL)


def test_every_declared_symbol_is_exported(libsem):
    L = libsem.lib()
    missing = [n for n in declared_symbols() if not hasattr(L, n)]
    assert not missing, missing
    assert set(declared_symbols()) <= set(libsem.EXPORTED) | {"sem_last_error"}


def test_invalid_arguments_return_einval_without_device_work(libsem):
    L = libsem.lib()
    h = C.c_void_p()
    # null descriptor
    assert L.sem_mesh_create(None, None, C.byref(h)) == libsem.SEM_EINVAL
    assert "null" in libsem.last_error()
    for bad in [dict(ex=0), dict(N=0), dict(N=libsem.SEM_MAX_ORDER + 1), dict(bc=7),
                dict(geom=5), dict(jitter=0.7)]:
        args = dict(ex=2, ey=2, ez=2, N=3, jitter=0.1, seed=1, bc=0, geom=0, verts=None)
        args.update(bad)
        desc = libsem.sem_mesh_desc(**args)
        st = L.sem_mesh_create(C.byref(desc), None, C.byref(h))
        assert st == libsem.SEM_EINVAL, (bad, st)
        assert libsem.last_error()
        assert not h.value
    # maximum sizes: more than 2^31 elements, more than 2^31 - 1 local points
    for ex, N, msg in ((1300, 3, "too many elements"), (120, 11, "too large")):
        desc = libsem.sem_mesh_desc(ex=ex, ey=ex, ez=ex, N=N, jitter=0.1, seed=1, bc=0, geom=0,
                                    verts=None)
        assert L.sem_mesh_create(C.byref(desc), None, C.byref(h)) == libsem.SEM_EINVAL
        assert msg in libsem.last_error() and not h.value
    # null handles are rejected
    assert L.sem_ax(None, 0, None, None, 0, None) == libsem.SEM_EINVAL
    assert L.sem_gs(None, 0, None, None) == libsem.SEM_EINVAL
    assert L.sem_pmg_setup(None, None, None, C.byref(h)) == libsem.SEM_EINVAL
    info = libsem.sem_solve_info()
    desc = libsem.sem_solve_desc(0, 1e-8, 10, 1)
    assert L.sem_solve(None, None, None, None, C.byref(desc), C.byref(info), None) == \
        libsem.SEM_EINVAL
    assert L.sem_inject_wait_error(None, None) == libsem.SEM_EINVAL
    assert L.sem_batch_create(None, None, 0, None, C.byref(h)) == libsem.SEM_EINVAL
    assert L.sem_batch_solve(None, None, None) == libsem.SEM_EINVAL
    assert L.sem_batch_info(None, None, None, None) == libsem.SEM_EINVAL
    assert L.sem_batch_autotune(None, None, 0, 0, None, None, None) == libsem.SEM_EINVAL
    assert L.sem_batch_destroy(None) == libsem.SEM_OK
    # batch descriptions and requests are checked before any device work
    bd = libsem.sem_batch_desc(cheb_degree=3, smoother_dtype=1, coarse_tol=0.2, coarse_maxit=30)
    good = libsem.make_request(2, 2, 2, 5)
    for bad in (dict(N=1), dict(solver=libsem.SEM_SOLVER_PCG), dict(bc=1), dict(ex=0)):
        r = libsem.make_request(bad.get("ex", 2), 2, 2, bad.get("N", 5), bc=bad.get("bc", 0),
                                solver=bad.get("solver", libsem.SEM_SOLVER_FLEXCG))
        arr = (libsem.sem_request * 2)(good, r)
        assert L.sem_batch_create(C.byref(bd), arr, 2, None, C.byref(h)) == libsem.SEM_EINVAL, bad
        assert not h.value
    bd.ax_fill[3] = -1.0
    arr = (libsem.sem_request * 1)(good)
    assert L.sem_batch_create(C.byref(bd), arr, 1, None, C.byref(h)) == libsem.SEM_EINVAL
    assert "ax_fill" in libsem.last_error()
    assert L.sem_dot_noalloc(None, None, None, None, None) == libsem.SEM_EINVAL
    assert "null argument" in libsem.last_error()
    assert L.sem_mesh_destroy(None) == libsem.SEM_OK
    assert L.sem_pmg_destroy(None) == libsem.SEM_OK


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2110_01716_gb300 import sem

    monkeypatch.setattr(sem, "_lib", None)
    monkeypatch.setattr(sem, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not built"):
        sem.lib()


def test_injected_allocation_failure_returns_enomem_without_device_work(libsem):
    """Host-side fault injection: the armed allocation fails with SEM_ENOMEM
    before reaching the CUDA allocator (no GPU is needed to see it) and the
    call returns no handle."""
    L = libsem.lib()
    assert L.sem_inject_alloc_failure(-1) == libsem.SEM_EINVAL
    desc = libsem.sem_mesh_desc(ex=2, ey=2, ez=2, N=3, jitter=0.1, seed=1, bc=0, geom=0,
                                verts=None)
    h = C.c_void_p()
    try:
        assert L.sem_inject_alloc_failure(1) == libsem.SEM_OK
        assert L.sem_mesh_create(C.byref(desc), None, C.byref(h)) == libsem.SEM_ENOMEM
        assert "injected" in libsem.last_error()
        assert not h.value
    finally:
        assert L.sem_inject_alloc_failure(0) == libsem.SEM_OK
