"""GPU parity of the operator, gather-scatter, mesh fields and inner product
against the FP64 oracle, through the C ABI.

Tolerances (norm-wise, max |gpu - oracle| / max |oracle|):
  FP64: 1e-12 (Ax, gs, fields), FP32: 64 * Np * 2^-24 (Ax with float factors).
Sizes span several CTA tiles with ragged tails (E not a multiple of the
elements per CTA) and the grid-stride loop (more elements than one grid).
"""

import numpy as np
import pytest

import oracle
from paper_2110_01716_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2110_01716_gb300 import sem  # noqa: E402

DEV = torch.device("cuda:0")
TOL64 = 1e-12


def rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def tol32(N):
    return 64 * (N + 1) * 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_2110_01716_gb300 import build

    build.build()
    oracle.build()


def make(ex, ey, ez, N, bc=0, geom=sem.SEM_GEOM_STORED, seed=3, arith=sem.SEM_ARITH_PAIR):
    v = inputs.box_vertices(ex, ey, ez, 0.1, seed)
    return (sem.Mesh(ex, ey, ez, N, bc, geom, verts=v, f64_arith=arith),
            oracle.Level(ex, ey, ez, N, bc, v), v)


# (geometry, FP64 arithmetic): stored factors with FP32-pair or native FP64
# arithmetic, and recomputed trilinear factors (native FP64)
MODES = [(sem.SEM_GEOM_STORED, sem.SEM_ARITH_PAIR), (sem.SEM_GEOM_STORED, sem.SEM_ARITH_NATIVE),
         (sem.SEM_GEOM_TRILINEAR, sem.SEM_ARITH_NATIVE)]


CASES = [(1, 1, 1, 1), (2, 3, 2, 2), (3, 2, 4, 3), (5, 3, 2, 4), (2, 2, 3, 5), (3, 4, 2, 6),
         (5, 7, 9, 7), (2, 3, 3, 8), (3, 2, 2, 9), (2, 2, 2, 10), (2, 1, 2, 11)]


@pytest.mark.parametrize("ex,ey,ez,N", CASES)
@pytest.mark.parametrize("geom,arith", MODES)
def test_ax_fp64_matches_oracle(ex, ey, ez, N, geom, arith):
    m, L, _ = make(ex, ey, ez, N, geom=geom, arith=arith)
    u = inputs.random_field(L.nl, 11)
    ud = torch.tensor(u, device=DEV)
    wd = torch.empty_like(ud)
    sem.sem_ax(m, sem.SEM_F64, ud, wd, sem.SEM_AX_LOCAL)
    assert rel(wd.cpu().numpy(), L.ax_local(u)) < TOL64
    sem.sem_ax(m, sem.SEM_F64, ud, wd, sem.SEM_AX_ASSEMBLED)
    assert rel(wd.cpu().numpy(), L.ax(u)) < TOL64


@pytest.mark.parametrize("ex,ey,ez,N", [(3, 2, 4, 3), (5, 7, 9, 7), (2, 2, 3, 5), (2, 2, 2, 10)])
@pytest.mark.parametrize("geom", [sem.SEM_GEOM_STORED, sem.SEM_GEOM_TRILINEAR])
def test_ax_fp32_matches_oracle_within_stated_tolerance(ex, ey, ez, N, geom):
    m, L, _ = make(ex, ey, ez, N, geom=geom)
    u = inputs.random_field(L.nl, 12)
    ud = torch.tensor(u, device=DEV, dtype=torch.float32)
    wd = torch.empty_like(ud)
    sem.sem_ax(m, sem.SEM_F32, ud, wd, sem.SEM_AX_ASSEMBLED)
    # the oracle applied to the same float-rounded input
    ref = L.ax(ud.double().cpu().numpy())
    err = rel(wd.double().cpu().numpy(), ref)
    assert err < tol32(N), err


def test_ax_dirichlet_and_neumann_masks():
    for bc in (0, 1):
        m, L, _ = make(3, 3, 2, 4, bc=bc)
        u = inputs.random_field(L.nl, 5)
        ud = torch.tensor(u, device=DEV)
        wd = torch.empty_like(ud)
        sem.sem_ax(m, sem.SEM_F64, ud, wd, sem.SEM_AX_ASSEMBLED)
        assert rel(wd.cpu().numpy(), L.ax(u)) < TOL64


def test_ax_pair_arithmetic_on_wide_dynamic_range():
    """FP32-pair arithmetic keeps FP64 accuracy for inputs spanning many
    decades, signed zeros and exact zeros."""
    m, L, _ = make(3, 2, 2, 6)
    rng = np.random.Generator(np.random.PCG64(77))
    u = rng.uniform(-1, 1, L.nl) * 10.0 ** rng.uniform(-30, 30, L.nl)
    u[::17] = 0.0
    u[5::19] = -0.0
    ud = torch.tensor(u, device=DEV)
    wd = torch.empty_like(ud)
    sem.sem_ax(m, sem.SEM_F64, ud, wd, sem.SEM_AX_LOCAL)
    assert rel(wd.cpu().numpy(), L.ax_local(u)) < TOL64
    for scale in (1e-20, 1e20):
        v = inputs.random_field(L.nl, 4) * scale
        sem.sem_ax(m, sem.SEM_F64, torch.tensor(v, device=DEV), wd, sem.SEM_AX_LOCAL)
        assert rel(wd.cpu().numpy(), L.ax_local(v)) < TOL64


def test_ax_nan_propagates():
    m, L, _ = make(2, 2, 2, 3)
    for arith in (sem.SEM_ARITH_PAIR, sem.SEM_ARITH_NATIVE):
        m, L, _ = make(2, 2, 2, 3, arith=arith)
        u = inputs.random_field(L.nl, 4)
        u[10] = np.nan
        wd = torch.empty(L.nl, device=DEV, dtype=torch.float64)
        sem.sem_ax(m, sem.SEM_F64, torch.tensor(u, device=DEV), wd, sem.SEM_AX_LOCAL)
        assert torch.isnan(wd).any()


def test_ax_grid_stride_many_elements():
    # more elements than one grid of CTAs covers
    m, L, _ = make(24, 22, 21, 7)
    u = inputs.random_field(L.nl, 13)
    ud = torch.tensor(u, device=DEV)
    wd = torch.empty_like(ud)
    sem.sem_ax(m, sem.SEM_F64, ud, wd, sem.SEM_AX_ASSEMBLED)
    assert rel(wd.cpu().numpy(), L.ax(u)) < TOL64


@pytest.mark.parametrize("ex,ey,ez,N", [(1, 1, 1, 1), (3, 2, 4, 3), (5, 7, 9, 7), (2, 3, 2, 11)])
@pytest.mark.parametrize("dtype", [sem.SEM_F64, sem.SEM_F32])
def test_gs_matches_oracle_and_copies_are_identical(ex, ey, ez, N, dtype):
    m, L, _ = make(ex, ey, ez, N)
    u = inputs.random_field(L.nl, 21)
    td = torch.float64 if dtype == sem.SEM_F64 else torch.float32
    ud = torch.tensor(u, device=DEV, dtype=td)
    sem.sem_gs(m, dtype, ud)
    got = ud.double().cpu().numpy()
    u_in = u if dtype == sem.SEM_F64 else u.astype(np.float32).astype(np.float64)
    ref = L.gs(u_in)
    tol = TOL64 if dtype == sem.SEM_F64 else 8 * 2.0 ** -24
    assert rel(got, ref) < tol
    # every copy of a node holds the same bits
    ids = L.ids
    order = np.argsort(ids, kind="stable")
    g = got[order]
    s = ids[order]
    same = s[1:] == s[:-1]
    assert np.all(g[1:][same] == g[:-1][same])


def test_gs_of_ones_is_multiplicity_and_fields():
    m, L, _ = make(4, 3, 5, 6)
    ones = torch.ones(L.nl, device=DEV, dtype=torch.float64)
    sem.sem_gs(m, sem.SEM_F64, ones)
    assert np.array_equal(ones.cpu().numpy(), L.mult)
    out = torch.empty(L.nl, device=DEV, dtype=torch.float64)
    X = L.X
    for which, ref in [(sem.SEM_FIELD_X, X[:, 0].ravel()), (sem.SEM_FIELD_Y, X[:, 1].ravel()),
                       (sem.SEM_FIELD_Z, X[:, 2].ravel()), (sem.SEM_FIELD_MASS, L.B),
                       (sem.SEM_FIELD_MULT, L.mult), (sem.SEM_FIELD_MASK, L.mask),
                       (sem.SEM_FIELD_DINV, L.dinv)]:
        sem.sem_mesh_field(m, which, out)
        assert rel(out.cpu().numpy(), ref) < TOL64, which


def test_builtin_vertex_generator_matches_input_module():
    v = inputs.box_vertices(4, 3, 5, 0.1, seed=9)
    m_builtin = sem.Mesh(4, 3, 5, 4, 0, jitter=0.1, seed=9)
    m_given = sem.Mesh(4, 3, 5, 4, 0, verts=v)
    a = torch.empty(m_given.n_local, device=DEV, dtype=torch.float64)
    b = torch.empty_like(a)
    for which in (sem.SEM_FIELD_X, sem.SEM_FIELD_Y, sem.SEM_FIELD_Z):
        sem.sem_mesh_field(m_builtin, which, a)
        sem.sem_mesh_field(m_given, which, b)
        assert torch.equal(a, b)


def test_dot_matches_oracle():
    m, L, _ = make(3, 4, 2, 5)
    u = L.gs(inputs.random_field(L.nl, 1)) / L.mult
    v = L.gs(inputs.random_field(L.nl, 2)) / L.mult
    got = sem.sem_dot(m, torch.tensor(u, device=DEV), torch.tensor(v, device=DEV))
    ref = L.dot(u, v)
    assert abs(got - ref) < 1e-12 * np.sqrt(L.dot(u, u) * L.dot(v, v))


def test_ax_is_deterministic():
    m, L, _ = make(6, 5, 4, 7)
    ud = torch.tensor(inputs.random_field(L.nl, 3), device=DEV)
    w1 = torch.empty_like(ud)
    w2 = torch.empty_like(ud)
    sem.sem_ax(m, sem.SEM_F64, ud, w1, sem.SEM_AX_ASSEMBLED)
    sem.sem_ax(m, sem.SEM_F64, ud, w2, sem.SEM_AX_ASSEMBLED)
    assert torch.equal(w1, w2)
    assert sem.sem_dot(m, w1, w1) == sem.sem_dot(m, w2, w2)


def _element_vertices(v, ex, ey, e):
    ix, iy, iz = e % ex, (e // ex) % ey, e // (ex * ey)
    out = np.zeros((8, 3))
    for c in range(2):
        for b in range(2):
            for a in range(2):
                out[a + 2 * b + 4 * c] = v[(ix + a) + (ex + 1) * ((iy + b) + (ey + 1) * (iz + c))]
    return out


@pytest.mark.parametrize("k,geom,arith", [(64, sem.SEM_GEOM_STORED, sem.SEM_ARITH_PAIR),
                                          (64, sem.SEM_GEOM_STORED, sem.SEM_ARITH_NATIVE),
                                          (48, sem.SEM_GEOM_TRILINEAR, sem.SEM_ARITH_NATIVE)])
def test_ax_full_size_sampled_elements(k, geom, arith):
    """Operator-sweep sizes in the benchmark's launch configuration: the local
    operator of sampled elements against the oracle run on those elements."""
    N = 7
    v = inputs.box_vertices(k, k, k, 0.1, seed=2 + k)
    m = sem.Mesh(k, k, k, N, 0, geom, verts=v, f64_arith=arith)
    Np3 = (N + 1) ** 3
    u = inputs.random_field(m.n_local, 100 + k)
    ud = torch.tensor(u, device=DEV)
    wd = torch.empty_like(ud)
    sem.sem_ax(m, sem.SEM_F64, ud, wd, sem.SEM_AX_LOCAL)
    rng = np.random.Generator(np.random.PCG64(k))
    sample = np.unique(np.concatenate([rng.integers(0, k ** 3, 40), [0, k ** 3 - 1]]))
    w = wd.cpu().numpy()
    for e in sample:
        ev = _element_vertices(v, k, k, int(e))
        # one-element oracle mesh with this element's corners
        lat = np.zeros((8, 3))
        for c in range(2):
            for b in range(2):
                for a in range(2):
                    lat[a + 2 * (b + 2 * c)] = ev[a + 2 * b + 4 * c]
        Lo = oracle.Level(1, 1, 1, N, 1, lat)
        ref = Lo.ax_local(u[e * Np3:(e + 1) * Np3])
        assert rel(w[e * Np3:(e + 1) * Np3], ref) < TOL64, e
