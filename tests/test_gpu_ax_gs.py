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


# FP32 on stored factors runs the fused operator, whose CTAs walk x-lines of
# elements: meshes with few lines split them into segments (seams), many
# lines (2 x 31 x 30) take whole lines, ex < elements per chunk leaves CTA
# slots idle; odd ex gives ragged chunks.
FP32_CASES = [(3, 2, 4, 3), (5, 7, 9, 7), (2, 2, 3, 5), (2, 2, 2, 10), (40, 2, 2, 7), (13, 3, 2, 4),
              (1, 3, 5, 2), (7, 1, 1, 1), (2, 31, 30, 3), (3, 31, 30, 7), (9, 2, 3, 11)]


@pytest.mark.parametrize("ex,ey,ez,N", FP32_CASES)
@pytest.mark.parametrize("geom", [sem.SEM_GEOM_STORED, sem.SEM_GEOM_TRILINEAR])
@pytest.mark.parametrize("bc", [0, 1])
def test_ax_fp32_matches_oracle_within_stated_tolerance(ex, ey, ez, N, geom, bc):
    if geom == sem.SEM_GEOM_TRILINEAR and ey * ez > 100:
        pytest.skip("the trilinear FP32 operator does not depend on the line split")
    m, L, _ = make(ex, ey, ez, N, bc=bc, geom=geom)
    u = inputs.random_field(L.nl, 12)
    ud = torch.tensor(u, device=DEV, dtype=torch.float32)
    wd = torch.empty_like(ud)
    sem.sem_ax(m, sem.SEM_F32, ud, wd, sem.SEM_AX_ASSEMBLED)
    # the oracle applied to the same float-rounded input
    ref = L.ax(ud.double().cpu().numpy())
    w = wd.double().cpu().numpy()
    err = rel(w, ref)
    assert err < tol32(N), err
    # copies of every node are bit-identical and masked nodes exactly zero
    ids = L.ids
    lo = np.full(L.ng, np.inf)
    hi = np.full(L.ng, -np.inf)
    np.minimum.at(lo, ids, w)
    np.maximum.at(hi, ids, w)
    assert np.array_equal(lo, hi)
    assert np.all(w[L.mask == 0] == 0)
    sem.sem_ax(m, sem.SEM_F32, ud, wd, sem.SEM_AX_LOCAL)
    assert rel(wd.double().cpu().numpy(), L.ax_local(ud.double().cpu().numpy())) < tol32(N)


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


# ---------------------------------------------------------------- 16-bit factors
# FP16 / BF16 storage of the six factors (per element and factor scale), FP32
# vectors and arithmetic.  Two checks: (1) against the FP64 oracle applied to
# the same stored factors, whose rounding tests/quant16.py defines
# independently, within the FP32 tolerance; (2) against the exact operator,
# point by point, within the bound the storage rounding implies:
#   |w - A u| <= |D|^T H |D| |u| + tol32 * max|A u|,  H_e = h * scale_e,
# h = half an ulp at 1 (2^-12 FP16, 2^-9 BF16), scale_e the element's scale.
from quant16 import quantise_factors  # noqa: E402

G16_KINDS = [(sem.SEM_F16, "f16", 2.0 ** -12), (sem.SEM_BF16, "bf16", 2.0 ** -9)]


@pytest.mark.parametrize("ex,ey,ez,N", [(3, 2, 4, 3), (5, 7, 9, 7), (2, 2, 3, 5), (2, 2, 2, 10),
                                        (1, 1, 1, 1)])
@pytest.mark.parametrize("kind,name,h", G16_KINDS)
def test_ax_16bit_factors_match_oracle_on_stored_values(ex, ey, ez, N, kind, name, h):
    m, L, _ = make(ex, ey, ez, N)
    Np3 = (N + 1) ** 3
    u = inputs.random_field(L.nl, 21)
    ud = torch.tensor(u, device=DEV, dtype=torch.float32)
    u32 = ud.double().cpu().numpy()
    wd = torch.empty_like(ud)
    sem.sem_ax(m, kind, ud, wd, sem.SEM_AX_LOCAL)
    w = wd.double().cpu().numpy()
    Gq, sc = quantise_factors(L.G, L.E, Np3, name)
    ref = oracle.ax_local(N, L.D, Gq, u32)
    err = rel(w, ref)
    assert err < tol32(N), err
    # (2) elementwise bound against the exact (unrounded) operator
    exact = L.ax_local(u32)
    H = np.repeat(h * sc.astype(np.float64), 6 * Np3)
    bound = oracle.ax_local(N, np.abs(L.D), H, np.abs(u32)) + tol32(N) * np.max(np.abs(exact))
    assert np.all(np.abs(w - exact) <= bound)
    # assembled form: gs and mask of the local result
    sem.sem_ax(m, kind, ud, wd, sem.SEM_AX_ASSEMBLED)
    ref_a = L.mask * oracle.gs(L.ids, L.ng, ref)
    assert rel(wd.double().cpu().numpy(), ref_a) < tol32(N)


def test_ax_16bit_full_size_sampled_elements():
    """64^3 elements of order 7 (the operator-sweep size): sampled elements
    against the oracle on their own stored factors."""
    e, N = 64, 7
    v = inputs.box_vertices(e, e, e, 0.1, 9)
    m = sem.Mesh(e, e, e, N, 0, verts=v)
    Np3 = (N + 1) ** 3
    nl = e ** 3 * Np3
    ud = torch.rand(nl, device=DEV, generator=torch.Generator(DEV).manual_seed(4),
                    dtype=torch.float32) * 2 - 1
    wd = torch.empty_like(ud)
    rng = np.random.Generator(np.random.PCG64(e))
    sample = np.unique(np.concatenate([rng.integers(0, e ** 3, 12), [0, e ** 3 - 1]]))
    for kind, name, _ in G16_KINDS:
        sem.sem_ax(m, kind, ud, wd, sem.SEM_AX_LOCAL)
        for el in sample:
            Lo = oracle.Level(1, 1, 1, N, 1, _element_vertices(v, e, e, int(el)))
            Gq, _ = quantise_factors(Lo.G, 1, Np3, name)
            ue = ud[el * Np3:(el + 1) * Np3].double().cpu().numpy()
            ref = oracle.ax_local(N, Lo.D, Gq, ue)
            got = wd[el * Np3:(el + 1) * Np3].double().cpu().numpy()
            assert rel(got, ref) < tol32(N), (name, el)


def _sub_box(v, ex, ey, ez, c, r=1):
    """Vertices and global element indices of the box of elements within r of
    element c = (cx, cy, cz), clipped to the mesh; also c's index inside it."""
    lo = [max(0, c[d] - r) for d in range(3)]
    hi = [min((ex, ey, ez)[d] - 1, c[d] + r) for d in range(3)]
    n = [hi[d] - lo[d] + 1 for d in range(3)]
    V = np.asarray(v).reshape(ez + 1, ey + 1, ex + 1, 3)
    sub = V[lo[2]:hi[2] + 2, lo[1]:hi[1] + 2, lo[0]:hi[0] + 2].reshape(-1, 3)
    els = [(lo[0] + a) + ex * ((lo[1] + b) + ey * (lo[2] + g))
           for g in range(n[2]) for b in range(n[1]) for a in range(n[0])]
    centre = (c[0] - lo[0]) + n[0] * ((c[1] - lo[1]) + n[1] * (c[2] - lo[2]))
    return n, np.ascontiguousarray(sub), np.array(els), centre


@pytest.mark.parametrize("kind,name", [(sem.SEM_F32, None), (sem.SEM_F16, "f16"),
                                       (sem.SEM_BF16, "bf16")])
def test_ax_fp32_assembled_full_size_sampled(kind, name):
    """The assembled FP32 operator at the benchmark's size (48^3 elements,
    N = 7, Neumann) and launch configuration: every node of a sampled element
    against the oracle's assembled operator on the box of elements around it,
    which holds all copies of those nodes."""
    e, N = 48, 7
    v = inputs.box_vertices(e, e, e, 0.1, 3)
    m = sem.Mesh(e, e, e, N, 1, verts=v)
    Np3 = (N + 1) ** 3
    ud = torch.rand(m.n_local, device=DEV, generator=torch.Generator(DEV).manual_seed(8),
                    dtype=torch.float32) * 2 - 1
    wd = torch.empty_like(ud)
    sem.sem_ax(m, kind, ud, wd, sem.SEM_AX_ASSEMBLED)
    rng = np.random.Generator(np.random.PCG64(48))
    cents = [tuple(int(x) for x in rng.integers(0, e, 3)) for _ in range(6)]
    cents += [(0, 0, 0), (e - 1, e - 1, e - 1), (0, e - 1, 17), (23, 0, e - 1)]
    u3 = ud.view(-1, Np3)
    w3 = wd.view(-1, Np3)
    for c in cents:
        n, sub, els, centre = _sub_box(v, e, e, e, c)
        Lo = oracle.Level(*n, N, 1, sub)
        us = u3[torch.tensor(els, device=DEV)].double().cpu().numpy().reshape(-1)
        if name is None:
            ref = Lo.ax(us)
        else:
            Gq, _ = quantise_factors(Lo.G, Lo.E, Np3, name)
            ref = oracle.gs(Lo.ids, Lo.ng, oracle.ax_local(N, Lo.D, Gq, us))
        ref_c = ref.reshape(-1, Np3)[centre]
        got = w3[els[centre]].double().cpu().numpy()
        assert rel(got, ref_c) < tol32(N), c


@pytest.mark.parametrize("N", [3, 7])
@pytest.mark.parametrize("bc", [0, 1])
def test_operator_invariants_symmetry_null_space_and_gs(N, bc):
    """Invariants of the assembled FP64 operator and of gs on the GPU, which
    need no reference output: u^T A v = v^T A u in the unique-dof product for
    continuous u, v; A 1 = 0 under Neumann; gs(u) = mult u for continuous u."""
    m, L, _ = make(3, 2, 2, N, bc=bc)

    def cont(seed):
        return L.gs(inputs.random_field(L.nl, seed)) / L.mult * L.mask

    def A(x):
        xd = torch.tensor(x, device=DEV)
        wd = torch.empty_like(xd)
        sem.sem_ax(m, sem.SEM_F64, xd, wd, sem.SEM_AX_ASSEMBLED)
        return wd.cpu().numpy()

    u, v = cont(21), cont(22)
    Au, Av = A(u), A(v)
    uAv, vAu = np.sum(u * Av / L.mult), np.sum(v * Au / L.mult)
    assert abs(uAv - vAu) <= 1e-11 * np.sqrt(np.sum(u * Au / L.mult) * np.sum(v * Av / L.mult))
    if bc == 1:
        assert np.abs(A(np.ones(L.nl))).max() <= 1e-11 * np.abs(Au).max()
    ud = torch.tensor(u, device=DEV)
    sem.sem_gs(m, sem.SEM_F64, ud)
    assert np.abs(ud.cpu().numpy() - L.mult * u).max() <= 1e-14 * np.abs(L.mult * u).max()
