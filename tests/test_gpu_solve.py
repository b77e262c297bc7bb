"""GPU parity of the solvers against the FP64 oracle, through the C ABI.

* Jacobi-PCG: the residual of the GPU solution, recomputed by the oracle,
  meets the tolerance; the solution matches the oracle's solution.
* pMG V-cycle with an FP64 smoother and a fixed number of coarse iterations
  is a fixed linear map: it matches the oracle's V-cycle to 1e-10.
* FlexCG + pMG (FP64 and FP32 smoothers) reaches 1e-8; the final error against
  the oracle's solution is reported and bounded.
* Status codes: SEM_ENOTCONV at max_iter, SEM_EINVAL for a Neumann right-hand
  side that is not mean-free.
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


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_2110_01716_gb300 import build

    build.build()
    oracle.build()


def rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def manufactured(L):
    X = L.X
    us = (np.sin(np.pi * X[:, 0]) * np.sin(np.pi * X[:, 1]) * np.sin(np.pi * X[:, 2])).ravel()
    return us, L.assembled_rhs(3 * np.pi ** 2 * us)


def fourier_rhs(L, seed=3):
    a, k, phi = inputs.fourier_modes(seed)
    X = L.X
    f = sum(a[m] * np.cos(2 * np.pi * (k[m, 0] * X[:, 0] + k[m, 1] * X[:, 1] + k[m, 2] * X[:, 2])
                          + phi[m]) for m in range(len(a))).ravel()
    b = L.gs(L.B * f)
    return b - L.dot(b, np.ones(L.nl)) / L.ng


def residual(L, b, x):
    r = b - L.ax(x)
    return np.sqrt(L.dot(r, r)) / np.sqrt(L.dot(b, b))


@pytest.mark.parametrize("e,N", [(8, 7), (3, 5), (2, 1)])
def test_jacobi_pcg_manufactured(e, N):
    v = inputs.box_vertices(e, e, e, 0.1, 1)
    m = sem.Mesh(e, e, e, N, sem.SEM_DIRICHLET, verts=v)
    L = oracle.Level(e, e, e, N, 0, v)
    us, b = manufactured(L)
    bd = torch.tensor(b, device=DEV)
    xd = torch.zeros_like(bd)
    info = sem.sem_solve(m, None, bd, xd, sem.SEM_SOLVER_PCG, tol=1e-10, max_iter=2000)
    assert info["status"] == sem.SEM_OK, info
    x = xd.cpu().numpy()
    assert residual(L, b, x) <= 1.05e-10
    xo, io = L.pcg(b, tol=1e-10, maxit=2000)
    assert abs(info["iters"] - io["iters"]) <= 2
    assert rel(x, xo) < 1e-8
    if (e, N) == (8, 7):
        assert np.max(np.abs(x - us)) < 1e-9  # discretisation error of the config-1 problem


def test_pcg_check_every_and_host_buffers():
    v = inputs.box_vertices(4, 4, 4, 0.1, 1)
    m = sem.Mesh(4, 4, 4, 6, 0, verts=v)
    L = oracle.Level(4, 4, 4, 6, 0, v)
    _, b = manufactured(L)
    x_host = np.zeros(L.nl)
    info = sem.sem_solve_host(m, None, b.copy(), x_host, sem.SEM_SOLVER_PCG, tol=1e-9,
                              max_iter=1000, check_every=8)
    assert info["status"] == sem.SEM_OK
    assert info["iters"] % 8 == 0
    assert residual(L, b, x_host) <= 1.05e-9


def test_pcg_not_converged_status():
    m = sem.Mesh(3, 3, 3, 5, 0, jitter=0.1, seed=2)
    L = oracle.Level(3, 3, 3, 5, 0, inputs.box_vertices(3, 3, 3, 0.1, 2))
    _, b = manufactured(L)
    bd = torch.tensor(b, device=DEV)
    xd = torch.zeros_like(bd)
    info = sem.sem_solve(m, None, bd, xd, sem.SEM_SOLVER_PCG, tol=1e-12, max_iter=3)
    assert info["status"] == sem.SEM_ENOTCONV and info["iters"] == 3
    xo, io = L.pcg(b, tol=0.0, maxit=3)
    assert rel(xd.cpu().numpy(), xo) < 1e-10  # same three iterates


def test_neumann_rhs_must_be_mean_free():
    m = sem.Mesh(2, 2, 2, 3, sem.SEM_NEUMANN, jitter=0.1, seed=1)
    bd = torch.ones(m.n_local, device=DEV, dtype=torch.float64)
    xd = torch.zeros_like(bd)
    with pytest.raises(sem.SemError) as ei:
        sem.sem_solve(m, None, bd, xd, sem.SEM_SOLVER_PCG, tol=1e-8, max_iter=10)
    assert ei.value.status == sem.SEM_EINVAL


@pytest.mark.parametrize("bc,orders,arith", [(0, (5, 3, 1), sem.SEM_ARITH_PAIR),
                                             (1, (7, 3, 1), sem.SEM_ARITH_PAIR),
                                             (1, (7, 3, 1), sem.SEM_ARITH_NATIVE),
                                             (0, (4, 2), sem.SEM_ARITH_PAIR),
                                             (1, (3, 1), sem.SEM_ARITH_NATIVE),
                                             (0, (7, 4, 2, 1), sem.SEM_ARITH_PAIR),
                                             (1, (7, 4, 2, 1), sem.SEM_ARITH_PAIR)])
def test_vcycle_fp64_matches_oracle(bc, orders, arith):
    e = (3, 2, 4)
    v = inputs.box_vertices(*e, 0.1, 5)
    m = sem.Mesh(*e, orders[0], bc, verts=v, f64_arith=arith)
    P = sem.Pmg(m, orders=orders, smoother_dtype=sem.SEM_F64, coarse_tol=0.0, coarse_maxit=12,
                seed=4)
    Po = oracle.PMG(*e, list(orders), bc, v, cheb_degree=2, lanczos_steps=20, seed=4,
                    coarse_tol=0.0, coarse_maxit=12)
    for lvl in range(len(orders) - 1):
        lo, hi = P.lam(lvl)
        olo, ohi = Po.lam(lvl)
        assert abs(hi - ohi) < 1e-10 * ohi and abs(lo - olo) < 1e-10 * olo
    L = Po.levels[0]
    r = L.gs(inputs.random_field(L.nl, 8)) * L.mask
    if bc == 1:
        r -= L.dot(r, np.ones(L.nl)) / L.ng
    zd = torch.empty(L.nl, device=DEV, dtype=torch.float64)
    sem.sem_pmg_vcycle(P, torch.tensor(r, device=DEV), zd)
    assert rel(zd.cpu().numpy(), Po.vcycle(r)) < 1e-10


@pytest.mark.parametrize("e,bc", [((4, 3, 3), 0), ((4, 3, 3), 1), ((2, 31, 30), 1), ((5, 2, 3), 0)])
@pytest.mark.parametrize("orders", [(7, 3, 1), (7, 4, 2, 1)])
def test_vcycle_fp32_close_to_fp64_oracle(e, bc, orders):
    """FP32 smoothing (operator with the Chebyshev update fused in): boxes
    whose x-lines are split into segments and, at 2 x 31 x 30, whole lines;
    the bench's schedules."""
    v = inputs.box_vertices(*e, 0.1, 6)
    m = sem.Mesh(*e, 7, bc, verts=v)
    P = sem.Pmg(m, orders=orders, smoother_dtype=sem.SEM_F32, coarse_tol=0.0, coarse_maxit=20)
    Po = oracle.PMG(*e, list(orders), bc, v, coarse_tol=0.0, coarse_maxit=20)
    L = Po.levels[0]
    b = manufactured(L)[1] if bc == 0 else fourier_rhs(L)
    zd = torch.empty(L.nl, device=DEV, dtype=torch.float64)
    sem.sem_pmg_vcycle(P, torch.tensor(b, device=DEV), zd)
    err = rel(zd.cpu().numpy(), Po.vcycle(b))
    assert err < 1e-4, err  # single precision smoothing, stated tolerance


@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("dtype", [sem.SEM_F64, sem.SEM_F32, sem.SEM_F16, sem.SEM_BF16])
def test_flexcg_pmg_reaches_1e8(bc, dtype):
    e = 6
    v = inputs.box_vertices(e, e, e, 0.1, 3)
    m = sem.Mesh(e, e, e, 7, bc, verts=v)
    L = oracle.Level(e, e, e, 7, bc, v)
    b = manufactured(L)[1] if bc == 0 else fourier_rhs(L)
    P = sem.Pmg(m, orders=(7, 3, 1), smoother_dtype=dtype, coarse_tol=1e-2, coarse_maxit=50)
    bd = torch.tensor(b, device=DEV)
    xd = torch.zeros_like(bd)
    info = sem.sem_solve(m, P, bd, xd, sem.SEM_SOLVER_FLEXCG, tol=1e-8, max_iter=100)
    assert info["status"] == sem.SEM_OK, info
    x = xd.cpu().numpy()
    assert residual(L, b, x) <= 1.05e-8
    Po = oracle.PMG(e, e, e, [7, 3, 1], bc, v, coarse_tol=1e-2, coarse_maxit=50)
    xo, io = Po.flexpcg(b, tol=1e-8, maxit=100)
    if bc == 1:
        x = x - L.dot(x, np.ones(L.nl)) / L.ng
        xo = xo - L.dot(xo, np.ones(L.nl)) / L.ng
    err = rel(x, xo)
    assert err < 1e-6, err
    assert info["iters"] <= io["iters"] + 3


@pytest.mark.parametrize("dtype,tol", [(sem.SEM_F16, 16 * 2.0 ** -11),
                                       (sem.SEM_BF16, 16 * 2.0 ** -8)])
def test_vcycle_16bit_factors_close_to_fp64_oracle(dtype, tol):
    """16-bit factor storage perturbs the smoothed operators by about the
    16-bit unit roundoff u16; the V-cycle output stays within 16 u16."""
    e = (4, 3, 3)
    v = inputs.box_vertices(*e, 0.1, 6)
    m = sem.Mesh(*e, 7, 0, verts=v)
    P = sem.Pmg(m, orders=(7, 3, 1), smoother_dtype=dtype, coarse_tol=0.0, coarse_maxit=20)
    Po = oracle.PMG(*e, [7, 3, 1], 0, v, coarse_tol=0.0, coarse_maxit=20)
    L = Po.levels[0]
    _, b = manufactured(L)
    zd = torch.empty(L.nl, device=DEV, dtype=torch.float64)
    sem.sem_pmg_vcycle(P, torch.tensor(b, device=DEV), zd)
    err = rel(zd.cpu().numpy(), Po.vcycle(b))
    assert err < tol, err


@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("e", [(6, 6, 6), (5, 7, 3), (12, 3, 5), (17, 16, 9)])
def test_multigrid_coarse_mode_solves_the_n1_problem(bc, e):
    """Single-level hierarchy at N = 1: the V-cycle is the coarse solve itself;
    its residual, recomputed by the oracle, meets the requested tolerance."""
    v = inputs.box_vertices(*e, 0.1, 7)
    m = sem.Mesh(*e, 1, bc, verts=v)
    L = oracle.Level(*e, 1, bc, v)
    b = L.gs(inputs.random_field(L.nl, 5)) * L.mask
    if bc == 1:
        b -= L.dot(b, np.ones(L.nl)) / L.ng
    P = sem.Pmg(m, orders=(1,), coarse_tol=1e-9, coarse_maxit=60, coarse_mode=sem.SEM_COARSE_MG)
    zd = torch.empty(L.nl, device=DEV, dtype=torch.float64)
    sem.sem_pmg_vcycle(P, torch.tensor(b, device=DEV), zd)
    z = zd.cpu().numpy()
    assert residual(L, b, z) <= 1.05e-9
    # copies of each node hold the same bits (the result is a continuous field)
    ids = L.ids
    lo = np.full(L.ng, np.inf)
    hi = np.full(L.ng, -np.inf)
    np.minimum.at(lo, ids, z)
    np.maximum.at(hi, ids, z)
    assert np.array_equal(lo, hi)


@pytest.mark.parametrize("bc", [0, 1])
def test_flexcg_with_multigrid_coarse_solve(bc):
    e = 8
    v = inputs.box_vertices(e, e, e, 0.1, 3)
    m = sem.Mesh(e, e, e, 7, bc, verts=v)
    L = oracle.Level(e, e, e, 7, bc, v)
    b = manufactured(L)[1] if bc == 0 else fourier_rhs(L)
    P = sem.Pmg(m, orders=(7, 3, 1), cheb_degree=3, smoother_dtype=sem.SEM_F32, coarse_tol=1e-2,
                coarse_maxit=100, coarse_mode=sem.SEM_COARSE_MG)
    bd = torch.tensor(b, device=DEV)
    xd = torch.zeros_like(bd)
    info = sem.sem_solve(m, P, bd, xd, sem.SEM_SOLVER_FLEXCG, tol=1e-8, max_iter=100)
    assert info["status"] == sem.SEM_OK, info
    assert residual(L, b, xd.cpu().numpy()) <= 1.05e-8
    assert info["iters"] <= 15


def test_multigrid_coarse_mode_needs_order_one():
    m = sem.Mesh(3, 3, 3, 4, 0, jitter=0.1, seed=2)
    with pytest.raises(sem.SemError) as ei:
        sem.Pmg(m, orders=(4, 2), coarse_mode=sem.SEM_COARSE_MG)
    assert ei.value.status == sem.SEM_EINVAL


# ---------------------------------------------------------------- FGMRES
@pytest.mark.parametrize("restart", [8, 3])
@pytest.mark.parametrize("bc", [0, 1])
def test_fgmres_jacobi_matches_oracle(restart, bc):
    """With a fixed (Jacobi) preconditioner FGMRES is a fixed map after a
    given number of steps: the GPU iterate and residual match the oracle's,
    with and without restarts."""
    e, N = (3, 2, 2), 5
    v = inputs.box_vertices(*e, 0.1, 4)
    m = sem.Mesh(*e, N, bc, verts=v)
    Po = oracle.PMG(*e, [N, 1], bc, v)
    L = Po.levels[0]
    b = manufactured(L)[1] if bc == 0 else fourier_rhs(L)
    bd = torch.tensor(b, device=DEV)
    xd = torch.zeros_like(bd)
    info = sem.sem_solve(m, None, bd, xd, sem.SEM_SOLVER_FGMRES, tol=0.0, max_iter=7,
                         restart=restart)
    assert info["status"] == sem.SEM_ENOTCONV and info["iters"] == 7
    xo, io = Po.fgmres(b, tol=0.0, restart=restart, maxit=7, precond=False)
    assert rel(xd.cpu().numpy(), xo) < 1e-9
    assert abs(info["res"] - io["res"]) <= 1e-9 * io["res0"]
    assert abs(info["res"] - residual(L, b, xd.cpu().numpy()) * np.sqrt(L.dot(b, b))) \
        <= 1e-9 * io["res0"]


@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("dtype", [sem.SEM_F64, sem.SEM_F32])
def test_fgmres_pmg_reaches_1e8(bc, dtype):
    e = 6
    v = inputs.box_vertices(e, e, e, 0.1, 3)
    m = sem.Mesh(e, e, e, 7, bc, verts=v)
    L = oracle.Level(e, e, e, 7, bc, v)
    b = manufactured(L)[1] if bc == 0 else fourier_rhs(L)
    P = sem.Pmg(m, orders=(7, 3, 1), smoother_dtype=dtype, coarse_tol=1e-2, coarse_maxit=50)
    bd = torch.tensor(b, device=DEV)
    xd = torch.zeros_like(bd)
    info = sem.sem_solve(m, P, bd, xd, sem.SEM_SOLVER_FGMRES, tol=1e-8, max_iter=100, restart=20)
    assert info["status"] == sem.SEM_OK, info
    x = xd.cpu().numpy()
    assert residual(L, b, x) <= 1.001e-8
    assert abs(info["res"] / info["bnorm"] - residual(L, b, x)) <= 1e-12
    Po = oracle.PMG(e, e, e, [7, 3, 1], bc, v, coarse_tol=1e-2, coarse_maxit=50)
    xo, io = Po.fgmres(b, tol=1e-8, restart=20, maxit=100)
    if bc == 1:
        x = x - L.dot(x, np.ones(L.nl)) / L.ng
        xo = xo - L.dot(xo, np.ones(L.nl)) / L.ng
    assert rel(x, xo) < 1e-6
    assert abs(info["iters"] - io["iters"]) <= 2, (info["iters"], io["iters"])
    # restarted every 3 steps it still converges
    xd.zero_()
    info3 = sem.sem_solve(m, P, bd, xd, sem.SEM_SOLVER_FGMRES, tol=1e-8, max_iter=100, restart=3)
    assert info3["status"] == sem.SEM_OK
    assert residual(L, b, xd.cpu().numpy()) <= 1.001e-8


def test_fgmres_argument_checks():
    m = sem.Mesh(2, 2, 2, 3, 0)
    bd = torch.zeros(m.n_local, device=DEV, dtype=torch.float64)
    xd = torch.zeros_like(bd)
    for bad in (-1, 33):
        with pytest.raises(sem.SemError) as ex:
            sem.sem_solve(m, None, bd, xd, sem.SEM_SOLVER_FGMRES, restart=bad)
        assert ex.value.status == sem.SEM_EINVAL
    # zero right-hand side: converged at once
    info = sem.sem_solve(m, None, bd, xd, sem.SEM_SOLVER_FGMRES, tol=1e-8, restart=32)
    assert info["status"] == sem.SEM_OK and info["iters"] == 0


# ---------------------------------------------------------------- projection
def sequence_rhs(L, n, bc, seed=3):
    a, k, phi, om = inputs.fourier_sequence(seed)
    X = L.X
    f = sum(a[m] * np.cos(2 * np.pi * (k[m, 0] * X[:, 0] + k[m, 1] * X[:, 1]
                                       + k[m, 2] * X[:, 2]) + phi[m] + om[m] * n)
            for m in range(len(a))).ravel()
    b = L.gs(L.B * f)
    if bc == 0:
        return b * L.mask
    return b - L.dot(b, np.ones(L.nl)) / L.ng


@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("solver", [sem.SEM_SOLVER_FLEXCG, sem.SEM_SOLVER_FGMRES])
@pytest.mark.parametrize("Lmax", [30, 3])
def test_projection_sequence_matches_oracle(bc, solver, Lmax):
    """A smooth sequence of right-hand sides: every projected solve meets 1e-8
    (residual recomputed by the oracle), the basis grows (and restarts at
    Lmax) exactly as the oracle's, iterations follow the oracle's within one,
    and solutions agree to 1e-6."""
    e = 4
    v = inputs.box_vertices(e, e, e, 0.1, 3)
    m = sem.Mesh(e, e, e, 7, bc, verts=v)
    P = sem.Pmg(m, orders=(7, 3, 1), smoother_dtype=sem.SEM_F64, coarse_tol=1e-2,
                coarse_maxit=50)
    Q = sem.Projection(m, Lmax)
    Po = oracle.PMG(e, e, e, [7, 3, 1], bc, v, coarse_tol=1e-2, coarse_maxit=50)
    Qo = oracle.Projection(Po, Lmax)
    L = Po.levels[0]
    its = []
    ones = np.ones(L.nl)
    for n in range(8):
        b = sequence_rhs(L, n, bc)
        bd = torch.tensor(b, device=DEV)
        xd = torch.empty_like(bd)
        info = sem.sem_solve_projected(m, P, Q, bd, xd, solver, tol=1e-8, max_iter=100,
                                       restart=20)
        assert info["status"] == sem.SEM_OK, info
        x = xd.cpu().numpy()
        assert residual(L, b, x) <= 1.001e-8
        xo, io = Qo.solve(b, tol=1e-8, solver="fgmres" if solver == sem.SEM_SOLVER_FGMRES
                          else "flexcg", restart=20)
        assert Q.nvec == Qo.nvec <= Lmax
        assert abs(info["iters"] - io["iters"]) <= 1, (n, info["iters"], io["iters"])
        bn = np.sqrt(L.dot(b, b))
        assert abs(info["res0"] - io["res_proj"]) <= 1e-6 * bn
        if bc == 1:
            x = x - L.dot(x, ones) / L.ng
            xo = xo - L.dot(xo, ones) / L.ng
        assert rel(x, xo) < 1e-6
        its.append(info["iters"])
    assert its[-1] < its[0], its


def test_projection_reproduces_a_right_hand_side_in_its_span():
    e = 3
    v = inputs.box_vertices(e, e, e, 0.1, 5)
    m = sem.Mesh(e, e, e, 5, 0, verts=v)
    P = sem.Pmg(m, orders=(5, 2, 1), smoother_dtype=sem.SEM_F64, coarse_tol=1e-3,
                coarse_maxit=100)
    Q = sem.Projection(m, 8)
    L = oracle.Level(e, e, e, 5, 0, v)
    xs = []
    for n in range(3):
        bd = torch.tensor(sequence_rhs(L, n, 0), device=DEV)
        xd = torch.empty_like(bd)
        sem.sem_solve_projected(m, P, Q, bd, xd, sem.SEM_SOLVER_FLEXCG, tol=1e-12, max_iter=200)
        xs.append(xd.cpu().numpy())
    target = 0.3 * xs[0] - 1.7 * xs[2]
    b = L.ax(target)
    bd = torch.tensor(b, device=DEV)
    xd = torch.empty_like(bd)
    info = sem.sem_solve_projected(m, P, Q, bd, xd, sem.SEM_SOLVER_FLEXCG, tol=1e-8)
    assert info["iters"] == 0 and info["res0"] <= 1e-8 * info["bnorm"]
    assert rel(xd.cpu().numpy(), target) <= 1e-8
    with pytest.raises(sem.SemError):
        sem.Projection(m, 32)


# ---------------------------------------------------------------- Schwarz smoother
@pytest.mark.parametrize("bc,orders,e", [(0, (5, 2, 1), (3, 2, 2)), (1, (7, 3, 1), (2, 3, 2)),
                                         (0, (4, 2), (2, 2, 3)), (1, (3, 1), (4, 3, 2))])
def test_schwarz_vcycle_fp64_matches_oracle(bc, orders, e):
    """Chebyshev-Schwarz smoothing in FP64 with a fixed coarse iteration
    count is a fixed linear map: the GPU (fast diagonalisation) matches the
    oracle (dense local solves) to 1e-10, and so do the Chebyshev intervals
    (Lanczos on M A)."""
    v = inputs.box_vertices(*e, 0.1, 7)
    m = sem.Mesh(*e, orders[0], bc, verts=v)
    P = sem.Pmg(m, orders=orders, smoother_dtype=sem.SEM_F64, coarse_tol=0.0, coarse_maxit=12,
                seed=4, cheb_degree=2, smoother=sem.SEM_SMOOTH_ASM)
    Po = oracle.PMG(*e, list(orders), bc, v, cheb_degree=2, lanczos_steps=20, seed=4,
                    coarse_tol=0.0, coarse_maxit=12, smoother="asm")
    for lvl in range(len(orders) - 1):
        lo, hi = P.lam(lvl)
        olo, ohi = Po.lam(lvl)
        assert abs(hi - ohi) < 1e-10 * ohi and abs(lo - olo) < 1e-10 * olo
    L = Po.levels[0]
    r = L.gs(inputs.random_field(L.nl, 8)) * L.mask
    if bc == 1:
        r -= L.dot(r, np.ones(L.nl)) / L.ng
    zd = torch.empty(L.nl, device=DEV, dtype=torch.float64)
    sem.sem_pmg_vcycle(P, torch.tensor(r, device=DEV), zd)
    assert rel(zd.cpu().numpy(), Po.vcycle(r)) < 1e-10


@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("dtype", [sem.SEM_F64, sem.SEM_F32])
def test_schwarz_flexcg_reaches_1e8(bc, dtype):
    e = (3, 3, 2)
    v = inputs.box_vertices(*e, 0.1, 3)
    m = sem.Mesh(*e, 7, bc, verts=v)
    L = oracle.Level(*e, 7, bc, v)
    b = manufactured(L)[1] if bc == 0 else fourier_rhs(L)
    its = {}
    for sm in (sem.SEM_SMOOTH_JACOBI, sem.SEM_SMOOTH_ASM):
        P = sem.Pmg(m, orders=(7, 3, 1), smoother_dtype=dtype, cheb_degree=3, coarse_tol=1e-2,
                    coarse_maxit=50, smoother=sm)
        bd = torch.tensor(b, device=DEV)
        xd = torch.zeros_like(bd)
        info = sem.sem_solve(m, P, bd, xd, sem.SEM_SOLVER_FLEXCG, tol=1e-8, max_iter=100)
        assert info["status"] == sem.SEM_OK, info
        assert residual(L, b, xd.cpu().numpy()) <= 1.001e-8
        its[sm] = info["iters"]
    assert its[sem.SEM_SMOOTH_ASM] < its[sem.SEM_SMOOTH_JACOBI], its


@pytest.mark.parametrize("bc,orders,e", [(0, (5, 2, 1), (3, 2, 2)), (1, (7, 3, 1), (2, 3, 2)),
                                         (0, (9, 4, 1), (2, 2, 2)), (1, (3, 1), (4, 3, 2))])
def test_schwarz_tc_vcycle_close_to_fp64_oracle(bc, orders, e):
    """Local solves on the tensor cores (TF32 head + remainder products into
    FP32 accumulators): the V-cycle stays within FP32 accuracy of the FP64
    oracle's (dense local solves), like the CUDA-core FP32 Schwarz V-cycle,
    and the Chebyshev intervals are the oracle's."""
    v = inputs.box_vertices(*e, 0.1, 7)
    m = sem.Mesh(*e, orders[0], bc, verts=v)
    Po = oracle.PMG(*e, list(orders), bc, v, cheb_degree=2, lanczos_steps=20, seed=4,
                    coarse_tol=0.0, coarse_maxit=12, smoother="asm")
    L = Po.levels[0]
    r = L.gs(inputs.random_field(L.nl, 8)) * L.mask
    if bc == 1:
        r -= L.dot(r, np.ones(L.nl)) / L.ng
    zo = Po.vcycle(r)
    out = {}
    for sm in (sem.SEM_SMOOTH_ASM, sem.SEM_SMOOTH_ASM_TC):
        P = sem.Pmg(m, orders=orders, smoother_dtype=sem.SEM_F32, coarse_tol=0.0, coarse_maxit=12,
                    seed=4, cheb_degree=2, smoother=sm)
        for lvl in range(len(orders) - 1):
            lo, hi = P.lam(lvl)
            olo, ohi = Po.lam(lvl)
            assert abs(hi - ohi) < 1e-10 * ohi and abs(lo - olo) < 1e-10 * olo
        zd = torch.empty(L.nl, device=DEV, dtype=torch.float64)
        sem.sem_pmg_vcycle(P, torch.tensor(r, device=DEV), zd)
        out[sm] = zd.cpu().numpy()
        assert rel(out[sm], zo) < 1e-4, (sm, rel(out[sm], zo))
    assert rel(out[sem.SEM_SMOOTH_ASM_TC], out[sem.SEM_SMOOTH_ASM]) < 1e-4


@pytest.mark.parametrize("bc", [0, 1])
def test_schwarz_tc_flexcg_reaches_1e8(bc):
    e = (3, 3, 2)
    v = inputs.box_vertices(*e, 0.1, 3)
    m = sem.Mesh(*e, 7, bc, verts=v)
    L = oracle.Level(*e, 7, bc, v)
    b = manufactured(L)[1] if bc == 0 else fourier_rhs(L)
    its = {}
    for sm in (sem.SEM_SMOOTH_ASM, sem.SEM_SMOOTH_ASM_TC):
        P = sem.Pmg(m, orders=(7, 3, 1), smoother_dtype=sem.SEM_F32, cheb_degree=3,
                    coarse_tol=1e-2, coarse_maxit=50, smoother=sm)
        bd = torch.tensor(b, device=DEV)
        xd = torch.zeros_like(bd)
        info = sem.sem_solve(m, P, bd, xd, sem.SEM_SOLVER_FLEXCG, tol=1e-8, max_iter=100)
        assert info["status"] == sem.SEM_OK, info
        assert residual(L, b, xd.cpu().numpy()) <= 1.001e-8
        its[sm] = info["iters"]
    assert abs(its[sem.SEM_SMOOTH_ASM_TC] - its[sem.SEM_SMOOTH_ASM]) <= 1, its


@pytest.mark.parametrize("bc,orders,e", [(0, (5, 2, 1), (3, 2, 2)), (1, (7, 3, 1), (2, 3, 2))])
def test_schwarz_tf32_vcycle_within_tf32_accuracy(bc, orders, e):
    """TF32 local solves (operands rounded once to 11 significant bits, FP32
    accumulation): the V-cycle stays within 1e-2 of the FP64 oracle's, a
    bound a few hundred TF32 unit roundoffs (2^-11) wide."""
    v = inputs.box_vertices(*e, 0.1, 7)
    m = sem.Mesh(*e, orders[0], bc, verts=v)
    Po = oracle.PMG(*e, list(orders), bc, v, cheb_degree=2, lanczos_steps=20, seed=4,
                    coarse_tol=0.0, coarse_maxit=12, smoother="asm")
    L = Po.levels[0]
    r = L.gs(inputs.random_field(L.nl, 8)) * L.mask
    if bc == 1:
        r -= L.dot(r, np.ones(L.nl)) / L.ng
    P = sem.Pmg(m, orders=orders, smoother_dtype=sem.SEM_F32, coarse_tol=0.0, coarse_maxit=12,
                seed=4, cheb_degree=2, smoother=sem.SEM_SMOOTH_ASM_TF32)
    zd = torch.empty(L.nl, device=DEV, dtype=torch.float64)
    sem.sem_pmg_vcycle(P, torch.tensor(r, device=DEV), zd)
    err = rel(zd.cpu().numpy(), Po.vcycle(r))
    assert err < 1e-2, err


@pytest.mark.parametrize("bc", [0, 1])
def test_schwarz_tf32_flexcg_reaches_1e8(bc):
    """The flexible outer CG absorbs the TF32 rounding of the smoother."""
    e = (3, 3, 2)
    v = inputs.box_vertices(*e, 0.1, 3)
    m = sem.Mesh(*e, 7, bc, verts=v)
    L = oracle.Level(*e, 7, bc, v)
    b = manufactured(L)[1] if bc == 0 else fourier_rhs(L)
    its = {}
    for sm in (sem.SEM_SMOOTH_ASM, sem.SEM_SMOOTH_ASM_TF32):
        P = sem.Pmg(m, orders=(7, 3, 1), smoother_dtype=sem.SEM_F32, cheb_degree=3,
                    coarse_tol=1e-2, coarse_maxit=50, smoother=sm)
        bd = torch.tensor(b, device=DEV)
        xd = torch.zeros_like(bd)
        info = sem.sem_solve(m, P, bd, xd, sem.SEM_SOLVER_FLEXCG, tol=1e-8, max_iter=100)
        assert info["status"] == sem.SEM_OK, info
        assert residual(L, b, xd.cpu().numpy()) <= 1.001e-8
        its[sm] = info["iters"]
    assert its[sem.SEM_SMOOTH_ASM_TF32] <= its[sem.SEM_SMOOTH_ASM] + 2, its


def test_schwarz_tc_needs_fp32_smoothing():
    m = sem.Mesh(2, 2, 2, 5, 0)
    for sm in (sem.SEM_SMOOTH_ASM_TC, sem.SEM_SMOOTH_ASM_TF32):
        with pytest.raises(sem.SemError) as ex:
            sem.Pmg(m, orders=(5, 2, 1), smoother_dtype=sem.SEM_F64, smoother=sm)
        assert ex.value.status == sem.SEM_EINVAL


def test_schwarz_order_limit():
    m = sem.Mesh(2, 2, 2, 10, 0)
    with pytest.raises(sem.SemError) as ex:
        sem.Pmg(m, orders=(10, 5, 1), smoother=sem.SEM_SMOOTH_ASM)
    assert ex.value.status == sem.SEM_EINVAL


# ---------------------------------------------------------------- CUDA graph
GRAPH_CASES = [
    # bc, orders, coarse mode, smoother, smoother dtype
    (0, (7, 3, 1), sem.SEM_COARSE_JACOBI, sem.SEM_SMOOTH_JACOBI, sem.SEM_F32),
    (1, (7, 3, 1), sem.SEM_COARSE_MG, sem.SEM_SMOOTH_JACOBI, sem.SEM_F32),
    (0, (5, 3), sem.SEM_COARSE_JACOBI, sem.SEM_SMOOTH_JACOBI, sem.SEM_F64),
    (1, (7, 3, 1), sem.SEM_COARSE_JACOBI, sem.SEM_SMOOTH_ASM, sem.SEM_F32),
    (0, (7, 3, 1), sem.SEM_COARSE_JACOBI, sem.SEM_SMOOTH_JACOBI, sem.SEM_F16),
    (0, (7, 3, 1), sem.SEM_COARSE_JACOBI, sem.SEM_SMOOTH_ASM_TC, sem.SEM_F32),
]


def _graph_problem(bc, orders, e=(5, 4, 3), seed=4):
    v = inputs.box_vertices(*e, 0.1, seed)
    m = sem.Mesh(*e, orders[0], bc, verts=v)
    L = oracle.Level(*e, orders[0], bc, v)
    b = manufactured(L)[1] if bc == 0 else fourier_rhs(L)
    return m, L, b


@pytest.mark.parametrize("bc,orders,cmode,smoother,dtype", GRAPH_CASES)
def test_graph_flexcg_matches_host_loop_bitwise(bc, orders, cmode, smoother, dtype):
    """The device-driven loop runs the same kernels on the same data as the
    host-driven one: same iterations, same bits, on first capture, on replay
    and after a capture for another x."""
    m, L, b = _graph_problem(bc, orders)
    P = sem.Pmg(m, orders=orders, smoother_dtype=dtype, coarse_tol=1e-2, coarse_maxit=60,
                coarse_mode=cmode, smoother=smoother)
    bd = torch.tensor(b, device=DEV)
    xe = torch.zeros_like(bd)
    ie = sem.sem_solve(m, P, bd, xe, sem.SEM_SOLVER_FLEXCG, tol=1e-8, max_iter=100)
    assert ie["status"] == sem.SEM_OK and ie["iters"] >= 3, ie
    for xg in (torch.zeros_like(bd), torch.zeros_like(bd), None):
        if xg is None:
            xg = torch.zeros_like(bd)  # a third buffer: the graph is captured again
        ig = sem.sem_solve(m, P, bd, xg, sem.SEM_SOLVER_FLEXCG, tol=1e-8, max_iter=100,
                           use_graph=True)
        assert ig["status"] == sem.SEM_OK and ig["iters"] == ie["iters"], (ig, ie)
        assert ig["res"] == ie["res"]
        assert torch.equal(xg, xe)
    assert residual(L, b, xg.cpu().numpy()) <= 1.05e-8


def test_graph_launches_are_counted_per_kernel_class():
    """A graph solve's kernels are counted under their own classes (from the
    tally taken at capture, times the replays): the same per-class launch
    counts as the host-driven loop, which launches the same kernels."""
    m, L, b = _graph_problem(1, (7, 3, 1))
    P = sem.Pmg(m, orders=(7, 3, 1), coarse_tol=1e-2, coarse_maxit=60, coarse_mode=sem.SEM_COARSE_MG)
    bd = torch.tensor(b, device=DEV)
    counts = []
    for g in (False, True, True):
        x = torch.zeros_like(bd)
        sem.sem_solve(m, P, bd, x, sem.SEM_SOLVER_FLEXCG, tol=1e-8, max_iter=100, use_graph=g,
                      zero_guess=True)  # warm-up (and the capture)
        sem.sem_trace_enable(True, "")
        sem.sem_trace_read(reset=True)
        info = sem.sem_solve(m, P, bd, x, sem.SEM_SOLVER_FLEXCG, tol=1e-8, max_iter=100,
                             use_graph=g, zero_guess=True)
        tr = sem.sem_trace_read(reset=True)
        sem.sem_trace_enable(False, "")
        assert info["iters"] >= 3
        # the loop's own control kernels (arm, stop) exist only in the graph
        counts.append({k: v["launches"] for k, v in tr.items()
                       if v["launches"] and not k.startswith("graph_ctl")})
    assert counts[1] == counts[0], (counts[0], counts[1])
    assert counts[2] == counts[0]


@pytest.mark.parametrize("max_iter", [1, 2, 3, 5])
def test_graph_flexcg_stops_at_max_iter(max_iter):
    m, L, b = _graph_problem(0, (7, 3, 1))
    P = sem.Pmg(m, orders=(7, 3, 1), coarse_tol=1e-2, coarse_maxit=60)
    bd = torch.tensor(b, device=DEV)
    xe, xg = torch.zeros_like(bd), torch.zeros_like(bd)
    ie = sem.sem_solve(m, P, bd, xe, sem.SEM_SOLVER_FLEXCG, tol=1e-14, max_iter=max_iter)
    ig = sem.sem_solve(m, P, bd, xg, sem.SEM_SOLVER_FLEXCG, tol=1e-14, max_iter=max_iter,
                       use_graph=True)
    assert ie["status"] == ig["status"] == sem.SEM_ENOTCONV
    assert ie["iters"] == ig["iters"] == max_iter
    assert torch.equal(xg, xe)


def test_graph_follows_a_new_pmg_and_nonzero_guess():
    """A second hierarchy on the same mesh is captured afresh; a nonzero
    initial guess goes through the same path."""
    m, L, b = _graph_problem(0, (7, 3, 1))
    bd = torch.tensor(b, device=DEV)
    x0 = L.gs(inputs.random_field(L.nl, 9)) / L.gs(np.ones(L.nl)) * L.mask
    x0 = torch.tensor(x0, device=DEV)
    for degree in (2, 3):
        P = sem.Pmg(m, orders=(7, 3, 1), cheb_degree=degree, coarse_tol=1e-2, coarse_maxit=60)
        xe, xg = x0.clone(), x0.clone()
        ie = sem.sem_solve(m, P, bd, xe, sem.SEM_SOLVER_FLEXCG, tol=1e-9, max_iter=100)
        ig = sem.sem_solve(m, P, bd, xg, sem.SEM_SOLVER_FLEXCG, tol=1e-9, max_iter=100,
                           use_graph=True)
        assert ig["status"] == sem.SEM_OK and ig["iters"] == ie["iters"]
        assert torch.equal(xg, xe)
        P.close()


def test_graph_host_and_projected_solves():
    m, L, b = _graph_problem(1, (7, 3, 1))
    P = sem.Pmg(m, orders=(7, 3, 1), coarse_tol=1e-2, coarse_maxit=60)
    xe, xg = np.zeros(L.nl), np.zeros(L.nl)
    ie = sem.sem_solve_host(m, P, b, xe, sem.SEM_SOLVER_FLEXCG, tol=1e-8)
    ig = sem.sem_solve_host(m, P, b, xg, sem.SEM_SOLVER_FLEXCG, tol=1e-8, use_graph=True)
    assert ie["iters"] == ig["iters"] and np.array_equal(xe, xg)
    Qe, Qg = sem.Projection(m, 4), sem.Projection(m, 4)
    for n in range(6):
        bn = torch.tensor(sequence_rhs(L, n, 1), device=DEV)
        ye, yg = torch.zeros_like(bn), torch.zeros_like(bn)
        je = sem.sem_solve_projected(m, P, Qe, bn, ye, tol=1e-8)
        jg = sem.sem_solve_projected(m, P, Qg, bn, yg, tol=1e-8, use_graph=True)
        assert je["iters"] == jg["iters"] and je["status"] == jg["status"] == sem.SEM_OK
        assert torch.equal(ye, yg)


def test_graph_argument_checks():
    m = sem.Mesh(2, 2, 2, 3, 0)
    P = sem.Pmg(m, orders=(3, 1))
    bd = torch.zeros(m.n_local, device=DEV, dtype=torch.float64)
    xd = torch.zeros_like(bd)
    for solver, pmg in ((sem.SEM_SOLVER_PCG, None), (sem.SEM_SOLVER_FGMRES, P)):
        with pytest.raises(sem.SemError) as ex:
            sem.sem_solve(m, pmg, bd, xd, solver, use_graph=True)
        assert ex.value.status == sem.SEM_EINVAL
    # zero right-hand side: converged before any graph launch
    info = sem.sem_solve(m, P, bd, xd, sem.SEM_SOLVER_FLEXCG, use_graph=True)
    assert info["status"] == sem.SEM_OK and info["iters"] == 0


# ---------------------------------------------------------------- full size
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


@pytest.mark.parametrize("orders,degree", [((7, 4, 2, 1), 3), ((7, 3, 1), 2)])
def test_full_size_solve_residual_sampled_by_oracle(orders, degree):
    """The benchmark's solves (48^3 elements, N = 7, Neumann, pMG 7-4-2-1 with
    Chebyshev(3)-Jacobi and 7-3-1 with Chebyshev(2)-Jacobi in FP32,
    multigrid coarse solve, FlexCG to 1e-8):
    at every node of sampled elements the oracle recomputes the residual
    b - A x from the solution on the box of elements around them, and each
    entry is bounded by the global tolerance (|r_i| <= ||r|| <= 1e-8 ||b||,
    unique-point norms)."""
    e, N = 48, 7
    v = inputs.box_vertices(e, e, e, 0.1, 3)
    m = sem.Mesh(e, e, e, N, 1, verts=v)
    Np3 = (N + 1) ** 3
    u = torch.rand(m.n_local, device=DEV, dtype=torch.float64,
                   generator=torch.Generator(DEV).manual_seed(11)) * 2 - 1
    b = torch.empty_like(u)
    sem.sem_ax(m, sem.SEM_F64, u, b, sem.SEM_AX_ASSEMBLED)  # consistent: 1^T b = 0
    P = sem.Pmg(m, orders=orders, cheb_degree=degree, smoother_dtype=sem.SEM_F32,
                coarse_tol=0.2, coarse_maxit=30, coarse_mode=sem.SEM_COARSE_MG)
    x = torch.zeros_like(b)
    info = sem.sem_solve(m, P, b, x, sem.SEM_SOLVER_FLEXCG, tol=1e-8, max_iter=50)
    assert info["status"] == sem.SEM_OK and info["iters"] <= 12, info
    bnorm = float(np.sqrt(sem.sem_dot(m, b, b)))
    # the GPU's own FP64 residual (its operator is checked against the oracle
    # at this size elsewhere)
    ax = torch.empty_like(x)
    sem.sem_ax(m, sem.SEM_F64, x, ax, sem.SEM_AX_ASSEMBLED)
    r = b - ax
    assert np.sqrt(sem.sem_dot(m, r, r)) <= 1.001e-8 * bnorm
    rng = np.random.Generator(np.random.PCG64(4848))
    cents = [tuple(int(c) for c in rng.integers(0, e, 3)) for _ in range(6)]
    cents += [(0, 0, 0), (e - 1, e - 1, e - 1), (0, e - 1, 17), (23, 0, e - 1)]
    x3 = x.view(-1, Np3)
    b3 = b.view(-1, Np3)
    worst = 0.0
    for c in cents:
        n, sub, els, centre = _sub_box(v, e, e, e, c)
        Lo = oracle.Level(*n, N, 1, sub)
        xs = x3[torch.tensor(els, device=DEV)].cpu().numpy().reshape(-1)
        axo = Lo.ax(xs).reshape(-1, Np3)[centre]
        rc = b3[els[centre]].cpu().numpy() - axo
        worst = max(worst, float(np.max(np.abs(rc))))
    assert worst <= 1.001e-8 * bnorm, (worst, bnorm)


@pytest.mark.parametrize("solver", [sem.SEM_SOLVER_PCG, sem.SEM_SOLVER_FLEXCG,
                                    sem.SEM_SOLVER_FGMRES])
@pytest.mark.parametrize("bc", [0, 1])
def test_zero_guess_equals_zero_filled_guess(solver, bc):
    """zero_guess ignores x's input (here NaN) and gives the bits of a solve
    from a zero-filled x, on device and host buffers."""
    m, L, b = _graph_problem(bc, (7, 3, 1))
    P = None if solver == sem.SEM_SOLVER_PCG else sem.Pmg(m, orders=(7, 3, 1), coarse_tol=1e-2,
                                                         coarse_maxit=60)
    bd = torch.tensor(b, device=DEV)
    x0 = torch.zeros_like(bd)
    i0 = sem.sem_solve(m, P, bd, x0, solver, tol=1e-8, max_iter=2000)
    xn = torch.full_like(bd, float("nan"))
    i1 = sem.sem_solve(m, P, bd, xn, solver, tol=1e-8, max_iter=2000, zero_guess=True)
    assert i0["status"] == i1["status"] == sem.SEM_OK and i0["iters"] == i1["iters"]
    assert torch.equal(x0, xn)
    xh = np.full(L.nl, np.nan)
    i2 = sem.sem_solve_host(m, P, b, xh, solver, tol=1e-8, max_iter=2000, zero_guess=True)
    assert i2["iters"] == i0["iters"] and np.array_equal(xh, x0.cpu().numpy())
    with pytest.raises(sem.SemError):
        d = sem.sem_solve_desc(solver, 1e-8, 10, 1, 0, 0, 2)
        info = sem.sem_solve_info()
        sem.check(sem.lib().sem_solve(m.h, P.h if P else None, sem._ptr(bd), sem._ptr(x0),
                                      sem.C.byref(d), sem.C.byref(info), None))


@pytest.mark.parametrize("solver", [sem.SEM_SOLVER_FLEXCG, sem.SEM_SOLVER_FGMRES])
def test_wait_error_is_reported_by_the_next_solve_and_cleared(solver):
    """A kernel whose bounded wait runs out sets its level's error flag and
    leaves its work undone; the next solve returns SEM_ETIMEOUT and clears the
    flag, and the solve after it runs as before.  The flag is set from the
    host: nothing is made to fail on the device."""
    m, L, b = _graph_problem(0, (7, 3, 1))
    P = sem.Pmg(m, orders=(7, 3, 1), coarse_tol=1e-2, coarse_maxit=60)
    bd = torch.tensor(b, device=DEV)
    ok = sem.sem_solve(m, P, bd, torch.zeros_like(bd), solver, tol=1e-8, max_iter=200)
    assert ok["status"] == sem.SEM_OK
    sem.sem_inject_wait_error(m)
    with pytest.raises(sem.SemError) as ei:
        sem.sem_solve(m, P, bd, torch.zeros_like(bd), solver, tol=1e-8, max_iter=200)
    assert ei.value.status == sem.SEM_ETIMEOUT
    again = sem.sem_solve(m, P, bd, torch.zeros_like(bd), solver, tol=1e-8, max_iter=200)
    assert again["status"] == sem.SEM_OK and again["iters"] == ok["iters"]


def test_wait_error_is_reported_by_vcycle_and_staged_operator():
    """sem_pmg_vcycle and the staged FP32 operator read the wait flags too: a
    flag set from the host turns the next such call into SEM_ETIMEOUT (and is
    cleared), so a later solve on the mesh is not blamed for it."""
    m, L, b = _graph_problem(0, (7, 3, 1))
    P = sem.Pmg(m, orders=(7, 3, 1), coarse_tol=1e-2, coarse_maxit=60)
    bd = torch.tensor(b, device=DEV)
    z = torch.empty_like(bd)
    sem.sem_pmg_vcycle(P, bd, z)
    z_ok = z.clone()
    sem.sem_inject_wait_error(m)
    with pytest.raises(sem.SemError) as ei:
        sem.sem_pmg_vcycle(P, bd, z)
    assert ei.value.status == sem.SEM_ETIMEOUT
    sem.sem_pmg_vcycle(P, bd, z)
    assert torch.equal(z, z_ok)
    u = torch.tensor(inputs.random_field(L.nl, 3), device=DEV, dtype=torch.float32)
    w = torch.empty_like(u)
    sem.sem_inject_wait_error(m)
    with pytest.raises(sem.SemError) as ei:
        sem.sem_ax(m, sem.SEM_F32, u, w, sem.SEM_AX_ASSEMBLED)
    assert ei.value.status == sem.SEM_ETIMEOUT
    sem.sem_ax(m, sem.SEM_F32, u, w, sem.SEM_AX_ASSEMBLED)
    ok = sem.sem_solve(m, P, bd, torch.zeros_like(bd), sem.SEM_SOLVER_FLEXCG, tol=1e-8,
                       max_iter=200)
    assert ok["status"] == sem.SEM_OK
