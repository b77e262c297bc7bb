"""GPU parity of the multigrid-preconditioned coarse solve (SEM_COARSE_MG)
against its FP64 oracle (oracle/coarse_mg.py), through sem_pmg_coarse_solve.

The GPU runs the lattice multigrid V(2,2) cycle in FP32 inside an FP64
flexible CG; the oracle runs everything in FP64.  With a fixed iteration
count (coarse_tol 0) the two compute the same iterates up to the FP32
rounding of the preconditioner, so the solutions agree element by element
within TOL_MG (norm-wise, relative): each V-cycle output carries a relative
error of a few 2^-24 (stencils, transfers and the bottom inverse rounded to
FP32 once, FP32 arithmetic), and a few CG steps amplify it by at most the
ratio of the CG coefficients' sensitivities, well below 1e-4 at these sizes.
With a tolerance the iteration counts agree within one and the GPU's
residual, recomputed by the oracle, meets it."""

import numpy as np
import pytest

import oracle
from oracle import coarse_mg as cm
from paper_2110_01716_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2110_01716_gb300 import sem  # noqa: E402

DEV = torch.device("cuda:0")
TOL_MG = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_2110_01716_gb300 import build

    build.build()
    oracle.build()


def setup(ex, ey, ez, bc, maxit, tol=0.0, seed=4):
    v = inputs.box_vertices(ex, ey, ez, 0.1, seed)
    m = sem.Mesh(ex, ey, ez, 3, bc, verts=v)
    P = sem.Pmg(m, orders=(3, 1), smoother_dtype=sem.SEM_F64, coarse_tol=tol, coarse_maxit=maxit,
                coarse_mode=sem.SEM_COARSE_MG)
    L1 = oracle.Level(ex, ey, ez, 1, bc, v)
    rng = np.random.default_rng(seed)
    b = L1.gs(rng.standard_normal(L1.nl)) * L1.mask
    if bc == 1:
        b -= L1.dot(b, np.ones(L1.nl)) / L1.ng
    return m, P, L1, b


# (16, 8, 8): a 17 x 9 x 9 lattice, three multigrid levels; (6, 5, 7): two
@pytest.mark.parametrize("shape", [(16, 8, 8), (6, 5, 7)])
@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("maxit", [1, 3, 8])
def test_coarse_multigrid_iterates_match_oracle(shape, bc, maxit):
    m, P, L1, b = setup(*shape, bc, maxit)
    bd = torch.tensor(b, device=DEV)
    xd = torch.full_like(bd, float("nan"))
    sem.sem_pmg_coarse_solve(P, bd, xd)
    x = xd.cpu().numpy()
    xo, it = cm.coarse_solve(L1, b, 0.0, maxit)
    assert it == maxit
    err = np.abs(x - xo).max() / np.abs(xo).max()
    assert err <= TOL_MG, err
    # copies of every node are identical (continuous output)
    lo = np.full(L1.ng, np.inf)
    hi = np.full(L1.ng, -np.inf)
    np.minimum.at(lo, L1.ids, x)
    np.maximum.at(hi, L1.ids, x)
    assert np.array_equal(lo, hi)


@pytest.mark.parametrize("bc", [0, 1])
def test_coarse_multigrid_meets_its_tolerance(bc):
    tol = 1e-6
    m, P, L1, b = setup(16, 8, 8, bc, 30, tol=tol)
    bd = torch.tensor(b, device=DEV)
    xd = torch.zeros_like(bd)
    sem.sem_pmg_coarse_solve(P, bd, xd)
    it_gpu = P.coarse_iters()
    x = xd.cpu().numpy()
    xo, it = cm.coarse_solve(L1, b, tol, 30)
    assert abs(it_gpu - it) <= 1, (it_gpu, it)
    # residual on the unique nodes, recomputed with the oracle's operator
    A = cm.level0_operator(L1)
    owner = np.zeros(L1.ng, dtype=np.int64)
    owner[L1.ids] = np.arange(L1.nl)
    r0 = b[owner] - (b[owner].mean() if bc == 1 else 0.0)
    r = r0 - A @ x[owner]
    assert np.linalg.norm(r) <= 1.01 * tol * np.linalg.norm(r0)
