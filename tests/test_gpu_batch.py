"""Batched solves (sem_batch): many independent problems, uneven in size and
order, in one CUDA-graph launch.  Each result must equal bit for bit the
standalone sem_solve of the same problem (a mesh from the same request and a
pMG from the batch's description of it), meet the tolerance with its residual
recomputed by the oracle, and stay the same whatever work split the
autotuner picks."""

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
TOL = 1e-8

# (ex, ey, ez, N, bc): orders 2..9, both boundary conditions, ragged boxes
PROBLEMS = [(2, 2, 2, 2, 0), (3, 2, 2, 3, 1), (2, 3, 2, 4, 0), (3, 3, 2, 5, 0), (2, 2, 3, 6, 1),
            (4, 3, 3, 7, 0), (3, 3, 3, 8, 1), (2, 2, 2, 9, 0), (5, 4, 3, 7, 1), (6, 5, 4, 5, 0)]


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_2110_01716_gb300 import build

    build.build()
    oracle.build()


def host_rhs(ex, ey, ez, N, bc, seed):
    """b = gs(B f) for a smooth f on the oracle's level (masked under
    Dirichlet, mean-free under Neumann), and the oracle level itself."""
    v = inputs.box_vertices(ex, ey, ez, 0.1, seed)
    L = oracle.Level(ex, ey, ez, N, bc, v)
    a, k, phi = inputs.fourier_modes(seed)
    X = L.X
    f = sum(a[m] * np.cos(2 * np.pi * (k[m, 0] * X[:, 0] + k[m, 1] * X[:, 1] + k[m, 2] * X[:, 2])
                          + phi[m]) for m in range(len(a))).ravel()
    b = L.gs(L.B * f)
    if bc == 1:
        b -= L.dot(b, np.ones(L.nl)) / L.ng
    else:
        b *= L.mask
    return b, L


def make_batch(problems, smoother=sem.SEM_F32, max_iter=200, **kw):
    reqs, keep, bs, xs, levels = [], [], [], [], []
    for i, (ex, ey, ez, N, bc) in enumerate(problems):
        b, L = host_rhs(ex, ey, ez, N, bc, 10 + i)
        x = np.full(L.nl, np.nan)
        reqs.append(sem.make_request(ex, ey, ez, N, bc, 0.1, 10 + i, b=b, x=x, tol=TOL,
                                     max_iter=max_iter))
        keep += [b, x]
        bs.append(b)
        xs.append(x)
        levels.append(L)
    B = sem.Batch(reqs, smoother_dtype=smoother, keep=keep, **kw)
    return B, bs, xs, levels


def standalone(problem, seed, b, pmg_desc, use_graph, max_iter=200):
    ex, ey, ez, N, bc = problem
    m = sem.Mesh(ex, ey, ez, N, bc, jitter=0.1, seed=seed)
    P = sem.pmg_from_desc(m, pmg_desc)
    bd = torch.tensor(b, device=DEV)
    x = torch.full_like(bd, float("nan"))
    info = sem.sem_solve(m, P, bd, x, sem.SEM_SOLVER_FLEXCG, tol=TOL, max_iter=max_iter,
                         zero_guess=True, use_graph=use_graph, raise_on_notconv=False)
    out = x.cpu().numpy()
    P.close()
    m.close()
    return out, info


@pytest.mark.parametrize("smoother", [sem.SEM_F32, sem.SEM_F64])
def test_batch_equals_standalone_solves_bit_for_bit(smoother):
    B, bs, xs, levels = make_batch(PROBLEMS, smoother=smoother)
    infos = B.solve()
    for i, p in enumerate(PROBLEMS):
        assert infos[i]["status"] == sem.SEM_OK
        xr, inf_r = standalone(p, 10 + i, bs[i], B.pmg_desc(i), use_graph=(i % 2 == 0))
        assert inf_r["iters"] == infos[i]["iters"], (p, inf_r, infos[i])
        assert np.array_equal(xr, xs[i]), p
        assert infos[i]["res"] == inf_r["res"] and infos[i]["res0"] == inf_r["res0"]
        # the residual recomputed by the oracle meets the tolerance
        L = levels[i]
        r = bs[i] - L.ax(xs[i])
        assert np.sqrt(L.dot(r, r)) <= 1.01 * TOL * np.sqrt(L.dot(bs[i], bs[i])), p
    # a second launch gives the same bits
    first = [x.copy() for x in xs]
    infos2 = B.solve()
    assert [f["iters"] for f in infos2] == [f["iters"] for f in infos]
    for a, c in zip(first, xs):
        assert np.array_equal(a, c)
    B.close()


def test_autotuned_work_split_changes_no_bit():
    probs = PROBLEMS[:6]
    B, bs, xs, _ = make_batch(probs)
    B.solve()
    before = [x.copy() for x in xs]
    chosen, ms = B.autotune(candidates=(2.0, 0.5, 0.0625), reps=2)
    assert ms > 0
    assert all(v in (2.0, 0.5, 0.0625) for v in chosen.values())
    infos = B.solve()
    assert all(f["status"] == sem.SEM_OK for f in infos)
    for a, c in zip(before, xs):
        assert np.array_equal(a, c)
    info = B.info()
    assert info["dev_bytes"] > 0 and info["graph_nodes"] >= 2 * len(probs)
    B.close()


def test_batch_reports_enotconv_like_the_standalone_solve():
    probs = [(3, 3, 2, 5, 0), (2, 2, 3, 6, 1)]
    B, bs, xs, _ = make_batch(probs, max_iter=2)
    infos = B.solve(raise_on_fail=False)
    for i, p in enumerate(probs):
        assert infos[i]["status"] == sem.SEM_ENOTCONV and infos[i]["iters"] == 2
        xr, inf_r = standalone(p, 10 + i, bs[i], B.pmg_desc(i), use_graph=False, max_iter=2)
        assert np.array_equal(xr, xs[i])
    with pytest.raises(sem.SemError) as ei:
        B.solve()
    assert ei.value.status == sem.SEM_ENOTCONV
    B.close()


def test_batch_manufactured_rhs_and_invalid_requests():
    reqs = [sem.make_request(3, 3, 3, 7, sem.SEM_DIRICHLET, 0.1, 5, tol=TOL),
            sem.make_request(2, 3, 2, 5, sem.SEM_DIRICHLET, 0.1, 6, tol=TOL)]
    xs = []
    for r, (ex, ey, ez, N) in zip(reqs, [(3, 3, 3, 7), (2, 3, 2, 5)]):
        x = np.zeros(ex * ey * ez * (N + 1) ** 3)
        r.x = x.ctypes.data
        xs.append(x)
    B = sem.Batch(reqs, keep=xs)
    infos = B.solve()
    for x, (ex, ey, ez, N, seed), f in zip(xs, [(3, 3, 3, 7, 5), (2, 3, 2, 5, 6)], infos):
        L = oracle.Level(ex, ey, ez, N, 0, inputs.box_vertices(ex, ey, ez, 0.1, seed))
        X = L.X
        us = (np.sin(np.pi * X[:, 0]) * np.sin(np.pi * X[:, 1]) * np.sin(np.pi * X[:, 2])).ravel()
        b = L.assembled_rhs(3 * np.pi ** 2 * us)
        r = b - L.ax(x)
        assert np.sqrt(L.dot(r, r)) <= 1.05 * TOL * np.sqrt(L.dot(b, b))
        assert np.max(np.abs(x - us * L.mask)) < 1e-3
        assert f["status"] == sem.SEM_OK
    B.close()
    # a Neumann right-hand side that is not mean-free is rejected at creation
    v = np.ones(2 * 2 * 2 * 4 ** 3)
    with pytest.raises(sem.SemError) as ei:
        sem.Batch([sem.make_request(2, 2, 2, 3, sem.SEM_NEUMANN, 0.1, 1, b=v)], keep=[v])
    assert ei.value.status == sem.SEM_EINVAL
