"""The continuous-batching server (sem_server_*, sem_submit, sem_poll) on
batches of independent problems of mixed sizes and orders.

* Every result meets its tolerance (residual recomputed by the oracle) and,
  for host-given right-hand sides, equals bit for bit the direct sem_solve of
  the same problem: the solves are deterministic, so neither concurrency nor
  the worker count changes a bit.
* The manufactured right-hand side built on the device gives the oracle's
  manufactured solution to discretisation accuracy.
* Poll semantics, setup reuse, the memory budget and the autotuner.
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
# (ex, ey, ez, N, seed): mixed sizes and orders, a few shapes repeated
BATCH = [(2, 2, 2, 5, 1), (3, 2, 2, 7, 2), (4, 4, 3, 3, 3), (2, 3, 2, 9, 4), (3, 3, 3, 7, 5),
         (2, 2, 2, 5, 1), (5, 4, 4, 5, 6), (3, 2, 2, 7, 2), (2, 2, 3, 4, 7), (4, 3, 3, 7, 8)]


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_2110_01716_gb300 import build

    build.build()
    oracle.build()


def _problem(ex, ey, ez, N, seed):
    v = inputs.box_vertices(ex, ey, ez, 0.1, seed)
    L = oracle.Level(ex, ey, ez, N, 0, v)
    X = L.X
    us = (np.sin(np.pi * X[:, 0]) * np.sin(np.pi * X[:, 1]) * np.sin(np.pi * X[:, 2])).ravel()
    return L, us, L.assembled_rhs(3 * np.pi ** 2 * us)


def _residual(L, b, x):
    r = b - L.ax(x)
    return np.sqrt(L.dot(r, r)) / np.sqrt(L.dot(b, b))


def _run(workers, problems, solver=sem.SEM_SOLVER_FLEXCG, **kw):
    S = sem.Server(workers=workers, **kw)
    xs, tickets = [], []
    for (ex, ey, ez, N, seed), (L, us, b) in zip(BATCH, problems):
        x = np.zeros(L.nl)
        xs.append(x)
        tickets.append(S.submit(ex, ey, ez, N, sem.SEM_DIRICHLET, 0.1, seed, b=b, x=x,
                                solver=solver, tol=1e-8))
    infos = [S.wait(t) for t in tickets]
    stats = S.stats()
    S.close()
    return xs, infos, stats


@pytest.mark.parametrize("solver", [sem.SEM_SOLVER_FLEXCG, sem.SEM_SOLVER_FGMRES])
def test_batch_results_meet_tolerance_and_equal_direct_solves(solver):
    problems = [_problem(*p) for p in BATCH]
    xs, infos, stats = _run(4, problems, solver=solver)
    assert stats["completed"] == len(BATCH) and stats["failed"] == 0
    assert stats["setups_built"] + stats["setups_reused"] == len(BATCH)
    for (ex, ey, ez, N, seed), (L, us, b), x, info in zip(BATCH, problems, xs, infos):
        assert info["status"] == sem.SEM_OK, info
        assert _residual(L, b, x) <= 1.001e-8
        assert info["time_ms"] > 0
    # the direct solve of one problem with the same hierarchy: the same bits
    (ex, ey, ez, N, seed), (L, us, b) = BATCH[4], problems[4]
    m = sem.Mesh(ex, ey, ez, N, 0, jitter=0.1, seed=seed)
    P = sem.Pmg(m, orders=(N, N // 2, 1), cheb_degree=3, smoother_dtype=sem.SEM_F32,
                coarse_tol=1e-1, coarse_maxit=30, coarse_mode=sem.SEM_COARSE_MG)
    bd = torch.tensor(b, device=DEV)
    xd = torch.zeros_like(bd)
    sem.sem_solve(m, P, bd, xd, solver, tol=1e-8, max_iter=200)
    assert np.array_equal(xd.cpu().numpy(), xs[4])


def test_worker_count_changes_no_bit():
    problems = [_problem(*p) for p in BATCH]
    x1, _, s1 = _run(1, problems)
    x6, _, s6 = _run(6, problems, cache_per_shape=0)
    for a, b in zip(x1, x6):
        assert np.array_equal(a, b)
    assert s6["setups_reused"] == 0 and s6["setups_built"] == len(BATCH)


def test_manufactured_rhs_on_device_solves_the_manufactured_problem():
    S = sem.Server(workers=2)
    out = []
    for ex, N in ((4, 7), (3, 9)):
        L, us, b = _problem(ex, ex, ex, N, 11)
        x = np.zeros(L.nl)
        t = S.submit(ex, ex, ex, N, sem.SEM_DIRICHLET, 0.1, 11, x=x, tol=1e-12, max_iter=400)
        out.append((L, us, b, x, t))
    for L, us, b, x, t in out:
        info = S.wait(t)
        assert info["status"] == sem.SEM_OK
        # the device right-hand side is the oracle's up to rounding: the solution
        # meets the oracle's system to 1e-10 and approximates sin sin sin
        assert _residual(L, b, x) <= 1e-10
        assert np.max(np.abs(x - us)) < 1e-5
    S.close()


def test_poll_semantics_cache_and_budget():
    S = sem.Server(workers=2, hbm_budget=1, cache_per_shape=1)  # budget 1 byte: one at a time
    t = [S.submit(3, 3, 2, 5, sem.SEM_DIRICHLET, 0.1, 5, tol=1e-8) for _ in range(3)]
    for tk in t:
        info = S.wait(tk)
        assert info["status"] == sem.SEM_OK
        with pytest.raises(sem.SemError) as ex:  # the ticket is released
            S.poll(tk)
        assert ex.value.status == sem.SEM_EINVAL
    st = S.stats()
    assert st["completed"] == 3 and st["setups_built"] + st["setups_reused"] == 3
    assert st["setups_built"] >= 1
    for bad in (dict(N=0), dict(N=12)):
        with pytest.raises(sem.SemError) as ex:
            S.submit(2, 2, 2, bad["N"], sem.SEM_DIRICHLET, 0.1, 1)
        assert ex.value.status == sem.SEM_EINVAL
    with pytest.raises(sem.SemError):  # the manufactured right-hand side is Dirichlet
        S.submit(2, 2, 2, 3, sem.SEM_NEUMANN, 0.1, 1)
    S.close()


def test_cache_reuses_setups_of_one_shape():
    S = sem.Server(workers=1, cache_per_shape=1)
    for _ in range(3):
        assert S.wait(S.submit(3, 2, 2, 7, sem.SEM_DIRICHLET, 0.1, 9))["status"] == sem.SEM_OK
    st = S.stats()
    assert st["setups_built"] == 1 and st["setups_reused"] == 2
    assert st["hbm_in_use"] > 0
    S.close()


def test_autotune_picks_a_worker_count():
    reqs = [sem.make_request(ex, ey, ez, N, sem.SEM_DIRICHLET, 0.1, seed)
            for ex, ey, ez, N, seed in BATCH]
    w, rate = sem.server_autotune(reqs, max_workers=4, cache_per_shape=0)
    assert w in (1, 2, 4) and rate > 0


def test_graph_requests_equal_host_loop_requests():
    """FlexCG requests with use_graph give the same bits as without, with
    setups reused across requests (the graph is captured per setup)."""
    problems = [_problem(*p) for p in BATCH]
    xs, infos, _ = _run(3, problems)
    S = sem.Server(workers=3)
    xg, tickets = [], []
    for (ex, ey, ez, N, seed), (L, us, b) in zip(BATCH, problems):
        x = np.zeros(L.nl)
        xg.append(x)
        tickets.append(S.submit(ex, ey, ez, N, sem.SEM_DIRICHLET, 0.1, seed, b=b, x=x,
                                tol=1e-8, use_graph=True))
    ig = [S.wait(t) for t in tickets]
    S.close()
    for a, b_, ia, ib in zip(xs, xg, infos, ig):
        assert ib["status"] == sem.SEM_OK and ia["iters"] == ib["iters"]
        assert np.array_equal(a, b_)
    with pytest.raises(sem.SemError):
        S2 = sem.Server(workers=1)
        try:
            S2.submit(2, 2, 2, 3, sem.SEM_DIRICHLET, 0.1, 1, solver=sem.SEM_SOLVER_PCG,
                      use_graph=True)
        finally:
            S2.close()


def test_admission_counts_measured_setup_bytes():
    """After a new shape's first solve the server holds that setup's measured
    device bytes (mesh with its workspaces, hierarchy, b and x), not the
    first estimate of 200 bytes per local point + 64 MiB; a reuse adds
    nothing; an unseen shape of a measured order is admitted from the
    measured bytes per point."""
    S = sem.Server(workers=1, cache_per_shape=1)
    ex, ey, ez, N = 3, 3, 2, 5
    nl = ex * ey * ez * (N + 1) ** 3
    S.wait(S.submit(ex, ey, ez, N, sem.SEM_DIRICHLET, 0.1, 7, tol=1e-8))
    st = S.stats()
    held = st["hbm_in_use"]
    assert held > 0 and held != 200 * nl + (64 << 20)
    assert held < 200 * nl + (64 << 20)  # far below the first estimate at this size
    S.wait(S.submit(ex, ey, ez, N, sem.SEM_DIRICHLET, 0.1, 7, tol=1e-8))
    st2 = S.stats()
    assert st2["setups_reused"] == 1 and st2["hbm_in_use"] == held
    S.close()
