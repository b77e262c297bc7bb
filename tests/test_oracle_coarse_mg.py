"""Pins of the coarse-solve oracle (oracle/coarse_mg.py): the lattice
multigrid that preconditions the N = 1 coarse-grid CG.  Each function is
checked against something other than itself: interpolation of linear
functions, the variational (Galerkin) identity through the fine operator,
the energy through the SEM level's own inner product, the Chebyshev error
polynomial in closed form, exact solves by numpy, and, for the V-cycle, the
brute-force symmetry and contraction of its matrix.  A few plausible
mistakes are planted (monkeypatched) to show that the pins catch them."""

import numpy as np
import pytest

import oracle
from oracle import coarse_mg as cm
from paper_2110_01716_gb300 import inputs


@pytest.fixture(scope="module", autouse=True)
def _build():
    oracle.build()


def level1(ex, ey, ez, bc, seed=7):
    return oracle.Level(ex, ey, ez, 1, bc, inputs.box_vertices(ex, ey, ez, 0.1, seed))


def hierarchy(L):
    return cm.Hierarchy(cm.level0_operator(L), L.ex + 1, L.ey + 1, L.ez + 1, L.bc == 0)


def check_prolongation():
    for n in range(3, 12):
        P = cm.prolongation_1d(n)
        c = np.array(cm.coarse_points(n), dtype=float)
        assert np.allclose(P @ c, np.arange(n), atol=0, rtol=0)  # linear functions exactly
        assert np.array_equal(P.sum(axis=1), np.ones(n))


def test_prolongation_interpolates_linear_functions_exactly():
    check_prolongation()


@pytest.mark.parametrize("bc", [0, 1])
def test_level0_operator_energy_symmetry_and_null_space(bc):
    L = level1(4, 3, 5, bc)
    A = cm.level0_operator(L)
    assert np.allclose(A, A.T, atol=1e-14 * np.abs(A).max())
    rng = np.random.default_rng(3)
    keep = cm.level_keep(L)
    v = rng.standard_normal(L.ng) * keep
    # energy through the SEM level's unique-dof inner product (another path)
    u = v[L.ids]
    e_level = L.dot(u, L.ax(u))
    assert abs(v @ A @ v - e_level) <= 1e-12 * abs(e_level)
    k = np.flatnonzero(keep)
    ev = np.linalg.eigvalsh(A[np.ix_(k, k)])
    if bc == 1:
        assert np.abs(A @ np.ones(L.ng)).max() <= 1e-13 * np.abs(A).max()
        assert ev[1] > 1e-8 * ev[-1]  # null space exactly the constants
    else:
        assert ev[0] > 0


@pytest.mark.parametrize("bc", [0, 1])
def test_galerkin_operators_are_variational(bc):
    L = level1(8, 8, 8, bc)
    H = hierarchy(L)
    assert H.nlev >= 2
    rng = np.random.default_rng(5)
    for l in range(H.nlev - 1):
        u = rng.standard_normal(H.A[l + 1].shape[0]) * H.keep[l + 1]
        w = rng.standard_normal(H.A[l + 1].shape[0]) * H.keep[l + 1]
        Pu, Pw = H.P[l] @ u, H.P[l] @ w
        fine = Pu @ (H.A[l] @ Pw)  # through the fine operator
        assert abs(u @ H.A[l + 1] @ w - fine) <= 1e-12 * np.abs(H.A[l]).sum()
        if bc == 1:
            assert np.abs(H.A[l + 1] @ np.ones(len(u))).max() <= 1e-12 * np.abs(H.A[l + 1]).max()


def check_chebyshev():
    lam = np.linspace(0.3, 2.0, 9)
    A = np.diag(lam)
    dinv = np.ones(9)
    lmin, lmax = 0.2, 2.2
    b = np.linspace(1.0, 2.0, 9)
    x = cm.chebyshev(A, dinv, b, np.zeros(9), 2, lmin, lmax, from_zero=True)
    th, de = 0.5 * (lmax + lmin), 0.5 * (lmax - lmin)
    T2 = lambda s: 2 * s * s - 1  # noqa: E731
    p = T2((th - lam) / de) / T2(th / de)  # error polynomial
    assert np.allclose(x, (1 - p) * b / lam, rtol=1e-14, atol=0)
    # from a nonzero start the error is multiplied by the same polynomial
    x0 = np.cos(np.arange(9.0))
    x1 = cm.chebyshev(A, dinv, b, x0, 2, lmin, lmax, from_zero=False)
    xs = b / lam
    assert np.allclose(x1 - xs, p * (x0 - xs), rtol=1e-12, atol=1e-14)


def test_chebyshev_matches_the_closed_form_error_polynomial():
    check_chebyshev()


def check_power_estimate(L):
    H = hierarchy(L)
    for l in range(H.nlev):
        k = np.flatnonzero(H.keep[l])
        A = H.A[l][np.ix_(k, k)]
        d = np.sqrt(H.dinv[l][k])
        lmax = np.linalg.eigvalsh(d[:, None] * A * d[None, :])[-1]
        est = H.lam[l] / 1.1
        assert 0.9 * lmax <= est <= 1.0001 * lmax


@pytest.mark.parametrize("bc", [0, 1])
def test_power_estimate_is_close_to_the_largest_eigenvalue(bc):
    check_power_estimate(level1(6, 7, 5, bc))


def check_bottom(bc):
    L = level1(4, 3, 3, bc)
    A = cm.level0_operator(L)
    keep = cm.level_keep(L)
    inv = cm.bottom_inverse(A, keep, bc == 0)
    rng = np.random.default_rng(9)
    b = rng.standard_normal(L.ng) * keep
    if bc == 1:
        b -= b.mean()
    x = inv @ b
    assert np.allclose(A @ x, b, atol=1e-10 * np.abs(b).max())
    if bc == 1:
        assert abs(x.sum()) <= 1e-10 * np.abs(x).max() * len(x)
    else:
        assert np.all(x[keep == 0] == 0)


@pytest.mark.parametrize("bc", [0, 1])
def test_bottom_solve_is_exact(bc):
    check_bottom(bc)


def vcycle_matrix(H):
    n = H.A[0].shape[0]
    return H.vcycle(np.eye(n))


def check_vcycle(L):
    H = hierarchy(L)
    M = vcycle_matrix(H)
    k = np.flatnonzero(H.keep[0])
    assert np.abs(M - M.T).max() <= 1e-10 * np.abs(M).max()
    E = np.eye(len(k)) - M[np.ix_(k, k)] @ H.A[0][np.ix_(k, k)]
    if L.bc == 1:  # on mean-free vectors
        Q = np.eye(len(k)) - np.ones((len(k), len(k))) / len(k)
        E = Q @ E @ Q
    rho = np.abs(np.linalg.eigvals(E)).max()
    assert rho < 0.6, rho
    return rho


@pytest.mark.parametrize("bc", [0, 1])
def test_vcycle_is_symmetric_and_contracts(bc):
    check_vcycle(level1(8, 8, 8, bc))


def check_two_level_formula(L):
    """With two levels the V(2,2) cycle is x1 = S b, x2 = x1 + C (b - A x1),
    x3 = x2 + S (b - A x2), S the degree-2 Chebyshev operator and
    C = P pinv(A_c) P^T: built here from those matrices (the pseudo-inverse by
    numpy) and compared with the oracle's cycle."""
    H = hierarchy(L)
    assert H.nlev == 2
    n = H.A[0].shape[0]
    I = np.eye(n)
    lam = H.lam[0]
    S = cm.chebyshev(H.A[0], H.dinv[0], I, np.zeros_like(I), 2, lam / 10, lam, from_zero=True)
    k = np.flatnonzero(H.keep[1])
    Ac_inv = np.zeros_like(H.A[1])
    Ac_inv[np.ix_(k, k)] = np.linalg.pinv(H.A[1][np.ix_(k, k)])
    Cc = H.P[0] @ Ac_inv @ H.P[0].T
    A = H.A[0]
    M = S + Cc @ (I - A @ S)
    M = M + S @ (I - A @ M)
    V = H.vcycle(I)
    kk = np.flatnonzero(H.keep[0])
    if L.bc == 1:  # compare on mean-free inputs and outputs
        Q = I - np.ones((n, n)) / n
        M, V = Q @ M @ Q, Q @ V @ Q
    assert np.abs(M - V)[np.ix_(kk, kk)].max() <= 1e-10 * np.abs(M).max()


@pytest.mark.parametrize("bc", [0, 1])
def test_two_level_cycle_matches_its_matrix_formula(bc):
    check_two_level_formula(level1(8, 8, 8, bc))


def check_coarse_solve(L):
    rng = np.random.default_rng(11)
    b = L.gs(rng.standard_normal(L.nl)) * L.mask
    if L.bc == 1:
        b -= L.dot(b, np.ones(L.nl)) / L.ng
    x, it = cm.coarse_solve(L, b, 1e-12, 200)
    A = cm.level0_operator(L)
    owner = np.zeros(L.ng, dtype=np.int64)
    owner[L.ids] = np.arange(L.nl)
    keep = cm.level_keep(L)
    k = np.flatnonzero(keep)
    bu = b[owner]
    if L.bc == 1:
        ref = np.linalg.lstsq(A, bu - bu.mean(), rcond=None)[0]
        ref -= ref.mean()
        xu = x[owner] - x[owner].mean()
    else:
        ref = np.zeros(L.ng)
        ref[k] = np.linalg.solve(A[np.ix_(k, k)], bu[k])
        xu = x[owner]
    assert np.abs(xu - ref).max() <= 1e-9 * np.abs(ref).max()
    assert it < 30
    # one iteration: x_1 = alpha z_0 with alpha = <r,z>/<z,Az>
    H = hierarchy(L)
    r = bu - (bu.mean() if L.bc == 1 else 0.0)
    z = H.vcycle(r)
    x1, it1 = cm.coarse_solve(L, b, 0.0, 1, H)
    assert it1 == 1
    assert np.allclose(x1[owner], (r @ z) / (z @ A @ z) * z, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("bc", [0, 1])
def test_coarse_solve_reaches_the_dense_solution(bc):
    check_coarse_solve(level1(16, 8, 8, bc))


# ---------------------------------------------------------------- planted mistakes

def _bad_prolongation(n):
    c = cm.coarse_points(n)
    P = np.zeros((n, len(c)))
    pos = {f: k for k, f in enumerate(c)}
    for i in range(n):
        if i in pos:
            P[i, pos[i]] = 1.0
        else:
            P[i, pos[i - 1]] = 0.25  # planted: uneven weights
            P[i, pos[i + 1]] = 0.75
    return P


def _bad_chebyshev(A, dinv, b, x, k, lmin, lmax, from_zero):
    dinv = cm._col(dinv, b)
    theta, delta = 0.5 * (lmax + lmin), 0.5 * (lmax - lmin)
    sigma = theta / delta
    rho = 1.0 / sigma
    r = b.copy() if from_zero else b - A @ x
    x = np.zeros_like(b) if from_zero else x.copy()
    d = dinv * r / theta
    x += d
    for _ in range(k - 1):
        rho_new = 1.0 / (2.0 * sigma - rho)
        r = r - A @ d
        d = rho_new * rho * d + (2.0 * rho_new / theta) * (dinv * r)  # planted: theta for delta
        x += d
        rho = rho_new
    return x


def _bad_power(A, dinv, keep):
    g = np.arange(A.shape[0])
    v = np.where(keep > 0, 1.0 + 0.5 * np.sin(0.7 * g + 0.3), 0.0)
    lam = 0.0
    for _ in range(cm.POWER_STEPS):
        v = v / np.sqrt(np.dot(v, v))
        w = A @ v  # planted: D^-1 left out
        lam = float(np.dot(v, w))
        v = w
    return lam


def _bad_bottom(A, keep, dirichlet):
    n = A.shape[0]
    inv = np.zeros((n, n))
    k = np.flatnonzero(keep > 0)
    inv[np.ix_(k, k)] = np.linalg.pinv(A[np.ix_(k, k)]) * 0.5  # planted: wrong scale
    return inv


def _bad_vcycle(self, b, l=0):
    if l == self.nlev - 1:
        return self.bottom @ b
    A, dinv, lam = self.A[l], self.dinv[l], self.lam[l]
    x = cm.chebyshev(A, dinv, b, np.zeros_like(b), 2, lam / 10.0, lam, from_zero=True)
    r = b - A @ x
    bc = 0.5 * (self.P[l].T @ r) * cm._col(self.keep[l + 1], r)  # planted: scaled restriction
    x = x + self.P[l] @ _bad_vcycle(self, bc, l + 1)
    return cm.chebyshev(A, dinv, b, x, 2, lam / 10.0, lam, from_zero=False)


PLANTED = [
    ("prolongation weights", "prolongation_1d", _bad_prolongation, check_prolongation),
    ("Chebyshev coefficient", "chebyshev", _bad_chebyshev, check_chebyshev),
    ("power iteration without D^-1", "power_lambda", _bad_power,
     lambda: check_power_estimate(level1(6, 7, 5, 0))),
    ("bottom scale", "bottom_inverse", _bad_bottom, lambda: check_bottom(1)),
]


@pytest.mark.parametrize("name,attr,bad,check", PLANTED, ids=[p[0] for p in PLANTED])
def test_planted_mistake_fails_a_pin(monkeypatch, name, attr, bad, check):
    monkeypatch.setattr(cm, attr, bad)
    with pytest.raises((AssertionError, np.linalg.LinAlgError)):
        check()


def test_planted_restriction_scale_fails_the_two_level_formula(monkeypatch):
    monkeypatch.setattr(cm.Hierarchy, "vcycle", _bad_vcycle)
    for bc in (0, 1):
        with pytest.raises(AssertionError):
            check_two_level_formula(level1(8, 8, 8, bc))
