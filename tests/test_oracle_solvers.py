"""Pins of the oracle's solvers: Jacobi-PCG, Chebyshev smoothing, Lanczos
bounds, the p-multigrid transfers and V-cycle, and flexible CG (CPU only).

Anchors: numpy's dense LAPACK solve and eigensolver on tiny meshes, the closed
form of the Chebyshev error polynomial, exactness of polynomial interpolation,
the adjoint identity between prolongation and restriction, the spectral
convergence of the manufactured problem, and iteration counts that stay flat
as the mesh is refined.
"""

import numpy as np
import pytest

from paper_2110_01716_gb300 import inputs

DIR, NEU = 0, 1


def level(orc, ex, ey, ez, N, bc, seed=3):
    return orc.Level(ex, ey, ez, N, bc, inputs.box_vertices(ex, ey, ez, 0.1, seed))


def dense_unique(L, apply):
    ids = L.ids
    rep = np.full(L.ng, -1)
    for l in range(ids.size - 1, -1, -1):
        rep[ids[l]] = l
    M = np.zeros((L.ng, L.ng))
    for g in range(L.ng):
        M[:, g] = apply((ids == g).astype(np.float64))[rep]
    return M, rep


def manufactured(L):
    X = L.X
    x, y, z = X[:, 0].ravel(), X[:, 1].ravel(), X[:, 2].ravel()
    us = np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)
    return us, L.assembled_rhs(3 * np.pi ** 2 * us)


def test_pcg_matches_dense_solve_dirichlet(orc):
    L = level(orc, 2, 2, 2, 4, DIR)
    A, rep = dense_unique(L, L.ax)
    keep = L.mask[rep] == 1.0
    b = L.gs(inputs.random_field(L.nl, 4)) * L.mask
    x, info = L.pcg(b, tol=1e-14, maxit=1000)
    assert info["status"] == 0
    ref = np.zeros(L.ng)
    ref[keep] = np.linalg.solve(A[np.ix_(keep, keep)], b[rep][keep])
    assert np.max(np.abs(x - ref[L.ids])) < 1e-10 * np.max(np.abs(ref))
    # the converged residual, recomputed, meets the stopping rule
    r = b - L.ax(x)
    assert np.sqrt(L.dot(r, r)) <= 1e-13 * np.sqrt(L.dot(b, b))


def test_pcg_from_a_nonzero_guess_matches_dense_solve(orc):
    """From a nonzero initial guess the solve reaches the same dense solution,
    and its initial residual norm is ||b - A x0|| with A the dense assembled
    matrix (unique-dof numbering)."""
    L = level(orc, 2, 2, 2, 4, DIR)
    A, rep = dense_unique(L, L.ax)
    keep = L.mask[rep] == 1.0
    b = L.gs(inputs.random_field(L.nl, 4)) * L.mask
    x0 = L.gs(inputs.random_field(L.nl, 5)) / L.mult * L.mask
    x, info = L.pcg(b, x0=x0, tol=1e-14, maxit=1000)
    assert info["status"] == 0
    ref = np.zeros(L.ng)
    ref[keep] = np.linalg.solve(A[np.ix_(keep, keep)], b[rep][keep])
    assert np.max(np.abs(x - ref[L.ids])) < 1e-10 * np.max(np.abs(ref))
    r0 = b[rep] - A @ x0[rep]
    assert abs(info["res0"] - np.linalg.norm(r0)) <= 1e-12 * np.linalg.norm(r0)


def test_pcg_neumann_matches_least_squares(orc):
    L = level(orc, 2, 2, 2, 3, NEU)
    A, rep = dense_unique(L, L.ax)
    g = L.gs(inputs.random_field(L.nl, 8))
    b_u = g[rep] - g[rep].mean()  # mean-zero over unique dofs
    b = b_u[L.ids]
    x, info = L.pcg(b, tol=1e-13, maxit=1000)
    assert info["status"] == 0
    ref = np.linalg.lstsq(A, b_u, rcond=None)[0]
    xu = x[rep]
    np.testing.assert_allclose(xu - xu.mean(), ref - ref.mean(), atol=1e-10 * np.abs(ref).max())


def test_pcg_plain_cg_and_zero_rhs(orc):
    L = level(orc, 2, 1, 2, 3, DIR)
    x, info = L.pcg(np.zeros(L.nl), x0=np.ones(L.nl) * L.mask, tol=1e-10)
    # b = 0: the stopping rule is reached only at x = 0
    assert info["res0"] > 0
    b = L.gs(inputs.random_field(L.nl, 2)) * L.mask
    x1, i1 = L.pcg(b, tol=1e-12, precond=True)
    x2, i2 = L.pcg(b, tol=1e-12, precond=False)
    assert i1["status"] == 0 and i2["status"] == 0
    np.testing.assert_allclose(x1, x2, atol=1e-9 * np.abs(x1).max())


def test_pcg_reports_nonconvergence(orc):
    L = level(orc, 2, 2, 2, 5, DIR)
    _, b = manufactured(L)
    x, info = L.pcg(b, tol=1e-12, maxit=3)
    assert info["status"] == 1 and info["iters"] == 3


def test_manufactured_solution_converges_spectrally(orc):
    errs = []
    for N in range(2, 10):
        L = level(orc, 2, 2, 2, N, DIR, seed=1)
        us, b = manufactured(L)
        u, info = L.pcg(b, tol=1e-13, maxit=3000)
        assert info["status"] == 0
        errs.append(np.max(np.abs(u - us * L.mask)))
    errs = np.array(errs)
    # error falls geometrically with N at fixed mesh (exponential convergence)
    assert np.all(errs[1:] < errs[:-1] / 5), errs
    assert errs[-1] < 1e-10


def test_manufactured_solution_at_8cube_order7(orc):
    L = level(orc, 8, 8, 8, 7, DIR, seed=1)
    us, b = manufactured(L)
    u, info = L.pcg(b, tol=1e-10, maxit=2000)
    assert info["status"] == 0
    assert np.max(np.abs(u - us)) < 1e-9


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_chebyshev_error_polynomial_closed_form(orc, k):
    # diagonal operator with a known spectrum; Jacobi scaling d
    n = 40
    rng = np.random.Generator(np.random.PCG64(k))
    d = rng.uniform(0.5, 2.0, n)
    lam = np.linspace(0.05, 1.0, n)  # spectrum of D^-1 A
    a = lam * d
    lo, hi = 0.1, 1.1
    e0 = rng.standard_normal(n)
    xstar = rng.standard_normal(n)
    b = a * xstar
    x0 = xstar - e0
    x = orc.cheb(n, lambda v: a * v, 1.0 / d, b, x0, k, lo, hi, x_zero=False)
    theta, delta = (hi + lo) / 2, (hi - lo) / 2
    T = np.polynomial.chebyshev.Chebyshev.basis(k)
    factor = T((theta - lam) / delta) / T(theta / delta)
    np.testing.assert_allclose(xstar - x, factor * e0, atol=1e-12)
    # starting from zero gives the same as x0 = 0 with x_zero=False
    xa = orc.cheb(n, lambda v: a * v, 1.0 / d, b, np.zeros(n), k, lo, hi, x_zero=True)
    xb = orc.cheb(n, lambda v: a * v, 1.0 / d, b, np.zeros(n), k, lo, hi, x_zero=False)
    np.testing.assert_allclose(xa, xb, atol=1e-13)


@pytest.mark.parametrize("k", [1, 2, 3, 5])
def test_chebyshev_on_MA_error_polynomial_closed_form(orc, k):
    """The Chebyshev smoothing with a general preconditioner M (the form of the
    Schwarz smoother): the error after k steps is
    T_k((theta - M A)/delta) / T_k(theta/delta) times the initial error, for a
    non-diagonal SPD M, evaluated through numpy's eigendecomposition of M A."""
    n = 30
    rng = np.random.Generator(np.random.PCG64(10 + k))
    a = rng.uniform(0.5, 2.0, n)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    M = Q @ np.diag(rng.uniform(0.2, 1.0, n)) @ Q.T
    lam, S = np.linalg.eig(M @ np.diag(a))
    lam, S = lam.real, S.real
    hi = 1.1 * lam.max()
    lo = hi / 10
    e0 = rng.standard_normal(n)
    xstar = rng.standard_normal(n)
    b = a * xstar
    x = orc.cheb_m(n, lambda v: a * v, lambda v: M @ v, b, xstar - e0, k, lo, hi, x_zero=False)
    theta, delta = (hi + lo) / 2, (hi - lo) / 2
    T = np.polynomial.chebyshev.Chebyshev.basis(k)
    factor = T((theta - lam) / delta) / T(theta / delta)
    ref = S @ (factor * np.linalg.solve(S, e0))
    np.testing.assert_allclose(xstar - x, ref, atol=1e-11 * np.abs(e0).max())
    xa = orc.cheb_m(n, lambda v: a * v, lambda v: M @ v, b, np.zeros(n), k, lo, hi, x_zero=True)
    xb = orc.cheb_m(n, lambda v: a * v, lambda v: M @ v, b, np.zeros(n), k, lo, hi,
                    x_zero=False)
    np.testing.assert_allclose(xa, xb, atol=1e-13 * np.abs(xb).max())


@pytest.mark.parametrize("bc", [DIR, NEU])
def test_lanczos_start_vector_from_the_published_generator(orc, bc):
    """The start vector of the Lanczos estimate: 2u - 1 at every copy of global
    node g, u the 53-bit fraction of splitmix64 value g (computed here by the
    input module's generator, pinned to the published stream), masked, and
    under Neumann minus its unique-dof mean."""
    L = level(orc, 3, 2, 2, 4, bc)
    seed = 12345
    v = L.lanczos_start(seed)
    ref = (2.0 * inputs.splitmix64_unit(seed, L.ids.astype(np.uint64)) - 1.0) * L.mask
    if bc == NEU:
        ref = ref - np.sum(ref / L.mult) / np.sum(1.0 / L.mult)
        assert abs(np.sum(v / L.mult)) <= 1e-12 * np.sum(np.abs(v) / L.mult)
    np.testing.assert_allclose(v, ref, rtol=0, atol=1e-15)


@pytest.mark.parametrize("bc", [DIR, NEU])
def test_lanczos_estimate_of_largest_eigenvalue(orc, bc):
    L = level(orc, 2, 2, 2, 4, bc)
    A, rep = dense_unique(L, L.ax)
    d = L.diag()[rep]
    keep = L.mask[rep] == 1.0
    As = A[np.ix_(keep, keep)] / np.sqrt(np.outer(d[keep], d[keep]))
    lmax = np.linalg.eigvalsh(As)[-1]
    est, steps = L.lanczos_max(20, seed=5)
    assert steps == 20
    assert est <= lmax * (1 + 1e-12)
    assert est >= 0.97 * lmax


@pytest.mark.parametrize("Nf,Nc", [(7, 3), (3, 1), (5, 2)])
def test_prolongation_exact_and_restriction_is_its_transpose(orc, Nf, Nc):
    v = inputs.box_vertices(2, 3, 2, 0.1, 6)
    F = orc.Level(2, 3, 2, Nf, NEU, v)
    Cl = orc.Level(2, 3, 2, Nc, NEU, v)
    J = orc.interp(Nf, Nc)
    # physical coordinates are trilinear in (r,s,t): interpolation reproduces them,
    # and products of two coordinates when Nc >= 2
    Xc, Xf = Cl.X, F.X
    fields = [(Xc[:, 0], Xf[:, 0]), (Xc[:, 2], Xf[:, 2])]
    if Nc >= 2:
        fields.append((Xc[:, 0] * Xc[:, 1], Xf[:, 0] * Xf[:, 1]))
    for fc, ff in fields:
        got = orc.interp3(F.E, Nf + 1, Nc + 1, J, fc.ravel())
        np.testing.assert_allclose(got, ff.ravel(), atol=1e-13)
    # <P u_c, v_f>_f = <u_c, R v_f>_c with R v = gs_c(J^T (v / mult_f))
    uc = Cl.gs(inputs.random_field(Cl.nl, 1)) / Cl.mult
    vf = F.gs(inputs.random_field(F.nl, 2)) / F.mult
    Pu = orc.interp3(F.E, Nf + 1, Nc + 1, J, uc)
    Rv = Cl.gs(orc.interp3(F.E, Nf + 1, Nc + 1, J, vf / F.mult, transpose=True))
    lhs, rhs = F.dot(Pu, vf), Cl.dot(uc, Rv)
    assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(lhs))


def test_two_level_vcycle_with_exact_coarse_solve(orc):
    v = inputs.box_vertices(2, 2, 2, 0.1, 2)
    P = orc.PMG(2, 2, 2, [4, 2], DIR, v, cheb_degree=2, coarse_tol=1e-15, coarse_maxit=5000)
    L = P.levels[0]
    M, rep = dense_unique(L, P.vcycle)
    A, _ = dense_unique(L, L.ax)
    keep = L.mask[rep] == 1.0
    M = M[np.ix_(keep, keep)]
    A = A[np.ix_(keep, keep)]
    # exact coarse solve and equal pre/post smoothing: M is symmetric
    assert np.max(np.abs(M - M.T)) < 1e-9 * np.max(np.abs(M))
    Eprop = np.eye(A.shape[0]) - M @ A
    rho = np.max(np.abs(np.linalg.eigvals(Eprop)))
    assert rho < 0.5, rho
    # the smoothing interval brackets the estimate
    lo, hi = P.lam(0)
    assert 0 < lo < hi


def test_flexcg_with_jacobi_equals_pcg(orc):
    v = inputs.box_vertices(3, 2, 2, 0.1, 4)
    P = orc.PMG(3, 2, 2, [5, 1], DIR, v)
    L = P.levels[0]
    _, b = manufactured(L)
    for its in (1, 5, 17):
        xf, fi = P.flexpcg(b, tol=0.0, maxit=its, precond=False)
        xp, pi = L.pcg(b, tol=0.0, maxit=its)
        assert fi["iters"] == pi["iters"] == its
        np.testing.assert_allclose(xf, xp, atol=1e-11 * np.abs(xp).max())


def test_flexcg_updates_are_A_conjugate_with_a_variable_preconditioner(orc):
    """With the flexible coefficient beta = <z', r' - r> / <z, r>, the new
    direction is A-conjugate to the previous one whatever the preconditioner
    did (p' = z' + beta p and A p = (r - r') / alpha give <p', A p> = 0); the
    Fletcher-Reeves coefficient <z', r'> / <z, r> keeps that only for a fixed
    linear preconditioner.  The pMG V-cycle with a coarse CG stopped at a loose
    tolerance is not linear, and FlexCG's successive updates x_{k+1} - x_k
    (parallel to the directions) must still be A-conjugate."""
    v = inputs.box_vertices(3, 3, 3, 0.1, 6)
    P = orc.PMG(3, 3, 3, [5, 2, 1], DIR, v, cheb_degree=2, coarse_tol=0.3, coarse_maxit=50)
    L = P.levels[0]
    _, b = manufactured(L)
    # the preconditioner is not linear here
    r1 = L.gs(L.mask * np.random.default_rng(1).uniform(-1, 1, L.nl)) * L.mask
    r2 = b
    lin = P.vcycle(r1) + P.vcycle(r2) - P.vcycle(r1 + r2)
    assert np.abs(lin).max() > 1e-4 * np.abs(P.vcycle(r1 + r2)).max()
    xs = [np.zeros(L.nl)]
    for its in (1, 2, 3, 4):
        x, info = P.flexpcg(b, tol=0.0, maxit=its)
        assert info["iters"] == its
        xs.append(x)
    d = [xs[k + 1] - xs[k] for k in range(4)]
    for k in range(3):
        Ad = L.ax(d[k])
        num = abs(L.dot(d[k + 1], Ad))
        den = np.sqrt(L.dot(d[k + 1], L.ax(d[k + 1])) * L.dot(d[k], Ad))
        assert num <= 1e-9 * den, (k, num / den)


@pytest.mark.slow
@pytest.mark.parametrize("bc", [DIR, NEU])
def test_pmg_flexcg_iterations_flat_under_refinement(orc, bc):
    """pMG-preconditioned FlexCG at N = 7 from E = 2^3 to 16^3 (4096
    elements, 2.1 M local points): every solve meets 1e-8, recomputed, and
    from 4^3 on the iteration count stays within two of itself."""
    iters = []
    for e in (2, 4, 8, 16):
        v = inputs.box_vertices(e, e, e, 0.1, 3)
        P = orc.PMG(e, e, e, [7, 3, 1], bc, v, cheb_degree=2, coarse_tol=1e-2,
                    coarse_maxit=50)
        L = P.levels[0]
        if bc == DIR:
            _, b = manufactured(L)
        else:
            a, k, phi = inputs.fourier_modes(3)
            X = L.X
            f = sum(a[m] * np.cos(2 * np.pi * (k[m, 0] * X[:, 0] + k[m, 1] * X[:, 1]
                                               + k[m, 2] * X[:, 2]) + phi[m])
                    for m in range(len(a))).ravel()
            b = L.gs(L.B * f)
            b -= L.dot(b, np.ones(L.nl)) / L.dot(np.ones(L.nl), np.ones(L.nl))
        x, info = P.flexpcg(b, tol=1e-8, maxit=200)
        assert info["status"] == 0
        r = b - L.ax(x)
        assert np.sqrt(L.dot(r, r)) <= 1.01e-8 * np.sqrt(L.dot(b, b))
        iters.append(info["iters"])
    assert iters[1] <= iters[0] + 4, iters
    assert max(iters[1:]) - min(iters[1:]) <= 2, iters
    assert max(iters) < 20, iters


# ---------------------------------------------------------------- FGMRES
def _dense_gmres_residuals(A, Minv_diag, r0, kmax):
    """Minimal residual norms of right-preconditioned GMRES, by direct least
    squares over an orthonormalised Krylov basis of A M (numpy QR / lstsq)."""
    AM = A * Minv_diag[None, :]
    cols = [r0 / np.linalg.norm(r0)]
    out = [np.linalg.norm(r0)]
    for k in range(1, kmax + 1):
        Q, _ = np.linalg.qr(np.stack(cols, axis=1))
        W = AM @ Q  # residual b - AM Q c, minimised over c
        c, *_ = np.linalg.lstsq(W, r0, rcond=None)
        out.append(np.linalg.norm(r0 - W @ c))
        v = AM @ cols[-1]
        cols.append(v / np.linalg.norm(v))
    return np.array(out)


def test_fgmres_with_jacobi_is_minimal_residual(orc):
    """With a fixed (Jacobi) preconditioner FGMRES is GMRES on A D^-1: every
    step's residual is the minimum over the Krylov space, computed here by
    dense least squares on the unique unknowns."""
    v = inputs.box_vertices(2, 2, 2, 0.1, 5)
    P = orc.PMG(2, 2, 2, [3, 1], DIR, v)
    L = P.levels[0]
    A, rep = dense_unique(L, L.ax)
    keep = L.mask[rep] == 1.0
    b = L.gs(inputs.random_field(L.nl, 6)) * L.mask
    x, info = P.fgmres(b, tol=0.0, restart=8, maxit=6, precond=False)
    Ak = A[np.ix_(keep, keep)]
    ref = _dense_gmres_residuals(Ak, 1.0 / np.diag(Ak), b[rep][keep], 6)
    np.testing.assert_allclose(info["hist"], ref, rtol=1e-8)
    # the iterate's true residual equals the last least-squares residual
    r = b - L.ax(x)
    assert abs(np.sqrt(L.dot(r, r)) - info["hist"][-1]) <= 1e-10 * info["hist"][0]


def test_fgmres_terminates_within_the_dimension(orc):
    """Without restart GMRES finds the exact solution in at most n steps
    (n = 3 unknowns: a 2x1x1 box of order 2 under Dirichlet)."""
    v = inputs.box_vertices(2, 1, 1, 0.1, 2)
    P = orc.PMG(2, 1, 1, [2, 1], DIR, v)
    L = P.levels[0]
    A, rep = dense_unique(L, L.ax)
    keep = L.mask[rep] == 1.0
    assert keep.sum() == 3
    b = L.gs(inputs.random_field(L.nl, 7)) * L.mask
    x, info = P.fgmres(b, tol=1e-13, restart=10, maxit=10, precond=False)
    assert info["status"] == 0 and info["iters"] <= 3
    ref = np.zeros(L.ng)
    ref[keep] = np.linalg.solve(A[np.ix_(keep, keep)], b[rep][keep])
    assert np.max(np.abs(x - ref[L.ids])) < 1e-11 * np.max(np.abs(ref))


@pytest.mark.parametrize("bc", [DIR, NEU])
def test_fgmres_restarted_and_pmg_preconditioned(orc, bc):
    """pMG-preconditioned FGMRES reaches 1e-8 (residual recomputed), with and
    without restarts, in no more iterations than FlexCG plus one; restarts
    keep the least-squares residuals non-increasing."""
    e = 3
    v = inputs.box_vertices(e, e, e, 0.1, 3)
    P = orc.PMG(e, e, e, [7, 3, 1], bc, v, cheb_degree=2, coarse_tol=1e-2, coarse_maxit=50)
    L = P.levels[0]
    if bc == DIR:
        _, b = manufactured(L)
    else:
        b = L.gs(inputs.random_field(L.nl, 9))
        b -= L.dot(b, np.ones(L.nl)) / L.dot(np.ones(L.nl), np.ones(L.nl))
    xf, fi = P.flexpcg(b, tol=1e-8, maxit=100)
    for restart in (30, 3):
        x, info = P.fgmres(b, tol=1e-8, restart=restart, maxit=100)
        assert info["status"] == 0
        r = b - L.ax(x)
        assert np.sqrt(L.dot(r, r)) <= 1.001e-8 * np.sqrt(L.dot(b, b))
        assert np.all(np.diff(info["hist"]) <= 1e-12 * info["hist"][0])
        if restart == 30:
            assert info["iters"] <= fi["iters"] + 1, (info["iters"], fi["iters"])


# ---------------------------------------------------------------- projection
def _sequence_rhs(L, n, bc, seed=3):
    a, k, phi, om = inputs.fourier_sequence(seed)
    X = L.X
    f = sum(a[m] * np.cos(2 * np.pi * (k[m, 0] * X[:, 0] + k[m, 1] * X[:, 1]
                                       + k[m, 2] * X[:, 2]) + phi[m] + om[m] * n)
            for m in range(len(a))).ravel()
    b = L.gs(L.B * f)
    if bc == DIR:
        return b * L.mask
    return b - L.dot(b, np.ones(L.nl)) / L.dot(np.ones(L.nl), np.ones(L.nl))


def test_projection_basis_is_a_orthonormal_and_best_fit(orc):
    """After a sequence of solves the kept basis is A-orthonormal (dense A from
    numpy), A p_i is stored exactly, and the projected residual equals the
    dense least-squares best fit in the A-norm."""
    e, N = 2, 4
    v = inputs.box_vertices(e, e, e, 0.1, 3)
    P = orc.PMG(e, e, e, [N, 2, 1], DIR, v, coarse_tol=1e-6, coarse_maxit=100)
    L = P.levels[0]
    A, rep = dense_unique(L, L.ax)
    Q = orc.Projection(P, 8)
    for n in range(5):
        Q.solve(_sequence_rhs(L, n, DIR), tol=1e-10)
    k = Q.nvec
    assert k == 5
    Pm = np.stack([Q.vector(i)[0][rep] for i in range(k)], axis=1)
    APm = np.stack([Q.vector(i)[1][rep] for i in range(k)], axis=1)
    np.testing.assert_allclose(A @ Pm, APm, atol=1e-10 * np.abs(APm).max())
    np.testing.assert_allclose(Pm.T @ A @ Pm, np.eye(k), atol=1e-9)
    # best fit of a new right-hand side: dense normal equations in the A-norm
    b = _sequence_rhs(L, 5, DIR)
    c = np.linalg.solve(Pm.T @ A @ Pm, Pm.T @ b[rep])
    rp_ref = np.linalg.norm(b[rep] - A @ Pm @ c)
    x, info = Q.solve(b, tol=1e-10)
    assert abs(info["res_proj"] - rp_ref) <= 1e-9 * np.linalg.norm(b[rep])
    r = b - L.ax(x)
    assert np.sqrt(L.dot(r, r)) <= 1.001e-10 * np.sqrt(L.dot(b, b))


def test_projection_basis_stays_a_orthonormal_after_loose_solves(orc):
    """Solved only to 1e-3, a correction keeps a visible component in the span
    of the basis; the one-pass Gram-Schmidt must still leave the basis
    A-orthonormal, its norm taken as dx^T A dx minus the squared coefficients
    (dense A from numpy)."""
    e, N = 2, 4
    v = inputs.box_vertices(e, e, e, 0.1, 5)
    P = orc.PMG(e, e, e, [N, 2, 1], DIR, v, coarse_tol=1e-6, coarse_maxit=100)
    L = P.levels[0]
    A, rep = dense_unique(L, L.ax)
    Q = orc.Projection(P, 8)
    for n in range(6):
        Q.solve(_sequence_rhs(L, 3 * n, DIR), tol=1e-3)
    k = Q.nvec
    assert k >= 4
    Pm = np.stack([Q.vector(i)[0][rep] for i in range(k)], axis=1)
    np.testing.assert_allclose(Pm.T @ A @ Pm, np.eye(k), atol=1e-9)


def test_projection_of_a_right_hand_side_in_the_span_is_exact(orc):
    e, N = 2, 4
    v = inputs.box_vertices(e, e, e, 0.1, 4)
    P = orc.PMG(e, e, e, [N, 1], DIR, v, coarse_tol=1e-6, coarse_maxit=100)
    L = P.levels[0]
    Q = orc.Projection(P, 8)
    xs = []
    for n in range(3):
        x, _ = Q.solve(_sequence_rhs(L, n, DIR), tol=1e-12)
        xs.append(x)
    target = 0.3 * xs[0] - 1.7 * xs[2]
    b = L.ax(target)
    x, info = Q.solve(b, tol=1e-8)
    assert info["iters"] == 0 and info["res_proj"] <= 1e-8 * np.sqrt(L.dot(b, b))
    assert np.max(np.abs(x - target)) <= 1e-8 * np.max(np.abs(target))


@pytest.mark.parametrize("bc", [DIR, NEU])
@pytest.mark.parametrize("solver", ["flexcg", "fgmres"])
def test_projection_cuts_iterations_on_a_smooth_sequence(orc, bc, solver):
    """Successive right-hand sides varying smoothly: every solve meets the
    tolerance (residual recomputed), later solves need fewer iterations than
    the first, and with Lmax = 3 the space restarts (never more than 3)."""
    e = 3
    v = inputs.box_vertices(e, e, e, 0.1, 3)
    P = orc.PMG(e, e, e, [7, 3, 1], bc, v, cheb_degree=2, coarse_tol=1e-2, coarse_maxit=50)
    L = P.levels[0]
    for Lmax in (30, 3):
        Q = orc.Projection(P, Lmax)
        its = []
        for n in range(8):
            b = _sequence_rhs(L, n, bc)
            x, info = Q.solve(b, tol=1e-8, solver=solver)
            assert info["status"] == 0
            r = b - L.ax(x)
            assert np.sqrt(L.dot(r, r)) <= 1.001e-8 * np.sqrt(L.dot(b, b))
            assert Q.nvec <= Lmax
            its.append(info["iters"])
        assert its[-1] < its[0], its
        if Lmax == 30:
            assert sum(its[4:]) <= sum(its[:4]) - 4, its
