"""Pins of the oracle's overlapping Schwarz smoother (CPU only).

Anchors: on undeformed boxes the SEM stiffness is exactly separable, so
(1) on one element under Dirichlet conditions the local problem is the whole
problem and the preconditioner is the exact inverse, and (2) on two elements
the local operator equals the principal submatrix of the assembled operator
(dense, from the oracle's own pinned Ax) on the extended points; plus
symmetry and positivity of the additive combination and convergence of
Chebyshev-Schwarz-preconditioned FlexCG.
"""

import numpy as np
import pytest

from paper_2110_01716_gb300 import inputs

DIR, NEU = 0, 1


def test_one_undeformed_element_is_solved_exactly(orc):
    for N in (3, 5):
        v = inputs.box_vertices(1, 1, 1, 0.0, 1)
        L = orc.Level(1, 1, 1, N, DIR, v)
        M = orc.ASM(L)
        u = L.gs(inputs.random_field(L.nl, 3)) / L.mult * L.mask  # continuous, masked
        z = M.apply(L.ax(u))
        assert np.max(np.abs(z - u)) <= 1e-11 * np.max(np.abs(u))


def _dense_assembled(L):
    ids = L.ids
    rep = np.full(L.ng, -1)
    for l in range(ids.size - 1, -1, -1):
        rep[ids[l]] = l
    A = np.zeros((L.ng, L.ng))
    for g in range(L.ng):
        A[:, g] = L.ax((ids == g).astype(np.float64))[rep]
    return A


@pytest.mark.parametrize("ex,ey", [(2, 1), (1, 2)])
def test_local_operator_is_the_assembled_operator_on_the_extended_points(orc, ex, ey):
    """Two undeformed elements of different lengths (Neumann): element 0's
    local operator on the points that carry data equals the assembled
    operator there (the remaining extended points are decoupled)."""
    N = 4
    v = inputs.box_vertices(ex, ey, 1, 0.0, 1).reshape(-1, 3).copy()
    # stretch the second element: vertex coordinates along the split direction
    d = 0 if ex == 2 else 1
    v[:, d] = np.where(v[:, d] > 0.75, 1.6, v[:, d])
    L = orc.Level(ex, ey, 1, N, NEU, v)
    M = orc.ASM(L)
    K = M.local_matrix(0)
    A = _dense_assembled(L)
    n = N + 3
    Np = N + 1
    # extended points of element 0 that carry data, and their global nodes
    keep, nodes = [], []
    for c in range(n):
        for b in range(n):
            for a in range(n):
                idx = [a - 1, b - 1, c - 1]
                out = [q for q in range(3) if idx[q] < 0 or idx[q] > N]
                if len(out) > 1:
                    continue
                if out:
                    q = out[0]
                    if q != d or idx[q] < 0:
                        continue  # no neighbour on that side
                    gx = [idx[0], idx[1], idx[2]]
                    gx[q] = N + 1  # first point past the shared face in global numbering
                else:
                    gx = idx
                g = gx[0] + (ex * N + 1) * (gx[1] + (ey * N + 1) * gx[2])
                keep.append(a + n * (b + n * c))
                nodes.append(g)
    keep, nodes = np.array(keep), np.array(nodes)
    np.testing.assert_allclose(K[np.ix_(keep, keep)], A[np.ix_(nodes, nodes)],
                               atol=1e-12 * np.abs(A).max())
    # every other point is decoupled: identity rows and columns
    rest = np.setdiff1d(np.arange(n ** 3), keep)
    sub = K[np.ix_(rest, keep)]
    assert np.all(sub == 0.0)


@pytest.mark.parametrize("bc", [DIR, NEU])
def test_schwarz_preconditioner_is_symmetric_positive(orc, bc):
    v = inputs.box_vertices(3, 2, 2, 0.1, 4)
    L = orc.Level(3, 2, 2, 4, bc, v)
    M = orc.ASM(L)
    rng = np.random.Generator(np.random.PCG64(9))
    u = L.gs(rng.uniform(-1, 1, L.nl)) / L.mult * L.mask
    w = L.gs(rng.uniform(-1, 1, L.nl)) / L.mult * L.mask
    Mu, Mw = M.apply(u), M.apply(w)
    assert abs(L.dot(Mu, w) - L.dot(u, Mw)) <= 1e-12 * np.sqrt(L.dot(Mu, Mu) * L.dot(w, w))
    assert L.dot(Mu, u) > 0
    # continuous output (copies equal)
    assert np.max(np.abs(L.gs(Mu) / L.mult - Mu)) <= 1e-14 * np.max(np.abs(Mu))


@pytest.mark.parametrize("bc", [DIR, NEU])
def test_chebyshev_schwarz_pmg_converges_faster_than_jacobi(orc, bc):
    e = 3
    v = inputs.box_vertices(e, e, e, 0.1, 3)
    its = {}
    for sm in ("jacobi", "asm"):
        P = orc.PMG(e, e, e, [5, 2, 1], bc, v, cheb_degree=2, coarse_tol=1e-2,
                    coarse_maxit=50, smoother=sm)
        L = P.levels[0]
        b = L.gs(L.B * np.cos(2 * np.pi * L.X[:, 0].ravel()) * np.sin(np.pi * L.X[:, 1].ravel()))
        if bc == DIR:
            b = b * L.mask
        else:
            b = b - L.dot(b, np.ones(L.nl)) / L.dot(np.ones(L.nl), np.ones(L.nl))
        x, info = P.flexpcg(b, tol=1e-8, maxit=100)
        assert info["status"] == 0
        r = b - L.ax(x)
        assert np.sqrt(L.dot(r, r)) <= 1.001e-8 * np.sqrt(L.dot(b, b))
        its[sm] = info["iters"]
    assert its["asm"] < its["jacobi"], its
