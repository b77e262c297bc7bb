"""Pins of the oracle's 1D basis, mesh geometry and numbering (CPU only).

Each check ties the oracle to something other than itself: closed forms from
the textbook GLL rule, numpy/scipy polynomial routines, exact integrals, and
counting arguments on the box lattice.
"""

import math
import os

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

from paper_2110_01716_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "gll_closed_forms.txt")


def _golden_gll():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        n, xs, ws = [t.strip() for t in line.split("|")]
        env = {"sqrt": math.sqrt}
        rows.append((int(n), [eval(t, env) for t in xs.split(",")],
                     [eval(t, env) for t in ws.split(",")]))
    return rows


@pytest.mark.parametrize("N,xs,ws", _golden_gll())
def test_gll_closed_forms(orc, N, xs, ws):
    x, w = orc.gll(N)
    np.testing.assert_allclose(x, xs, rtol=0, atol=1e-15)
    np.testing.assert_allclose(w, ws, rtol=1e-14, atol=0)


@pytest.mark.parametrize("N", range(1, 17))
def test_gll_nodes_are_roots_of_legendre_derivative(orc, N):
    x, w = orc.gll(N)
    assert x[0] == -1.0 and x[-1] == 1.0
    if N >= 2:
        c = np.zeros(N + 1)
        c[N] = 1.0
        roots = np.sort(npleg.legroots(npleg.legder(c)))
        np.testing.assert_allclose(x[1:-1], roots, atol=1e-13)
    # weights from numpy's Legendre evaluation
    c = np.zeros(N + 1)
    c[N] = 1.0
    PN = npleg.legval(x, c)
    np.testing.assert_allclose(w, 2.0 / (N * (N + 1) * PN ** 2), rtol=1e-13)


@pytest.mark.parametrize("N", range(1, 13))
def test_gll_quadrature_exact_to_degree_2N_minus_1(orc, N):
    x, w = orc.gll(N)
    assert abs(w.sum() - 2.0) < 1e-14
    for p in range(0, 2 * N):
        exact = 0.0 if p % 2 else 2.0 / (p + 1)
        assert abs(np.dot(w, x ** p) - exact) < 1e-13, p
    # degree 2N is not integrated exactly (it is a Lobatto, not a Gauss, rule)
    p = 2 * N
    assert abs(np.dot(w, x ** p) - 2.0 / (p + 1)) > 1e-9


@pytest.mark.parametrize("N", range(1, 13))
def test_dhat_matches_closed_form_and_differentiates_polynomials(orc, N):
    D = orc.dhat(N)
    x, _ = orc.gll(N)
    c = np.zeros(N + 1)
    c[N] = 1.0
    P = npleg.legval(x, c)
    # closed form: D_il = P_N(x_i) / (P_N(x_l)(x_i - x_l)), D_00 = -N(N+1)/4, D_NN = N(N+1)/4
    ref = np.zeros((N + 1, N + 1))
    for i in range(N + 1):
        for l in range(N + 1):
            if i != l:
                ref[i, l] = P[i] / (P[l] * (x[i] - x[l]))
    ref[0, 0] = -N * (N + 1) / 4.0
    ref[N, N] = N * (N + 1) / 4.0
    np.testing.assert_allclose(D, ref, atol=1e-11 * max(1, N * N))
    for p in range(0, N + 1):
        exact = p * x ** (p - 1) if p > 0 else np.zeros_like(x)
        np.testing.assert_allclose(D @ x ** p, exact, atol=1e-11 * N * N)
    np.testing.assert_allclose(D.sum(axis=1), 0.0, atol=1e-12 * N * N)
    # centro-antisymmetry of the GLL derivative matrix
    np.testing.assert_allclose(D[::-1, ::-1], -D, atol=1e-12 * N * N)


@pytest.mark.parametrize("Nf,Nc", [(7, 3), (3, 1), (9, 5), (5, 5), (8, 6), (6, 4), (4, 1)])
def test_interp_exact_on_coarse_polynomials(orc, Nf, Nc):
    from scipy.interpolate import BarycentricInterpolator

    J = orc.interp(Nf, Nc)
    xf, _ = orc.gll(Nf)
    xc, _ = orc.gll(Nc)
    np.testing.assert_allclose(J.sum(axis=1), 1.0, atol=1e-14)
    for p in range(Nc + 1):
        np.testing.assert_allclose(J @ xc ** p, xf ** p, atol=1e-13)
    # column j = coarse Lagrange basis j evaluated at the fine nodes (scipy)
    for j in range(Nc + 1):
        e = np.zeros(Nc + 1)
        e[j] = 1.0
        np.testing.assert_allclose(J[:, j], BarycentricInterpolator(xc, e)(xf), atol=1e-13)
    if Nf == Nc:
        np.testing.assert_allclose(J, np.eye(Nf + 1), atol=1e-15)


def test_box_vertices_generator():
    v = inputs.box_vertices(3, 2, 4, jitter=0.1, seed=7)
    assert v.shape == (4 * 3 * 5, 3)
    lat = np.stack(np.meshgrid(np.arange(5) / 4, np.arange(3) / 2, np.arange(4) / 3,
                               indexing="ij"), -1)[..., ::-1].reshape(-1, 3)
    d = v - lat
    assert np.all(np.abs(d) <= 0.1 * np.array([1 / 3, 1 / 2, 1 / 4]) + 1e-15)
    interior = np.all((lat > 0) & (lat < 1), axis=1)
    assert np.all(d[~interior] == 0.0)
    assert np.all(np.abs(d[interior]) > 0)
    # splitmix64 first outputs for seed 0 (published reference stream of the
    # generator: 0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F)
    got = inputs.splitmix64(0, np.arange(3, dtype=np.uint64))
    assert [int(g) for g in got] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_oracle_splitmix64_reference_stream(orc):
    """The oracle's own generator (the Lanczos start vector) against the
    published reference stream of splitmix64 for seed 0, and the stream
    offset: value i of seed s is value 0 of seed s + i * gamma."""
    ref = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    assert [orc.lib().orc_splitmix64(0, i) for i in range(3)] == ref
    gamma = 0x9E3779B97F4A7C15
    assert orc.lib().orc_splitmix64(2 * gamma % 2**64, 0) == ref[2]


@pytest.mark.parametrize("N", [2, 3, 5, 7])
def test_geometry_volume_and_moments_on_jittered_cube(orc, N):
    ex, ey, ez = 3, 2, 4
    v = inputs.box_vertices(ex, ey, ez, 0.1, seed=11)
    G, B, X = orc.geometry(ex, ey, ez, N, v)
    assert np.all(B > 0)
    # the jittered box tiles the unit cube, det J is quadratic per direction
    assert abs(B.sum() - 1.0) < 1e-13
    x, y, z = X[:, 0], X[:, 1], X[:, 2]
    assert abs((B * x).sum() - 0.5) < 1e-13
    if N >= 3:  # degree 4 per direction: needs 2N-1 >= 4
        assert abs((B * y * z).sum() - 0.25) < 1e-13
        assert abs((B * x * x).sum() - 1.0 / 3.0) < 1e-13
    # corners of every element are its vertices
    Np = N + 1
    corner = [0, N, N * Np, N + N * Np, N * Np * Np]
    for e, (ix, iy, iz) in enumerate([(a, b, c) for c in range(ez) for b in range(ey)
                                      for a in range(ex)]):
        vid = lambda a, b, c: (ix + a) + (ex + 1) * ((iy + b) + (ey + 1) * (iz + c))
        ref = [v[vid(0, 0, 0)], v[vid(1, 0, 0)], v[vid(0, 1, 0)], v[vid(1, 1, 0)],
               v[vid(0, 0, 1)]]
        for p, r in zip(corner, ref):
            np.testing.assert_allclose(X[e, :, p], r, atol=1e-15)


def test_geometry_undeformed_closed_form(orc):
    ex, ey, ez, N = 2, 3, 4, 4
    v = inputs.box_vertices(ex, ey, ez, 0.0, seed=0)
    G, B, X = orc.geometry(ex, ey, ez, N, v)
    _, w = orc.gll(N)
    W = np.einsum("k,j,i->kji", w, w, w).ravel()
    hx, hy, hz = 1 / ex, 1 / ey, 1 / ez
    jac = hx * hy * hz / 8
    for e in range(G.shape[0]):
        np.testing.assert_allclose(B[e], W * jac, rtol=1e-14)
        np.testing.assert_allclose(G[e, 0], W * jac * (2 / hx) ** 2, rtol=1e-14)
        np.testing.assert_allclose(G[e, 3], W * jac * (2 / hy) ** 2, rtol=1e-14)
        np.testing.assert_allclose(G[e, 5], W * jac * (2 / hz) ** 2, rtol=1e-14)
        for f in (1, 2, 4):
            assert np.max(np.abs(G[e, f])) < 1e-14 * np.max(G[e, 0])


def test_folded_element_is_rejected(orc):
    v = inputs.box_vertices(2, 2, 2, 0.0, seed=0)
    v = v.copy()
    centre = 1 + 3 * (1 + 3 * 1)
    v[centre, 0] = 1.2  # push the centre vertex through the x = 1 face
    with pytest.raises(ValueError):
        orc.geometry(2, 2, 2, 3, v)


@pytest.mark.parametrize("ex,ey,ez,N", [(1, 1, 1, 2), (2, 3, 4, 3), (4, 4, 4, 7), (3, 1, 2, 1)])
def test_numbering_and_multiplicity_counts(orc, ex, ey, ez, N):
    ids = orc.global_ids(ex, ey, ez, N)
    ng = (ex * N + 1) * (ey * N + 1) * (ez * N + 1)
    assert ids.min() == 0 and ids.max() == ng - 1
    assert np.unique(ids).size == ng
    mult = orc.gs(ids, ng, np.ones(ids.size))
    cnt = np.bincount(ids, minlength=ng)
    np.testing.assert_array_equal(mult, cnt[ids])
    # expected histogram of multiplicities on the lattice of element corners
    vals, counts = np.unique(cnt, return_counts=True)
    hist = dict(zip(vals.tolist(), counts.tolist()))
    n8 = (ex - 1) * (ey - 1) * (ez - 1)
    assert hist.get(8, 0) == n8
    n4 = (N - 1) * ((ex - 1) * (ey - 1) * ez + (ex - 1) * ey * (ez - 1) + ex * (ey - 1) * (ez - 1))
    # interior element edges carry N-1 nodes each, plus vertices on the box faces
    n4 += 2 * ((ex - 1) * (ey - 1) + (ey - 1) * (ez - 1) + (ex - 1) * (ez - 1))
    assert hist.get(4, 0) == n4
    assert sum(v * c for v, c in hist.items()) == ids.size
