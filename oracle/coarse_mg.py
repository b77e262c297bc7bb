"""FP64 oracle of the multigrid-preconditioned coarse solve (N = 1 level).

TEST INFRASTRUCTURE ONLY: imported by the tests, never by the library.

The paper treats its N = 1 coarse grid with algebraic multigrid on the host
(Sec. 4, Table 1: the coarse grid falls from 45 % to 11 % of the run once it
is handled well) and does not give that solver's construction.  The reading
taken here, stated once:

* Unknowns: the values at the vertices of the box, i.e. the unique nodes of
  the N = 1 level (lattice of (ex+1)(ey+1)(ez+1) points, node
  gx + nx (gy + ny gz)).  Level 0 operator: the assembled N = 1 SEM
  stiffness matrix on those nodes; under Dirichlet boundary nodes are
  eliminated (their rows and columns are zero on every level).
* Coarsening by two per direction: the coarse points of a 1D lattice of n
  points are the even indices and the last; a fine point between two coarse
  points takes half of each (linear interpolation in index space).
  Prolongation P = Pz (x) Py (x) Px, restriction P^T, Galerkin operators
  A_c = P^T A P.  Levels are added while the lattice has more than 128
  unknowns, more than 3 points in every direction and fewer than 8 levels.
* Smoothing: Chebyshev (degree 2) acceleration of point Jacobi on
  [lambda/10, lambda], lambda = 1.1 x the estimate of lambda_max(D^-1 A) by
  30 power iterations from v_g = 1 + sin(0.7 g + 0.3)/2 (kept nodes; Saad,
  Iterative Methods, Alg. 12.1 for the recurrence); one V(2,2) cycle: the
  pre-smoothing starts from zero, the post-smoothing from the corrected x.
* Bottom: the dense operator of the last level solved exactly; under
  Neumann the operator plus c 1 1^T (c = mean diagonal / n), which is exact
  on mean-free right-hand sides; under Dirichlet the kept unknowns only.
* Outer iteration: flexible CG (Notay; beta = -alpha <z_new, A p> / rho) in
  FP64 on level 0 from x = 0, preconditioned by one V-cycle per iteration;
  under Neumann the right-hand side first loses its mean; stop when
  <r, r> <= tol^2 <r0, r0> or after maxit iterations.

Every step is written out on dense matrices in the order above, so that a
reader can check it against the description; nothing here is shared with the
CUDA library.
"""

from __future__ import annotations

import numpy as np

MAX_BOTTOM = 128
MAX_LEVELS = 8
POWER_STEPS = 30


def coarse_points(n: int) -> list:
    """Indices of the coarse points of a 1D lattice of n points."""
    c = list(range(0, n, 2))
    if c[-1] != n - 1:
        c.append(n - 1)
    return c


def prolongation_1d(n: int) -> np.ndarray:
    """n x nc linear interpolation in index space."""
    c = coarse_points(n)
    P = np.zeros((n, len(c)))
    pos = {f: k for k, f in enumerate(c)}
    for i in range(n):
        if i in pos:
            P[i, pos[i]] = 1.0
        else:
            P[i, pos[i - 1]] = 0.5
            P[i, pos[i + 1]] = 0.5
    return P


def lattice_keep(nx: int, ny: int, nz: int, dirichlet: bool) -> np.ndarray:
    """1 for unknowns, 0 for eliminated (Dirichlet boundary) nodes."""
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    k = np.ones((nz, ny, nx))
    if dirichlet:
        bnd = (x == 0) | (y == 0) | (z == 0) | (x == nx - 1) | (y == ny - 1) | (z == nz - 1)
        k[bnd] = 0.0
    return k.ravel()


def level0_operator(level) -> np.ndarray:
    """Dense assembled N = 1 stiffness matrix on the lattice nodes (columns by
    unit vectors through the oracle level's assembled operator), with the
    eliminated nodes' rows and columns zero."""
    ids = level.ids
    n = level.ng
    A = np.zeros((n, n))
    owner = np.zeros(n, dtype=np.int64)
    owner[ids] = np.arange(level.nl)  # some local copy of every node
    for g in range(n):
        e = np.zeros(n)
        e[g] = 1.0
        A[:, g] = level.ax(e[ids])[owner]
    keep = level_keep(level)
    return A * keep[:, None] * keep[None, :]


def level_keep(level) -> np.ndarray:
    nx, ny, nz = level.ex + 1, level.ey + 1, level.ez + 1
    return lattice_keep(nx, ny, nz, level.bc == 0)


class Hierarchy:
    """Levels, transfers, smoother bounds and the bottom solve of the lattice
    multigrid built from level 0's operator A0 on an nx x ny x nz lattice."""

    def __init__(self, A0: np.ndarray, nx: int, ny: int, nz: int, dirichlet: bool):
        self.dirichlet = dirichlet
        self.A = [A0]
        self.dims = [(nx, ny, nz)]
        self.keep = [lattice_keep(nx, ny, nz, dirichlet)]
        self.P = []
        while (len(self.A) < MAX_LEVELS and self.A[-1].shape[0] > MAX_BOTTOM
               and min(self.dims[-1]) > 3):
            fx, fy, fz = self.dims[-1]
            P = np.kron(prolongation_1d(fz), np.kron(prolongation_1d(fy), prolongation_1d(fx)))
            cdims = (len(coarse_points(fx)), len(coarse_points(fy)), len(coarse_points(fz)))
            kf, kc = self.keep[-1], lattice_keep(*cdims, dirichlet)
            Af = self.A[-1] * kf[:, None] * kf[None, :]
            Ac = P.T @ Af @ P
            self.A.append(Ac * kc[:, None] * kc[None, :])
            self.P.append(P)
            self.dims.append(cdims)
            self.keep.append(kc)
        self.dinv = []
        self.lam = []
        for l, A in enumerate(self.A):
            d = np.diag(A)
            self.dinv.append(np.where((self.keep[l] > 0) & (d != 0), 1.0 / np.where(d != 0, d, 1), 0))
            self.lam.append(1.1 * power_lambda(A, self.dinv[-1], self.keep[l]))
        self.bottom = bottom_inverse(self.A[-1], self.keep[-1], dirichlet)

    @property
    def nlev(self):
        return len(self.A)

    def vcycle(self, b: np.ndarray, l: int = 0) -> np.ndarray:
        """One V(2,2) cycle for A_l x = b from x = 0 (b may be a block of
        column vectors)."""
        if l == self.nlev - 1:
            return self.bottom @ b
        A, dinv, lam = self.A[l], self.dinv[l], self.lam[l]
        x = chebyshev(A, dinv, b, np.zeros_like(b), 2, lam / 10.0, lam, from_zero=True)
        r = b - A @ x
        bc = (self.P[l].T @ r) * _col(self.keep[l + 1], r)
        x = x + self.P[l] @ self.vcycle(bc, l + 1)
        return chebyshev(A, dinv, b, x, 2, lam / 10.0, lam, from_zero=False)


def power_lambda(A: np.ndarray, dinv: np.ndarray, keep: np.ndarray) -> float:
    """Estimate of lambda_max(D^-1 A) by POWER_STEPS power iterations."""
    g = np.arange(A.shape[0])
    v = np.where(keep > 0, 1.0 + 0.5 * np.sin(0.7 * g + 0.3), 0.0)
    lam = 0.0
    for _ in range(POWER_STEPS):
        nv = np.sqrt(np.dot(v, v))
        if nv == 0.0:
            return 1.0
        v = v / nv
        w = dinv * (A @ v)
        lam = float(np.dot(v, w))
        v = w
    return lam


def _col(v, like):
    """v (one value per node) shaped to scale like (a vector or a block of
    column vectors)."""
    return v if like.ndim == 1 else v[:, None]


def chebyshev(A, dinv, b, x, k, lmin, lmax, from_zero):
    """k steps of Chebyshev-accelerated Jacobi on [lmin, lmax] (Saad,
    Alg. 12.1): d_0 = D^-1 r / theta, then d_{m+1} = rho_{m+1} rho_m d_m +
    (2 rho_{m+1} / delta) D^-1 r_{m+1}, x += d each step.  b and x may be
    blocks of column vectors."""
    dinv = _col(dinv, b)
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
        d = rho_new * rho * d + (2.0 * rho_new / delta) * (dinv * r)
        x += d
        rho = rho_new
    return x


def bottom_inverse(A: np.ndarray, keep: np.ndarray, dirichlet: bool) -> np.ndarray:
    """Dense inverse of the last level (kept unknowns only; Neumann: of
    A + c 1 1^T, c = mean diagonal / n)."""
    n = A.shape[0]
    Ad = A.copy()
    if not dirichlet:
        Ad = Ad + (np.trace(A) / n) / n * np.ones((n, n))
    inv = np.zeros((n, n))
    k = np.flatnonzero(keep > 0)
    inv[np.ix_(k, k)] = np.linalg.inv(Ad[np.ix_(k, k)])
    return inv


def coarse_solve(level, b_local: np.ndarray, tol: float, maxit: int, H: Hierarchy = None):
    """The coarse solve of a pMG V-cycle on the N = 1 level: b_local is the
    assembled E-layout right-hand side; returns (x_local, iterations)."""
    ids = level.ids
    n = level.ng
    owner = np.zeros(n, dtype=np.int64)
    owner[ids] = np.arange(level.nl)
    if H is None:
        H = Hierarchy(level0_operator(level), level.ex + 1, level.ey + 1, level.ez + 1,
                      level.bc == 0)
    A = H.A[0]
    r = b_local[owner].copy()
    if level.bc == 1:
        r -= r.mean()
    x = np.zeros(n)
    z = H.vcycle(r)
    rho = float(np.dot(r, z))
    bb = float(np.dot(r, r))
    p = z.copy()
    it = 0
    if bb > 0.0 and maxit > 0 and rho != 0.0:
        while True:
            it += 1
            w = A @ p
            alpha = rho / float(np.dot(p, w))
            x += alpha * p
            r -= alpha * w
            z = H.vcycle(r)
            rz, zw, rr = float(np.dot(r, z)), float(np.dot(z, w)), float(np.dot(r, r))
            if not (rr > tol * tol * bb) or it >= maxit or rr != rr or rz == 0.0:
                break
            beta = -alpha * zw / rho
            rho = rz
            p = z + beta * p
    return x[ids], it
