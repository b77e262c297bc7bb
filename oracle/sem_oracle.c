/*
 * sem_oracle.c -- plain, slow, FP64 CPU oracle of the SEM pressure-Poisson path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the smoke check and the benchmark's CPU
 * baseline leg do.  It shares no code, header, table or constant with the
 * CUDA library: every formula below is written out again from the paper
 * (Fischer et al., "Highly Optimized Full-Core Reactor Simulations on
 * Summit") and from the textbook definitions it relies on.
 *
 * Paper passages followed (section / equation):
 *   Sec. 2, Eq. (2) "field1"  tensor-product Lagrange basis on GLL points and the
 *                             isoparametric map x = x^e(r,s,t)
 *   Sec. 2, footnote 1        derivative matrix Dhat_il = dh_l/dr at xi_i and the
 *                             contraction u_r,ijk = sum_l Dhat_il u_ljk
 *   Sec. 2 (C0 continuity)    direct stiffness summation over shared nodes
 *   Sec. 3 (Stokes substep)   Jacobi-preconditioned CG
 *   Sec. 3 (pMG paragraph)    u_f = (J x J x J) u_c, Chebyshev-accelerated
 *                             point-Jacobi smoothing, 32-bit preconditioner option
 *   Sec. 3 (FlexCG/GMRES)     flexible CG for the nonsymmetric pMG preconditioner
 *   Sec. 3 (gs paragraph)     global vertex ids define the exchange pattern
 * Readings where the paper is silent (each stated at its function):
 *   geometric factors of a trilinear map, the inner product over unique dofs,
 *   the stopping norm, Chebyshev bounds from a Lanczos estimate, the coarse
 *   solve (Jacobi-PCG in FP64), restriction as the transpose of prolongation.
 *
 * Layouts: an element-local ("E-layout") vector holds E*(N+1)^3 doubles,
 * element-major, point (i,j,k) at i + Np*(j + Np*k) with i along r.  The six
 * geometric factors of an element are stored factor-major: G[e][f][point],
 * f = 0..5 <-> (rr, rs, rt, ss, st, tt).
 *
 * Every loop is scalar.  The only parallelism is an optional OpenMP loop over
 * elements in the local operator, which does not change any result.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846

/* ------------------------------------------------------------------ */
/* 1D basis (Sec. 2, Eq. 2 and footnote 1)                             */
/* ------------------------------------------------------------------ */

/* Legendre P_n(x) and its derivative by the three-term recurrences
 *   (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1},  P'_{k+1} = P'_{k-1} + (2k+1) P_k. */
static void legendre_pd(int n, double x, double *p, double *dp) {
  double p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0;
  if (n == 0) { *p = 1.0; *dp = 0.0; return; }
  for (int k = 1; k < n; ++k) {
    double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
    double d2 = d0 + (2.0 * k + 1.0) * p1;
    p0 = p1; p1 = p2; d0 = d1; d1 = d2;
  }
  *p = p1; *dp = d1;
}

double orc_legendre(int n, double x) {
  double p, dp;
  legendre_pd(n, x, &p, &dp);
  return p;
}

/* Gauss-Lobatto-Legendre nodes and weights of order N (N+1 points).
 * Nodes: -1, +1 and the N-1 roots of P'_N, found by Newton's method from the
 * Chebyshev-Gauss-Lobatto guesses -cos(pi i / N); the second derivative comes
 * from Legendre's equation (1-x^2) P'' = 2x P' - N(N+1) P.
 * Weights: w_i = 2 / (N (N+1) P_N(xi_i)^2).  Returns 0, or -1 if N < 1. */
int orc_gll(int N, double *xi, double *w) {
  if (N < 1) return -1;
  xi[0] = -1.0;
  xi[N] = 1.0;
  for (int i = 1; i < N; ++i) {
    double x = -cos(ORC_PI * i / N);
    for (int it = 0; it < 100; ++it) {
      double p, dp;
      legendre_pd(N, x, &p, &dp);
      double d2p = (2.0 * x * dp - N * (N + 1.0) * p) / (1.0 - x * x);
      double dx = dp / d2p;
      x -= dx;
      if (fabs(dx) < 1e-15) break;
    }
    xi[i] = x;
  }
  for (int i = 0; i <= N; ++i) {
    double p = orc_legendre(N, xi[i]);
    w[i] = 2.0 / (N * (N + 1.0) * p * p);
  }
  return 0;
}

/* Lagrange basis h_j on the nodes z[0..n] evaluated at x. */
static double lagrange(int n, const double *z, int j, double x) {
  double h = 1.0;
  for (int m = 0; m <= n; ++m)
    if (m != j) h *= (x - z[m]) / (z[j] - z[m]);
  return h;
}

/* Derivative h_j'(x) of the Lagrange basis, by the product rule. */
static double lagrange_deriv(int n, const double *z, int j, double x) {
  double s = 0.0;
  for (int m = 0; m <= n; ++m) {
    if (m == j) continue;
    double t = 1.0 / (z[j] - z[m]);
    for (int q = 0; q <= n; ++q)
      if (q != j && q != m) t *= (x - z[q]) / (z[j] - z[q]);
    s += t;
  }
  return s;
}

/* Derivative matrix (Sec. 2, footnote 1): D[i*(N+1)+l] = h_l'(xi_i). */
void orc_dhat(int N, const double *xi, double *D) {
  for (int i = 0; i <= N; ++i)
    for (int l = 0; l <= N; ++l) D[i * (N + 1) + l] = lagrange_deriv(N, xi, l, xi[i]);
}

/* Interpolation matrix (Sec. 3, pMG): J[i*(Nc+1)+j] = h_j^{(Nc)}(xi_i^{(Nf)}),
 * the coarse Lagrange basis evaluated at the fine GLL nodes. */
void orc_interp(int Nf, const double *xf, int Nc, const double *xc, double *J) {
  for (int i = 0; i <= Nf; ++i)
    for (int j = 0; j <= Nc; ++j) J[i * (Nc + 1) + j] = lagrange(Nc, xc, j, xf[i]);
}

/* ------------------------------------------------------------------ */
/* Mesh: box of ex*ey*ez trilinear hexes (Sec. 2, isoparametric map)   */
/* ------------------------------------------------------------------ */

/* Coordinates and geometric factors at the GLL points of every element.
 * verts: vertex grid [(ex+1)(ey+1)(ez+1)][3], vertex (a,b,c) at a + (ex+1)(b + (ey+1)c).
 * Element e = ix + ex (iy + ey iz); its corner (a,b,c) in {0,1}^3 is vertex
 * (ix+a, iy+b, iz+c).  The map is x(r,s,t) = sum_abc X_abc l_a(r) l_b(s) l_c(t),
 * l_0 = (1-r)/2, l_1 = (1+r)/2 (the isoparametric map of Sec. 2 restricted to
 * trilinear elements; the paper's meshes are curved, these are not).
 * Reading of "six geometric factors per point": with Jac_md = dx_m/dr_d and
 * W = w_i w_j w_k det(Jac),  G_de = W sum_m (Jac^{-1})_dm (Jac^{-1})_em,
 * the symmetric 3x3 metric that turns reference gradients into the physical
 * stiffness integrand; B = W is the diagonal GLL mass.
 * Outputs (any may be NULL): G [E][6][Np^3], B [E][Np^3], X [E][3][Np^3].
 * Returns 0, or -1 if some det(Jac) <= 0. */
int orc_geometry(int ex, int ey, int ez, int N, const double *verts, double *G, double *B,
                 double *X) {
  int Np = N + 1, Np3 = Np * Np * Np;
  double *xi = malloc(sizeof(double) * Np), *w = malloc(sizeof(double) * Np);
  orc_gll(N, xi, w);
  int bad = 0;
  for (int iz = 0; iz < ez; ++iz)
    for (int iy = 0; iy < ey; ++iy)
      for (int ix = 0; ix < ex; ++ix) {
        int64_t e = ix + (int64_t)ex * (iy + (int64_t)ey * iz);
        double V[2][2][2][3];
        for (int c = 0; c < 2; ++c)
          for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a) {
              int64_t v = (ix + a) + (int64_t)(ex + 1) * ((iy + b) + (int64_t)(ey + 1) * (iz + c));
              for (int m = 0; m < 3; ++m) V[c][b][a][m] = verts[3 * v + m];
            }
        for (int k = 0; k < Np; ++k)
          for (int j = 0; j < Np; ++j)
            for (int i = 0; i < Np; ++i) {
              double r = xi[i], s = xi[j], t = xi[k];
              double lr[2] = {(1 - r) / 2, (1 + r) / 2}, ls[2] = {(1 - s) / 2, (1 + s) / 2},
                     lt[2] = {(1 - t) / 2, (1 + t) / 2};
              double dl[2] = {-0.5, 0.5};
              double x[3] = {0, 0, 0}, Jac[3][3] = {{0}};
              for (int c = 0; c < 2; ++c)
                for (int b = 0; b < 2; ++b)
                  for (int a = 0; a < 2; ++a)
                    for (int m = 0; m < 3; ++m) {
                      double Xv = V[c][b][a][m];
                      x[m] += Xv * lr[a] * ls[b] * lt[c];
                      Jac[m][0] += Xv * dl[a] * ls[b] * lt[c];
                      Jac[m][1] += Xv * lr[a] * dl[b] * lt[c];
                      Jac[m][2] += Xv * lr[a] * ls[b] * dl[c];
                    }
              double det = Jac[0][0] * (Jac[1][1] * Jac[2][2] - Jac[1][2] * Jac[2][1]) -
                           Jac[0][1] * (Jac[1][0] * Jac[2][2] - Jac[1][2] * Jac[2][0]) +
                           Jac[0][2] * (Jac[1][0] * Jac[2][1] - Jac[1][1] * Jac[2][0]);
              if (!(det > 0)) bad = 1;
              /* inverse by the adjugate: Inv[d][m] = cofactor(m,d) / det */
              double Inv[3][3];
              Inv[0][0] = (Jac[1][1] * Jac[2][2] - Jac[1][2] * Jac[2][1]) / det;
              Inv[0][1] = (Jac[0][2] * Jac[2][1] - Jac[0][1] * Jac[2][2]) / det;
              Inv[0][2] = (Jac[0][1] * Jac[1][2] - Jac[0][2] * Jac[1][1]) / det;
              Inv[1][0] = (Jac[1][2] * Jac[2][0] - Jac[1][0] * Jac[2][2]) / det;
              Inv[1][1] = (Jac[0][0] * Jac[2][2] - Jac[0][2] * Jac[2][0]) / det;
              Inv[1][2] = (Jac[0][2] * Jac[1][0] - Jac[0][0] * Jac[1][2]) / det;
              Inv[2][0] = (Jac[1][0] * Jac[2][1] - Jac[1][1] * Jac[2][0]) / det;
              Inv[2][1] = (Jac[0][1] * Jac[2][0] - Jac[0][0] * Jac[2][1]) / det;
              Inv[2][2] = (Jac[0][0] * Jac[1][1] - Jac[0][1] * Jac[1][0]) / det;
              double W = w[i] * w[j] * w[k] * det;
              int64_t p = i + Np * (j + Np * k);
              if (G) {
                const int dd[6] = {0, 0, 0, 1, 1, 2}, ee[6] = {0, 1, 2, 1, 2, 2};
                for (int f = 0; f < 6; ++f) {
                  double g = 0.0;
                  for (int m = 0; m < 3; ++m) g += Inv[dd[f]][m] * Inv[ee[f]][m];
                  G[(e * 6 + f) * Np3 + p] = W * g;
                }
              }
              if (B) B[e * Np3 + p] = W;
              if (X)
                for (int m = 0; m < 3; ++m) X[(e * 3 + m) * Np3 + p] = x[m];
            }
      }
  free(xi);
  free(w);
  return bad ? -1 : 0;
}

/* Global id of every local node (Sec. 3, gs paragraph: the user provides a
 * global id per vertex).  On the box, local node (i,j,k) of element
 * (ix,iy,iz) is global lattice point (ix N + i, iy N + j, iz N + k), numbered
 * x-fastest on the (ex N + 1)(ey N + 1)(ez N + 1) lattice. */
void orc_global_ids(int ex, int ey, int ez, int N, int64_t *ids) {
  int Np = N + 1;
  int64_t nx = (int64_t)ex * N + 1, ny = (int64_t)ey * N + 1;
  for (int iz = 0; iz < ez; ++iz)
    for (int iy = 0; iy < ey; ++iy)
      for (int ix = 0; ix < ex; ++ix) {
        int64_t e = ix + (int64_t)ex * (iy + (int64_t)ey * iz);
        for (int k = 0; k < Np; ++k)
          for (int j = 0; j < Np; ++j)
            for (int i = 0; i < Np; ++i) {
              int64_t gx = (int64_t)ix * N + i, gy = (int64_t)iy * N + j, gz = (int64_t)iz * N + k;
              ids[e * Np * Np * Np + i + Np * (j + Np * k)] = gx + nx * (gy + ny * gz);
            }
      }
}

/* Dirichlet mask: 0 at nodes on the boundary of the box, 1 elsewhere
 * (bc = 0 Dirichlet); all ones for bc = 1 (Neumann). */
void orc_mask(int ex, int ey, int ez, int N, int bc, double *mask) {
  int Np = N + 1;
  for (int iz = 0; iz < ez; ++iz)
    for (int iy = 0; iy < ey; ++iy)
      for (int ix = 0; ix < ex; ++ix) {
        int64_t e = ix + (int64_t)ex * (iy + (int64_t)ey * iz);
        for (int k = 0; k < Np; ++k)
          for (int j = 0; j < Np; ++j)
            for (int i = 0; i < Np; ++i) {
              int64_t gx = (int64_t)ix * N + i, gy = (int64_t)iy * N + j, gz = (int64_t)iz * N + k;
              int onb = gx == 0 || gy == 0 || gz == 0 || gx == (int64_t)ex * N ||
                        gy == (int64_t)ey * N || gz == (int64_t)ez * N;
              mask[e * Np * Np * Np + i + Np * (j + Np * k)] = (bc == 0 && onb) ? 0.0 : 1.0;
            }
      }
}

/* ------------------------------------------------------------------ */
/* Operators                                                            */
/* ------------------------------------------------------------------ */

/* Local stiffness operator, element by element (Sec. 2, footnote 1):
 *   u_d = Dhat applied along direction d           (3 contractions)
 *   W_d = sum_e G_de u_e                            (pointwise, G symmetric)
 *   w   = sum_d Dhat^T applied along direction d to W_d
 * i.e. w^e = sum_d D_d^T (sum_e G_de D_e u^e). */
void orc_ax_local(int64_t E, int N, const double *D, const double *G, const double *u, double *w) {
  int Np = N + 1, Np3 = Np * Np * Np;
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < E; ++e) {
    double *ur = malloc(sizeof(double) * Np3), *us = malloc(sizeof(double) * Np3),
           *ut = malloc(sizeof(double) * Np3);
    const double *ue = u + e * Np3;
    const double *g = G + e * 6 * Np3;
    for (int k = 0; k < Np; ++k)
      for (int j = 0; j < Np; ++j)
        for (int i = 0; i < Np; ++i) {
          double a = 0, b = 0, c = 0;
          for (int l = 0; l < Np; ++l) {
            a += D[i * Np + l] * ue[l + Np * (j + Np * k)];
            b += D[j * Np + l] * ue[i + Np * (l + Np * k)];
            c += D[k * Np + l] * ue[i + Np * (j + Np * l)];
          }
          int p = i + Np * (j + Np * k);
          double Grr = g[0 * Np3 + p], Grs = g[1 * Np3 + p], Grt = g[2 * Np3 + p];
          double Gss = g[3 * Np3 + p], Gst = g[4 * Np3 + p], Gtt = g[5 * Np3 + p];
          ur[p] = Grr * a + Grs * b + Grt * c;
          us[p] = Grs * a + Gss * b + Gst * c;
          ut[p] = Grt * a + Gst * b + Gtt * c;
        }
    double *we = w + e * Np3;
    for (int k = 0; k < Np; ++k)
      for (int j = 0; j < Np; ++j)
        for (int i = 0; i < Np; ++i) {
          double s = 0;
          for (int l = 0; l < Np; ++l) {
            s += D[l * Np + i] * ur[l + Np * (j + Np * k)];
            s += D[l * Np + j] * us[i + Np * (l + Np * k)];
            s += D[l * Np + k] * ut[i + Np * (j + Np * l)];
          }
          we[i + Np * (j + Np * k)] = s;
        }
    free(ur);
    free(us);
    free(ut);
  }
}

/* Direct stiffness summation (Sec. 2, C0 continuity; Sec. 3, gs): every local
 * copy of a global node receives the sum over all copies.  Written as the
 * plain definition u <- Q Q^T u with a global accumulator of length ng. */
int orc_gs(int64_t nl, const int64_t *ids, int64_t ng, double *u) {
  double *acc = calloc((size_t)ng, sizeof(double));
  if (!acc) return -1;
  for (int64_t l = 0; l < nl; ++l) acc[ids[l]] += u[l];
  for (int64_t l = 0; l < nl; ++l) u[l] = acc[ids[l]];
  free(acc);
  return 0;
}

/* ------------------------------------------------------------------ */
/* One discretisation level: mesh, operator, inner product             */
/* ------------------------------------------------------------------ */

typedef struct orc_level {
  int ex, ey, ez, N, bc;
  int64_t E, nl, ng;
  double *xi, *w, *D;
  double *G, *B, *X;
  int64_t *ids;
  double *mult, *inv_mult, *mask, *dinv;
  double lam_lo, lam_hi;
  double *t0, *t1; /* scratch E-layout vectors */
} orc_level;

void orc_level_destroy(orc_level *L) {
  if (!L) return;
  free(L->xi); free(L->w); free(L->D); free(L->G); free(L->B); free(L->X);
  free(L->ids); free(L->mult); free(L->inv_mult); free(L->mask); free(L->dinv);
  free(L->t0); free(L->t1);
  free(L);
}

void orc_level_diag(orc_level *L, double *d);

/* Build a level of order N on the vertex grid verts (see orc_geometry). */
orc_level *orc_level_create(int ex, int ey, int ez, int N, int bc, const double *verts) {
  if (ex < 1 || ey < 1 || ez < 1 || N < 1) return NULL;
  orc_level *L = calloc(1, sizeof(orc_level));
  int Np = N + 1, Np3 = Np * Np * Np;
  L->ex = ex; L->ey = ey; L->ez = ez; L->N = N; L->bc = bc;
  L->E = (int64_t)ex * ey * ez;
  L->nl = L->E * Np3;
  L->ng = ((int64_t)ex * N + 1) * ((int64_t)ey * N + 1) * ((int64_t)ez * N + 1);
  L->xi = malloc(sizeof(double) * Np);
  L->w = malloc(sizeof(double) * Np);
  L->D = malloc(sizeof(double) * Np * Np);
  orc_gll(N, L->xi, L->w);
  orc_dhat(N, L->xi, L->D);
  L->G = malloc(sizeof(double) * L->E * 6 * Np3);
  L->B = malloc(sizeof(double) * L->nl);
  L->X = malloc(sizeof(double) * L->E * 3 * Np3);
  if (orc_geometry(ex, ey, ez, N, verts, L->G, L->B, L->X) != 0) {
    orc_level_destroy(L);
    return NULL;
  }
  L->ids = malloc(sizeof(int64_t) * L->nl);
  orc_global_ids(ex, ey, ez, N, L->ids);
  L->mult = malloc(sizeof(double) * L->nl);
  L->inv_mult = malloc(sizeof(double) * L->nl);
  for (int64_t l = 0; l < L->nl; ++l) L->mult[l] = 1.0;
  orc_gs(L->nl, L->ids, L->ng, L->mult);
  for (int64_t l = 0; l < L->nl; ++l) L->inv_mult[l] = 1.0 / L->mult[l];
  L->mask = malloc(sizeof(double) * L->nl);
  orc_mask(ex, ey, ez, N, bc, L->mask);
  L->dinv = malloc(sizeof(double) * L->nl);
  L->t0 = malloc(sizeof(double) * L->nl);
  L->t1 = malloc(sizeof(double) * L->nl);
  orc_level_diag(L, L->dinv);
  for (int64_t l = 0; l < L->nl; ++l) L->dinv[l] = L->mask[l] / L->dinv[l];
  return L;
}

int64_t orc_level_nl(const orc_level *L) { return L->nl; }
int64_t orc_level_ng(const orc_level *L) { return L->ng; }
void orc_level_copy(const orc_level *L, int what, double *out) {
  /* what: 0 mult, 1 mask, 2 dinv, 3 B, 4 X[E][3][Np3], 5 G[E][6][Np3], 6 D, 7 xi, 8 w */
  int Np = L->N + 1;
  switch (what) {
    case 0: memcpy(out, L->mult, sizeof(double) * L->nl); break;
    case 1: memcpy(out, L->mask, sizeof(double) * L->nl); break;
    case 2: memcpy(out, L->dinv, sizeof(double) * L->nl); break;
    case 3: memcpy(out, L->B, sizeof(double) * L->nl); break;
    case 4: memcpy(out, L->X, sizeof(double) * L->nl * 3); break;
    case 5: memcpy(out, L->G, sizeof(double) * L->nl * 6); break;
    case 6: memcpy(out, L->D, sizeof(double) * Np * Np); break;
    case 7: memcpy(out, L->xi, sizeof(double) * Np); break;
    case 8: memcpy(out, L->w, sizeof(double) * Np); break;
  }
}
void orc_level_ids(const orc_level *L, int64_t *out) { memcpy(out, L->ids, sizeof(int64_t) * L->nl); }

/* Assembled operator on the level: w = mask * gs(A_L u). */
void orc_level_ax(orc_level *L, const double *u, double *w) {
  orc_ax_local(L->E, L->N, L->D, L->G, u, w);
  orc_gs(L->nl, L->ids, L->ng, w);
  for (int64_t l = 0; l < L->nl; ++l) w[l] *= L->mask[l];
}

void orc_level_gs(orc_level *L, double *u) { orc_gs(L->nl, L->ids, L->ng, u); }

/* Reading (paper silent): inner product of E-layout vectors with copies equal
 * = Euclidean product over unique dofs = sum_l u_l v_l / mult_l. */
double orc_level_dot(const orc_level *L, const double *u, const double *v) {
  double s = 0.0;
  for (int64_t l = 0; l < L->nl; ++l) s += u[l] * v[l] * L->inv_mult[l];
  return s;
}

/* Diagonal of the assembled operator: local diagonal in closed form, then gs.
 * With D_1 = Dhat along r etc., the local diagonal at (i,j,k) is
 *   sum_a Dhat_ai^2 G_rr(a,j,k) + sum_b Dhat_bj^2 G_ss(i,b,k) + sum_c Dhat_ck^2 G_tt(i,j,c)
 *   + 2 Dhat_ii Dhat_jj G_rs(i,j,k) + 2 Dhat_ii Dhat_kk G_rt(i,j,k)
 *   + 2 Dhat_jj Dhat_kk G_st(i,j,k),
 * the cross terms surviving only where both indices are at an element face.
 * Output d is unmasked. */
void orc_level_diag(orc_level *L, double *d) {
  int Np = L->N + 1, Np3 = Np * Np * Np;
  const double *D = L->D;
  for (int64_t e = 0; e < L->E; ++e) {
    const double *g = L->G + e * 6 * Np3;
    for (int k = 0; k < Np; ++k)
      for (int j = 0; j < Np; ++j)
        for (int i = 0; i < Np; ++i) {
          int p = i + Np * (j + Np * k);
          double s = 0.0;
          for (int l = 0; l < Np; ++l) {
            s += D[l * Np + i] * D[l * Np + i] * g[0 * Np3 + l + Np * (j + Np * k)];
            s += D[l * Np + j] * D[l * Np + j] * g[3 * Np3 + i + Np * (l + Np * k)];
            s += D[l * Np + k] * D[l * Np + k] * g[5 * Np3 + i + Np * (j + Np * l)];
          }
          double Di = D[i * Np + i], Dj = D[j * Np + j], Dk = D[k * Np + k];
          s += 2.0 * Di * Dj * g[1 * Np3 + p];
          s += 2.0 * Di * Dk * g[2 * Np3 + p];
          s += 2.0 * Dj * Dk * g[4 * Np3 + p];
          d[e * Np3 + p] = s;
        }
  }
  orc_gs(L->nl, L->ids, L->ng, d);
}

/* ------------------------------------------------------------------ */
/* Jacobi-PCG (Sec. 3, Stokes substep)                                  */
/* ------------------------------------------------------------------ */

/* Reading of the tolerance (paper silent on the norm): stop when
 * ||r||_2 <= tol ||b||_2, both in the unique-dof inner product.  x is the
 * initial guess on entry.  Returns 0 when converged, 1 when maxit reached.
 * precond = 1: z = Dinv r (Jacobi); 0: z = mask r (plain CG).  tol <= 0 runs
 * exactly maxit iterations. */
int orc_pcg(orc_level *L, const double *b, double *x, double tol, int maxit, int precond,
            int *iters, double *res0, double *res) {
  int64_t n = L->nl;
  double *r = malloc(sizeof(double) * n), *z = malloc(sizeof(double) * n),
         *p = malloc(sizeof(double) * n), *w = malloc(sizeof(double) * n);
  orc_level_ax(L, x, w);
  for (int64_t l = 0; l < n; ++l) r[l] = b[l] - w[l];
  double bnorm = sqrt(orc_level_dot(L, b, b));
  double rnorm = sqrt(orc_level_dot(L, r, r));
  *res0 = rnorm;
  int k = 0, status = 1;
  if (rnorm <= tol * bnorm || rnorm == 0.0) status = 0;
  if (status != 0) {
    for (int64_t l = 0; l < n; ++l) z[l] = (precond ? L->dinv[l] : L->mask[l]) * r[l];
    for (int64_t l = 0; l < n; ++l) p[l] = z[l];
    double rho = orc_level_dot(L, r, z);
    while (k < maxit) {
      orc_level_ax(L, p, w);
      double alpha = rho / orc_level_dot(L, p, w);
      for (int64_t l = 0; l < n; ++l) x[l] += alpha * p[l];
      for (int64_t l = 0; l < n; ++l) r[l] -= alpha * w[l];
      ++k;
      rnorm = sqrt(orc_level_dot(L, r, r));
      if (rnorm <= tol * bnorm) { status = 0; break; }
      for (int64_t l = 0; l < n; ++l) z[l] = (precond ? L->dinv[l] : L->mask[l]) * r[l];
      double rho1 = orc_level_dot(L, r, z);
      double beta = rho1 / rho;
      rho = rho1;
      for (int64_t l = 0; l < n; ++l) p[l] = z[l] + beta * p[l];
    }
  }
  *iters = k;
  *res = rnorm;
  free(r); free(z); free(p); free(w);
  return status;
}

/* ------------------------------------------------------------------ */
/* Chebyshev-accelerated Jacobi smoothing (Sec. 3, pMG smoothers)       */
/* ------------------------------------------------------------------ */

typedef void (*orc_apply_fn)(void *ctx, const double *in, double *out);

/* Degree-k Chebyshev iteration for A x = b preconditioned by diag(dinv), on the
 * interval [lmin, lmax] of the spectrum of Dinv A (the standard three-term
 * recurrence of Chebyshev acceleration, Saad, Iterative Methods, Alg. 12.1):
 *   theta = (lmax+lmin)/2, delta = (lmax-lmin)/2, sigma = theta/delta, rho = 1/sigma
 *   r = b - A x;  d = Dinv r / theta
 *   repeat k times:  x += d;  (unless last) r -= A d;
 *                    rho' = 1/(2 sigma - rho);  d = rho' rho d + (2 rho'/delta) Dinv r;  rho = rho'
 * The error after the call is T_k((theta - Dinv A)/delta) / T_k(theta/delta)
 * times the error before it.  x_zero = 1 skips the first product (x = 0). */
void orc_cheb(int64_t n, orc_apply_fn A, void *ctx, const double *dinv, const double *b,
              double *x, int k, double lmin, double lmax, int x_zero) {
  double *r = malloc(sizeof(double) * n), *d = malloc(sizeof(double) * n),
         *ad = malloc(sizeof(double) * n);
  double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin);
  double sigma = theta / delta, rho = 1.0 / sigma;
  if (x_zero) {
    for (int64_t l = 0; l < n; ++l) { x[l] = 0.0; r[l] = b[l]; }
  } else {
    A(ctx, x, ad);
    for (int64_t l = 0; l < n; ++l) r[l] = b[l] - ad[l];
  }
  for (int64_t l = 0; l < n; ++l) d[l] = dinv[l] * r[l] / theta;
  for (int it = 1; it <= k; ++it) {
    for (int64_t l = 0; l < n; ++l) x[l] += d[l];
    if (it == k) break;
    A(ctx, d, ad);
    for (int64_t l = 0; l < n; ++l) r[l] -= ad[l];
    double rho1 = 1.0 / (2.0 * sigma - rho);
    for (int64_t l = 0; l < n; ++l) d[l] = rho1 * rho * d[l] + (2.0 * rho1 / delta) * dinv[l] * r[l];
    rho = rho1;
  }
  free(r); free(d); free(ad);
}

static void level_apply(void *ctx, const double *in, double *out) {
  orc_level_ax((orc_level *)ctx, in, out);
}

/* splitmix64 (Steele, Lea, Flood 2014; Vigna's reference constants), used as a
 * counter-based generator: value i of stream `seed` is mix(seed + (i+1) * gamma). */
static uint64_t splitmix64_at(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* Value i of stream seed, exported so that the generator can be checked
 * against the published reference stream. */
uint64_t orc_splitmix64(uint64_t seed, uint64_t i) { return splitmix64_at(seed, i); }

/* Largest eigenvalue of the symmetric tridiagonal (a diagonal, b off-diagonal,
 * size m) by bisection on the Sturm sequence count. */
static double tridiag_max_eig(int m, const double *a, const double *b) {
  double lo = a[0], hi = a[0];
  for (int i = 0; i < m; ++i) {
    double rad = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i < m - 1 ? fabs(b[i]) : 0.0);
    if (a[i] - rad < lo) lo = a[i] - rad;
    if (a[i] + rad > hi) hi = a[i] + rad;
  }
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    /* number of eigenvalues below mid */
    int cnt = 0;
    double q = 1.0;
    for (int i = 0; i < m; ++i) {
      double bb = i > 0 ? b[i - 1] * b[i - 1] : 0.0;
      q = a[i] - mid - (i > 0 ? bb / q : 0.0);
      if (q == 0.0) q = -1e-300;
      if (q < 0) ++cnt;
    }
    if (cnt == m) hi = mid; else lo = mid;
    if (hi - lo <= 1e-15 * fabs(hi)) break;
  }
  return hi;
}

/* Reading (paper silent on the Chebyshev interval): lambda_max of Dinv A is
 * estimated by m steps of Jacobi-PCG on A y = v (the Lanczos tridiagonal from
 * the CG coefficients), with v a splitmix64 field U(-1,1) keyed by global id
 * (continuous), masked, and mean-removed under Neumann.  Returns the
 * estimate; *steps_done receives the number of steps actually taken. */
static void jacobi_prec(void *ctx, const double *in, double *out) {
  const orc_level *L = (const orc_level *)ctx;
  for (int64_t l = 0; l < L->nl; ++l) out[l] = L->dinv[l] * in[l];
}

static double lanczos_max_m(orc_level *L, int m, uint64_t seed, void (*Mf)(void *, const double *, double *),
                            void *mctx, int *steps_done);

/* The Lanczos start vector: value 2 u - 1 at every local copy of global node
 * g, with u the 53-bit fraction of splitmix64 value g of stream seed
 * (continuous), masked, and under Neumann minus its unique-dof mean. */
void orc_lanczos_start(const orc_level *L, uint64_t seed, double *v) {
  int64_t n = L->nl;
  for (int64_t l = 0; l < n; ++l) {
    uint64_t bits = splitmix64_at(seed, (uint64_t)L->ids[l]);
    double u01 = (double)(bits >> 11) * (1.0 / 9007199254740992.0);
    v[l] = (2.0 * u01 - 1.0) * L->mask[l];
  }
  if (L->bc == 1) {
    double s = 0.0, c = 0.0;
    for (int64_t l = 0; l < n; ++l) { s += v[l] * L->inv_mult[l]; c += L->inv_mult[l]; }
    for (int64_t l = 0; l < n; ++l) v[l] -= s / c;
  }
}

double orc_level_lanczos_max(orc_level *L, int m, uint64_t seed, int *steps_done) {
  return lanczos_max_m(L, m, seed, jacobi_prec, L, steps_done);
}

/* The Lanczos estimate of the largest eigenvalue of M A from the
 * coefficients of m steps of M-preconditioned CG (M = D^{-1} or the Schwarz
 * preconditioner). */
static double lanczos_max_m(orc_level *L, int m, uint64_t seed, void (*Mf)(void *, const double *, double *),
                            void *mctx, int *steps_done) {
  int64_t n = L->nl;
  double *v = malloc(sizeof(double) * n), *r = malloc(sizeof(double) * n),
         *z = malloc(sizeof(double) * n), *p = malloc(sizeof(double) * n),
         *w = malloc(sizeof(double) * n);
  double *alph = malloc(sizeof(double) * (m + 1)), *bet = malloc(sizeof(double) * (m + 1));
  orc_lanczos_start(L, seed, v);
  for (int64_t l = 0; l < n; ++l) r[l] = v[l];
  Mf(mctx, r, z);
  for (int64_t l = 0; l < n; ++l) p[l] = z[l];
  double rho = orc_level_dot(L, r, z), rho_start = rho;
  int k = 0;
  for (; k < m; ++k) {
    orc_level_ax(L, p, w);
    double pw = orc_level_dot(L, p, w);
    double alpha = rho / pw;
    for (int64_t l = 0; l < n; ++l) r[l] -= alpha * w[l];
    Mf(mctx, r, z);
    double rho1 = orc_level_dot(L, r, z);
    double beta = rho1 / rho;
    alph[k] = alpha;
    bet[k] = beta;
    rho = rho1;
    if (!(rho1 > 1e-28 * rho_start)) { ++k; break; }
    for (int64_t l = 0; l < n; ++l) p[l] = z[l] + beta * p[l];
  }
  /* tridiagonal of the Lanczos process from the CG coefficients */
  double *ta = malloc(sizeof(double) * (k + 1)), *tb = malloc(sizeof(double) * (k + 1));
  for (int j = 0; j < k; ++j) {
    ta[j] = 1.0 / alph[j] + (j > 0 ? bet[j - 1] / alph[j - 1] : 0.0);
    if (j < k - 1) tb[j] = sqrt(bet[j]) / alph[j];
  }
  double lmax = tridiag_max_eig(k, ta, tb);
  *steps_done = k;
  free(v); free(r); free(z); free(p); free(w); free(alph); free(bet); free(ta); free(tb);
  return lmax;
}

/* ------------------------------------------------------------------ */
/* Overlapping Schwarz smoother with separable local problems (Sec. 3,  */
/* Eq. 3: local Poisson problems on elements extended by one layer into */
/* their neighbours, solved by fast diagonalisation)                     */
/* ------------------------------------------------------------------ */
/* Reading (the paper gives the structure, not the construction):
 * - The extended element has n = N + 3 points per direction: the element's
 *   own GLL points plus, on each side with a neighbour, the neighbour's
 *   second point from the shared face.  Beyond them the local problem is
 *   homogeneous Dirichlet.
 * - The local operator is separable, K = Bz x By x Ax + Bz x Ay x Bx +
 *   Az x By x Bx, with the 1D matrices of each direction taken from the 1D
 *   SEM stiffness (2/h) sum_q w_q D_qi D_qj and mass (h/2) w_i assembled over
 *   the neighbour, the element and the other neighbour, each with its own
 *   mean length h along that direction (the mean of the element's four edges
 *   in that direction), restricted to the extended points.  Without a
 *   neighbour the extension point is decoupled (a row and column of the
 *   identity in A and B); a Dirichlet boundary face decouples the face
 *   points too.
 * - Only face data enter (the paper exchanges faces, not edges or
 *   corners): extended points outside the element in two or three
 *   directions are not part of the local problem's data (they are zero on
 *   input and discarded on output).
 * - Additive combination: z = mask * sum_e R_e^T K_e^{-1} R_e r on unique
 *   nodes.  The oracle solves each K_e densely (Cholesky, factor computed at
 *   setup): the plain definition of what the fast diagonalisation computes. */
typedef struct orc_asm {
  orc_level *L;
  int n;
  double *h;     /* [E][3] */
  double *chol;  /* [E][n^3][n^3] lower Cholesky factors */
} orc_asm;

static void elem_lengths(const orc_level *L, double *h) {
  int Np = L->N + 1, Np3 = Np * Np * Np, N = L->N;
  for (int64_t e = 0; e < L->E; ++e) {
    const double *X = L->X + e * 3 * Np3;
    for (int d = 0; d < 3; ++d) {
      double s = 0.0;
      for (int q = 0; q < 4; ++q) {
        int c0[3] = {0, 0, 0};
        int o1 = (d + 1) % 3, o2 = (d + 2) % 3;
        c0[o1] = (q & 1) ? N : 0;
        c0[o2] = (q & 2) ? N : 0;
        int c1[3] = {c0[0], c0[1], c0[2]};
        c1[d] = N;
        int p0 = c0[0] + Np * (c0[1] + Np * c0[2]), p1 = c1[0] + Np * (c1[1] + Np * c1[2]);
        double len2 = 0.0;
        for (int m = 0; m < 3; ++m) {
          double dx = X[m * Np3 + p1] - X[m * Np3 + p0];
          len2 += dx * dx;
        }
        s += sqrt(len2);
      }
      h[e * 3 + d] = 0.25 * s;
    }
  }
}

/* element position along direction d and the element stride in d */
static void elem_pos(const orc_level *L, int64_t e, int d, int *pos, int *cnt, int64_t *stride) {
  int ix = (int)(e % L->ex), iy = (int)((e / L->ex) % L->ey), iz = (int)(e / ((int64_t)L->ex * L->ey));
  if (d == 0) { *pos = ix; *cnt = L->ex; *stride = 1; }
  else if (d == 1) { *pos = iy; *cnt = L->ey; *stride = L->ex; }
  else { *pos = iz; *cnt = L->ez; *stride = (int64_t)L->ex * L->ey; }
}

/* 1D extended stiffness A and mass B (n x n, row-major) of element e along d */
void orc_asm_1d(const orc_level *L, const double *h, int64_t e, int d, double *A, double *B) {
  int N = L->N, Np = N + 1, n = N + 3;
  double *Ar = malloc(sizeof(double) * Np * Np);
  for (int i = 0; i < Np; ++i)
    for (int j = 0; j < Np; ++j) {
      double s = 0.0;
      for (int q = 0; q < Np; ++q) s += L->w[q] * L->D[q * Np + i] * L->D[q * Np + j];
      Ar[i * Np + j] = s;
    }
  for (int q = 0; q < n * n; ++q) { A[q] = 0.0; B[q] = 0.0; }
  int pos, cnt;
  int64_t stride;
  elem_pos(L, e, d, &pos, &cnt, &stride);
  double he = h[e * 3 + d];
  for (int i = 0; i < Np; ++i) {
    for (int j = 0; j < Np; ++j) A[(i + 1) * n + (j + 1)] += (2.0 / he) * Ar[i * Np + j];
    B[(i + 1) * n + (i + 1)] += 0.5 * he * L->w[i];
  }
  if (pos > 0) {  /* left neighbour: its points N-1, N are extended points 0, 1 */
    double hl = h[(e - stride) * 3 + d];
    int li[2] = {N - 1, N}, ai[2] = {0, 1};
    for (int p = 0; p < 2; ++p) {
      for (int q = 0; q < 2; ++q) A[ai[p] * n + ai[q]] += (2.0 / hl) * Ar[li[p] * Np + li[q]];
      B[ai[p] * n + ai[p]] += 0.5 * hl * L->w[li[p]];
    }
  }
  if (pos < cnt - 1) {  /* right neighbour: its points 0, 1 are extended points N+1, N+2 */
    double hr = h[(e + stride) * 3 + d];
    int li[2] = {0, 1}, ai[2] = {N + 1, N + 2};
    for (int p = 0; p < 2; ++p) {
      for (int q = 0; q < 2; ++q) A[ai[p] * n + ai[q]] += (2.0 / hr) * Ar[li[p] * Np + li[q]];
      B[ai[p] * n + ai[p]] += 0.5 * hr * L->w[li[p]];
    }
  }
  /* decoupled points: missing extensions, and Dirichlet boundary faces */
  int dec[4], nd = 0;
  if (pos == 0) { dec[nd++] = 0; if (L->bc == 0) dec[nd++] = 1; }
  if (pos == cnt - 1) { dec[nd++] = N + 2; if (L->bc == 0) dec[nd++] = N + 1; }
  for (int t = 0; t < nd; ++t) {
    int a = dec[t];
    for (int q = 0; q < n; ++q) { A[a * n + q] = 0.0; A[q * n + a] = 0.0; B[a * n + q] = 0.0; B[q * n + a] = 0.0; }
    A[a * n + a] = 1.0;
    B[a * n + a] = 1.0;
  }
  free(Ar);
}

/* dense local operator K (n^3 x n^3) of element e, index a + n (b + n c) */
void orc_asm_local_matrix(const orc_asm *M, int64_t e, double *K) {
  int n = M->n, n3 = n * n * n;
  double *A[3], *B[3];
  for (int d = 0; d < 3; ++d) {
    A[d] = malloc(sizeof(double) * n * n);
    B[d] = malloc(sizeof(double) * n * n);
    orc_asm_1d(M->L, M->h, e, d, A[d], B[d]);
  }
  for (int p = 0; p < n3; ++p) {
    int a = p % n, b = (p / n) % n, c = p / (n * n);
    for (int q = 0; q < n3; ++q) {
      int a2 = q % n, b2 = (q / n) % n, c2 = q / (n * n);
      K[(size_t)p * n3 + q] = B[2][c * n + c2] * B[1][b * n + b2] * A[0][a * n + a2] +
                              B[2][c * n + c2] * A[1][b * n + b2] * B[0][a * n + a2] +
                              A[2][c * n + c2] * B[1][b * n + b2] * B[0][a * n + a2];
    }
  }
  for (int d = 0; d < 3; ++d) { free(A[d]); free(B[d]); }
}

orc_asm *orc_asm_create(orc_level *L) {
  orc_asm *M = calloc(1, sizeof(orc_asm));
  M->L = L;
  M->n = L->N + 3;
  int n3 = M->n * M->n * M->n;
  M->h = malloc(sizeof(double) * L->E * 3);
  elem_lengths(L, M->h);
  M->chol = malloc(sizeof(double) * (size_t)L->E * n3 * n3);
  for (int64_t e = 0; e < L->E; ++e) {
    double *K = M->chol + (size_t)e * n3 * n3;
    orc_asm_local_matrix(M, e, K);
    /* Cholesky K = C C^T in the lower triangle */
    for (int j = 0; j < n3; ++j) {
      double s = K[(size_t)j * n3 + j];
      for (int k = 0; k < j; ++k) s -= K[(size_t)j * n3 + k] * K[(size_t)j * n3 + k];
      double cj = sqrt(s);
      K[(size_t)j * n3 + j] = cj;
      for (int i = j + 1; i < n3; ++i) {
        double t = K[(size_t)i * n3 + j];
        for (int k = 0; k < j; ++k) t -= K[(size_t)i * n3 + k] * K[(size_t)j * n3 + k];
        K[(size_t)i * n3 + j] = t / cj;
      }
    }
  }
  return M;
}

void orc_asm_destroy(orc_asm *M) {
  if (!M) return;
  free(M->h); free(M->chol); free(M);
}

/* local index of extended point (a, b, c) of element e, or -1 if it carries
 * no face data (outside the element in two or more directions, or beyond a
 * side without a neighbour) */
static int64_t ext_point(const orc_level *L, int64_t e, int a, int b, int c) {
  int N = L->N, Np = N + 1, Np3 = Np * Np * Np;
  int idx[3] = {a - 1, b - 1, c - 1};
  int out = -1, nout = 0;
  for (int d = 0; d < 3; ++d)
    if (idx[d] < 0 || idx[d] > N) { out = d; ++nout; }
  if (nout == 0) return e * Np3 + idx[0] + Np * (idx[1] + Np * idx[2]);
  if (nout > 1) return -1;
  int pos, cnt;
  int64_t stride;
  elem_pos(L, e, out, &pos, &cnt, &stride);
  if (idx[out] < 0) {
    if (pos == 0) return -1;
    idx[out] = N - 1;
    return (e - stride) * Np3 + idx[0] + Np * (idx[1] + Np * idx[2]);
  }
  if (pos == cnt - 1) return -1;
  idx[out] = 1;
  return (e + stride) * Np3 + idx[0] + Np * (idx[1] + Np * idx[2]);
}

/* z = mask * sum_e R_e^T K_e^{-1} R_e r (r, z continuous E-layout vectors) */
void orc_asm_apply(const orc_asm *M, const double *r, double *z) {
  const orc_level *L = M->L;
  int n = M->n, n3 = n * n * n;
  double *acc = calloc(L->ng, sizeof(double));
  double *u = malloc(sizeof(double) * n3);
  int64_t *loc = malloc(sizeof(int64_t) * n3);
  for (int64_t e = 0; e < L->E; ++e) {
    for (int p = 0; p < n3; ++p) {
      loc[p] = ext_point(L, e, p % n, (p / n) % n, p / (n * n));
      u[p] = loc[p] >= 0 ? r[loc[p]] : 0.0;
    }
    const double *C = M->chol + (size_t)e * n3 * n3;
    for (int i = 0; i < n3; ++i) {  /* C y = u */
      double s = u[i];
      for (int k = 0; k < i; ++k) s -= C[(size_t)i * n3 + k] * u[k];
      u[i] = s / C[(size_t)i * n3 + i];
    }
    for (int i = n3 - 1; i >= 0; --i) {  /* C^T v = y */
      double s = u[i];
      for (int k = i + 1; k < n3; ++k) s -= C[(size_t)k * n3 + i] * u[k];
      u[i] = s / C[(size_t)i * n3 + i];
    }
    for (int p = 0; p < n3; ++p)
      if (loc[p] >= 0) acc[L->ids[loc[p]]] += u[p];
  }
  for (int64_t l = 0; l < L->nl; ++l) z[l] = acc[L->ids[l]] * L->mask[l];
  free(acc); free(u); free(loc);
}

/* Chebyshev smoothing (Saad Alg. 12.1) with a general preconditioner M in
 * place of the Jacobi diagonal: the same recurrence on M A. */
typedef void (*orc_prec_fn)(void *ctx, const double *in, double *out);
void orc_cheb_m(int64_t n, orc_apply_fn A, void *actx, orc_prec_fn Mf, void *mctx,
                const double *b, double *x, int k, double lmin, double lmax, int x_zero) {
  double *r = malloc(sizeof(double) * n), *d = malloc(sizeof(double) * n),
         *ad = malloc(sizeof(double) * n), *mr = malloc(sizeof(double) * n);
  double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin);
  double sigma = theta / delta, rho = 1.0 / sigma;
  if (x_zero) {
    for (int64_t l = 0; l < n; ++l) { x[l] = 0.0; r[l] = b[l]; }
  } else {
    A(actx, x, ad);
    for (int64_t l = 0; l < n; ++l) r[l] = b[l] - ad[l];
  }
  Mf(mctx, r, mr);
  for (int64_t l = 0; l < n; ++l) d[l] = mr[l] / theta;
  for (int it = 1; it <= k; ++it) {
    for (int64_t l = 0; l < n; ++l) x[l] += d[l];
    if (it == k) break;
    A(actx, d, ad);
    for (int64_t l = 0; l < n; ++l) r[l] -= ad[l];
    double rho1 = 1.0 / (2.0 * sigma - rho);
    Mf(mctx, r, mr);
    for (int64_t l = 0; l < n; ++l) d[l] = rho1 * rho * d[l] + (2.0 * rho1 / delta) * mr[l];
    rho = rho1;
  }
  free(r); free(d); free(ad); free(mr);
}

static void asm_prec(void *ctx, const double *in, double *out) {
  orc_asm_apply((const orc_asm *)ctx, in, out);
}

/* ------------------------------------------------------------------ */
/* p-multigrid V-cycle (Sec. 3, pMG paragraph) and FlexCG               */
/* ------------------------------------------------------------------ */

typedef struct orc_pmg {
  int nlev, cheb_degree, coarse_maxit;
  int smoother;          /* 0 Chebyshev-Jacobi, 1 Chebyshev-Schwarz */
  orc_asm *asmp[8];
  double coarse_tol;
  orc_level *lev[8];
  double *J[8]; /* J[l]: (N_l+1) x (N_{l+1}+1), coarse level l+1 to fine level l */
  double *x[8], *b[8], *r[8];
  int coarse_iters_last;
} orc_pmg;

void orc_pmg_destroy(orc_pmg *P) {
  if (!P) return;
  for (int l = 0; l < P->nlev; ++l) {
    orc_level_destroy(P->lev[l]);
    free(P->J[l]); free(P->x[l]); free(P->b[l]); free(P->r[l]);
    orc_asm_destroy(P->asmp[l]);
  }
  free(P);
}

/* Levels of orders Ns[0] > Ns[1] > ... (the paper's schedule notation, e.g.
 * 7-3-1).  Every level is built from the same vertex grid: the trilinear
 * geometry is rediscretised exactly at each order.  Chebyshev bounds per
 * smoothed level: lambda_hi = 1.1 * estimate (m Lanczos steps),
 * lambda_lo = lambda_hi / 10 (reading; the paper gives no bounds). */
orc_pmg *orc_pmg_create2(int ex, int ey, int ez, int nlev, const int *Ns, int bc,
                         const double *verts, int cheb_degree, int lanczos_steps, uint64_t seed,
                         double coarse_tol, int coarse_maxit, int smoother);

orc_pmg *orc_pmg_create(int ex, int ey, int ez, int nlev, const int *Ns, int bc,
                        const double *verts, int cheb_degree, int lanczos_steps, uint64_t seed,
                        double coarse_tol, int coarse_maxit) {
  return orc_pmg_create2(ex, ey, ez, nlev, Ns, bc, verts, cheb_degree, lanczos_steps, seed,
                         coarse_tol, coarse_maxit, 0);
}

/* smoother 1: Chebyshev acceleration of the overlapping Schwarz preconditioner
 * (orc_asm) on every smoothed level, interval from the Lanczos estimate of
 * lambda_max(M A) with the same rule. */
orc_pmg *orc_pmg_create2(int ex, int ey, int ez, int nlev, const int *Ns, int bc,
                         const double *verts, int cheb_degree, int lanczos_steps, uint64_t seed,
                         double coarse_tol, int coarse_maxit, int smoother) {
  if (nlev < 1 || nlev > 8) return NULL;
  orc_pmg *P = calloc(1, sizeof(orc_pmg));
  P->nlev = nlev;
  P->smoother = smoother;
  P->cheb_degree = cheb_degree;
  P->coarse_tol = coarse_tol;
  P->coarse_maxit = coarse_maxit;
  for (int l = 0; l < nlev; ++l) {
    P->lev[l] = orc_level_create(ex, ey, ez, Ns[l], bc, verts);
    if (!P->lev[l]) { P->nlev = l; orc_pmg_destroy(P); return NULL; }
    int64_t n = P->lev[l]->nl;
    P->x[l] = malloc(sizeof(double) * n);
    P->b[l] = malloc(sizeof(double) * n);
    P->r[l] = malloc(sizeof(double) * n);
  }
  for (int l = 0; l + 1 < nlev; ++l) {
    orc_level *F = P->lev[l], *C = P->lev[l + 1];
    P->J[l] = malloc(sizeof(double) * (F->N + 1) * (C->N + 1));
    orc_interp(F->N, F->xi, C->N, C->xi, P->J[l]);
    int steps;
    double est;
    if (smoother == 1) {
      P->asmp[l] = orc_asm_create(F);
      est = lanczos_max_m(F, lanczos_steps, seed, asm_prec, P->asmp[l], &steps);
    } else {
      est = orc_level_lanczos_max(F, lanczos_steps, seed, &steps);
    }
    F->lam_hi = 1.1 * est;
    F->lam_lo = F->lam_hi / 10.0;
  }
  return P;
}

double orc_pmg_lambda(const orc_pmg *P, int l, int hi) {
  return hi ? P->lev[l]->lam_hi : P->lev[l]->lam_lo;
}
orc_level *orc_pmg_level(orc_pmg *P, int l) { return P->lev[l]; }

/* Tensor-product interpolation per element: out = (J x J x J) in, with J of
 * size nf x nc (Sec. 3: u_f = (Jhat x Jhat x Jhat) u_c); transpose = 1 applies
 * (J^T x J^T x J^T) from fine to coarse instead. */
void orc_interp3(int64_t E, int nf, int nc, const double *J, const double *in, double *out,
                 int transpose) {
  int ni = transpose ? nf : nc, no = transpose ? nc : nf;
  int ni3 = ni * ni * ni, no3 = no * no * no;
  for (int64_t e = 0; e < E; ++e) {
    const double *ue = in + e * ni3;
    double *ve = out + e * no3;
    for (int k = 0; k < no; ++k)
      for (int j = 0; j < no; ++j)
        for (int i = 0; i < no; ++i) {
          double s = 0.0;
          for (int c = 0; c < ni; ++c)
            for (int b = 0; b < ni; ++b)
              for (int a = 0; a < ni; ++a) {
                double Ja = transpose ? J[a * nc + i] : J[i * nc + a];
                double Jb = transpose ? J[b * nc + j] : J[j * nc + b];
                double Jc = transpose ? J[c * nc + k] : J[k * nc + c];
                s += Ja * Jb * Jc * ue[a + ni * (b + ni * c)];
              }
          ve[i + no * (j + no * k)] = s;
        }
  }
}

static void vcycle(orc_pmg *P, int l) {
  orc_level *L = P->lev[l];
  int64_t n = L->nl;
  double *x = P->x[l], *b = P->b[l], *r = P->r[l];
  if (l == P->nlev - 1) {
    /* Reading: coarsest level solved by FP64 Jacobi-PCG from zero, to
     * coarse_tol relative or coarse_maxit iterations.  Under Neumann the
     * right-hand side is first made mean-free (projection onto the range). */
    if (L->bc == 1) {
      double s = 0.0, c = 0.0;
      for (int64_t i = 0; i < n; ++i) { s += b[i] * L->inv_mult[i]; c += L->inv_mult[i]; }
      for (int64_t i = 0; i < n; ++i) b[i] -= s / c;
    }
    for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
    int it;
    double r0, r1;
    orc_pcg(L, b, x, P->coarse_tol, P->coarse_maxit, 1, &it, &r0, &r1);
    P->coarse_iters_last = it;
    return;
  }
  orc_level *C = P->lev[l + 1];
  /* pre-smoothing from zero */
  if (P->smoother == 1)
    orc_cheb_m(n, level_apply, L, asm_prec, P->asmp[l], b, x, P->cheb_degree, L->lam_lo,
               L->lam_hi, 1);
  else
    orc_cheb(n, level_apply, L, L->dinv, b, x, P->cheb_degree, L->lam_lo, L->lam_hi, 1);
  /* residual */
  orc_level_ax(L, x, r);
  for (int64_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
  /* restriction = transpose of prolongation on unique dofs:
   * r_c = mask_c * gs_c( (J^T x J^T x J^T) (r / mult_f) ) */
  for (int64_t i = 0; i < n; ++i) r[i] *= L->inv_mult[i];
  orc_interp3(L->E, L->N + 1, C->N + 1, P->J[l], r, P->b[l + 1], 1);
  orc_level_gs(C, P->b[l + 1]);
  for (int64_t i = 0; i < C->nl; ++i) P->b[l + 1][i] *= C->mask[i];
  vcycle(P, l + 1);
  /* prolongation and correction: x += (J x J x J) e_c */
  orc_interp3(L->E, L->N + 1, C->N + 1, P->J[l], P->x[l + 1], r, 0);
  for (int64_t i = 0; i < n; ++i) x[i] += r[i];
  /* post-smoothing */
  if (P->smoother == 1)
    orc_cheb_m(n, level_apply, L, asm_prec, P->asmp[l], b, x, P->cheb_degree, L->lam_lo,
               L->lam_hi, 0);
  else
    orc_cheb(n, level_apply, L, L->dinv, b, x, P->cheb_degree, L->lam_lo, L->lam_hi, 0);
}

/* One V-cycle z = M(r) on the finest level. */
void orc_pmg_vcycle(orc_pmg *P, const double *r, double *z) {
  orc_level *L = P->lev[0];
  memcpy(P->b[0], r, sizeof(double) * L->nl);
  vcycle(P, 0);
  memcpy(z, P->x[0], sizeof(double) * L->nl);
}

int orc_pmg_coarse_iters(const orc_pmg *P) { return P->coarse_iters_last; }

/* Flexible CG (Sec. 3: FlexCG for the nonsymmetric pMG preconditioner) with
 * the Polak-Ribiere / Notay coefficient
 *   beta_k = (z_{k+1}, r_{k+1} - r_k) / (z_k, r_k).
 * precond = 1 uses one pMG V-cycle per iteration; precond = 0 uses Jacobi
 * on the finest level (then the iterates equal those of Jacobi-PCG up to
 * rounding).  Stopping rule and return value as orc_pcg. */
/* Flexible GMRES (Sec. 3: GMRES as the alternative outer solver to FlexCG;
 * Sec. 5: few vectors, classical Gram-Schmidt so that the orthogonalisation
 * needs one reduction).  Right preconditioning by the pMG V-cycle
 * (precond = 1) or by Jacobi (precond = 0); since the V-cycle may vary from
 * call to call, the preconditioned vectors z_j are kept and the update is
 * x = x0 + Z y (Saad, Iterative Methods for Sparse Linear Systems, Alg. 9.6).
 * Restart length m; the least-squares problem is reduced by Givens rotations
 * as the Arnoldi process goes, so |g_{j+1}| is the residual norm of the
 * current iterate.  Inner product: the unique-dof product of orc_level_dot.
 * A cycle ends when |g_{j+1}| <= tol ||b|| or after m steps; x is then formed
 * and its true residual recomputed, which decides convergence (restarting
 * from it otherwise).  hist (optional, maxit + 1 entries): ||r0|| and the
 * |g_{j+1}| of every step.  Returns 0 on convergence, 1 at maxit. */
int orc_fgmres(orc_pmg *P, int precond, const double *b, double *x, double tol, int m, int maxit,
               int *iters, double *res0, double *res, double *hist) {
  orc_level *L = P->lev[0];
  int64_t n = L->nl;
  double *V = malloc(sizeof(double) * n * (m + 1)), *Z = malloc(sizeof(double) * n * m),
         *w = malloc(sizeof(double) * n);
  double *H = calloc((size_t)(m + 1) * m, sizeof(double));  /* H[i*m + j] */
  double *cs = malloc(sizeof(double) * m), *sn = malloc(sizeof(double) * m),
         *g = malloc(sizeof(double) * (m + 1)), *y = malloc(sizeof(double) * m);
  double bnorm = sqrt(orc_level_dot(L, b, b));
  orc_level_ax(L, x, w);
  for (int64_t l = 0; l < n; ++l) V[l] = b[l] - w[l];
  double beta = sqrt(orc_level_dot(L, V, V));
  *res0 = beta;
  if (hist) hist[0] = beta;
  int k = 0, status = 1;
  if (beta <= tol * bnorm || beta == 0.0) status = 0;
  while (status != 0 && k < maxit) {
    for (int64_t l = 0; l < n; ++l) V[l] /= beta;
    for (int i = 0; i <= m; ++i) g[i] = 0.0;
    g[0] = beta;
    int cols = 0;
    for (int j = 0; j < m && k < maxit; ++j) {
      double *vj = V + (size_t)j * n, *zj = Z + (size_t)j * n, *vn = V + (size_t)(j + 1) * n;
      if (precond) orc_pmg_vcycle(P, vj, zj);
      else for (int64_t l = 0; l < n; ++l) zj[l] = L->dinv[l] * vj[l];
      orc_level_ax(L, zj, w);
      /* classical Gram-Schmidt: every coefficient from the same w */
      for (int i = 0; i <= j; ++i) H[i * m + j] = orc_level_dot(L, w, V + (size_t)i * n);
      for (int i = 0; i <= j; ++i)
        for (int64_t l = 0; l < n; ++l) w[l] -= H[i * m + j] * V[(size_t)i * n + l];
      double hn = sqrt(orc_level_dot(L, w, w));
      H[(j + 1) * m + j] = hn;
      for (int64_t l = 0; l < n; ++l) vn[l] = hn > 0.0 ? w[l] / hn : 0.0;
      /* previous rotations, then a new one that zeroes H[j+1][j] */
      for (int i = 0; i < j; ++i) {
        double a = H[i * m + j], c = H[(i + 1) * m + j];
        H[i * m + j] = cs[i] * a + sn[i] * c;
        H[(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
      }
      double a = H[j * m + j], c = H[(j + 1) * m + j];
      double d = sqrt(a * a + c * c);
      cs[j] = d > 0.0 ? a / d : 1.0;
      sn[j] = d > 0.0 ? c / d : 0.0;
      H[j * m + j] = d;
      H[(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++k;
      cols = j + 1;
      if (hist) hist[k] = fabs(g[j + 1]);
      if (fabs(g[j + 1]) <= tol * bnorm || hn == 0.0) break;
    }
    /* y = R^{-1} g by back substitution; x += Z y */
    for (int i = cols - 1; i >= 0; --i) {
      double s = g[i];
      for (int q = i + 1; q < cols; ++q) s -= H[i * m + q] * y[q];
      y[i] = s / H[i * m + i];
    }
    for (int i = 0; i < cols; ++i)
      for (int64_t l = 0; l < n; ++l) x[l] += y[i] * Z[(size_t)i * n + l];
    orc_level_ax(L, x, w);
    for (int64_t l = 0; l < n; ++l) V[l] = b[l] - w[l];
    beta = sqrt(orc_level_dot(L, V, V));
    if (beta <= tol * bnorm || beta == 0.0) status = 0;
  }
  *iters = k;
  *res = beta;
  free(V); free(Z); free(w); free(H); free(cs); free(sn); free(g); free(y);
  return status;
}

int orc_flexpcg(orc_pmg *P, int precond, const double *b, double *x, double tol, int maxit,
                int *iters, double *res0, double *res) {
  orc_level *L = P->lev[0];
  int64_t n = L->nl;
  double *r = malloc(sizeof(double) * n), *rold = malloc(sizeof(double) * n),
         *z = malloc(sizeof(double) * n), *p = malloc(sizeof(double) * n),
         *w = malloc(sizeof(double) * n);
  orc_level_ax(L, x, w);
  for (int64_t l = 0; l < n; ++l) r[l] = b[l] - w[l];
  double bnorm = sqrt(orc_level_dot(L, b, b));
  double rnorm = sqrt(orc_level_dot(L, r, r));
  *res0 = rnorm;
  int k = 0, status = 1;
  if (rnorm <= tol * bnorm || rnorm == 0.0) status = 0;
  if (status != 0) {
    if (precond) orc_pmg_vcycle(P, r, z);
    else for (int64_t l = 0; l < n; ++l) z[l] = L->dinv[l] * r[l];
    for (int64_t l = 0; l < n; ++l) p[l] = z[l];
    double rho = orc_level_dot(L, r, z);
    while (k < maxit) {
      orc_level_ax(L, p, w);
      double alpha = rho / orc_level_dot(L, p, w);
      for (int64_t l = 0; l < n; ++l) x[l] += alpha * p[l];
      for (int64_t l = 0; l < n; ++l) { rold[l] = r[l]; r[l] -= alpha * w[l]; }
      ++k;
      rnorm = sqrt(orc_level_dot(L, r, r));
      if (rnorm <= tol * bnorm) { status = 0; break; }
      if (precond) orc_pmg_vcycle(P, r, z);
      else for (int64_t l = 0; l < n; ++l) z[l] = L->dinv[l] * r[l];
      double zr = orc_level_dot(L, z, r), zro = orc_level_dot(L, z, rold);
      double beta = (zr - zro) / rho;
      rho = zr;
      for (int64_t l = 0; l < n; ++l) p[l] = z[l] + beta * p[l];
    }
  }
  *iters = k;
  *res = rnorm;
  free(r); free(rold); free(z); free(p); free(w);
  return status;
}

/* ------------------------------------------------------------------ projection
 * Projection onto previous solutions (Sec. 3, "Projection is key"): an
 * A-orthonormal basis P = [p_1 .. p_L] of earlier solutions, with A p_i kept
 * beside it.  For a new b the best fit in the A-norm is xbar = P P^T b
 * (coefficients p_i^T b, one reduction); the solver then only computes the
 * correction of A dx = b - A xbar, and x = xbar + dx.  The correction joins
 * the basis after one classical Gram-Schmidt pass in the A-inner product,
 * alpha_i = (A p_i)^T dx, p = dx - sum alpha_i p_i, with
 * ||p||_A^2 = dx^T A dx - sum alpha_i^2 (the same single reduction; the
 * paper notes dx is nearly A-orthogonal to P, so this is stable).  When L
 * reaches Lmax the space restarts from the latest solution alone.  Inner
 * products are the unique-dof product. */
typedef struct orc_proj {
  orc_level *L;
  int Lmax, nvec;
  double *P, *AP;  /* [Lmax][nl] */
} orc_proj;

orc_proj *orc_proj_create(orc_pmg *Pm, int Lmax) {
  orc_proj *Q = calloc(1, sizeof(orc_proj));
  Q->L = Pm->lev[0];
  Q->Lmax = Lmax;
  Q->P = calloc((size_t)Lmax * Q->L->nl, sizeof(double));
  Q->AP = calloc((size_t)Lmax * Q->L->nl, sizeof(double));
  return Q;
}

void orc_proj_destroy(orc_proj *Q) {
  if (!Q) return;
  free(Q->P); free(Q->AP); free(Q);
}

int orc_proj_nvec(const orc_proj *Q) { return Q->nvec; }
void orc_proj_vector(const orc_proj *Q, int i, double *p, double *ap) {
  int64_t n = Q->L->nl;
  memcpy(p, Q->P + (size_t)i * n, sizeof(double) * n);
  memcpy(ap, Q->AP + (size_t)i * n, sizeof(double) * n);
}

/* Add v (with Av = A v) to the basis after A-orthogonalisation; returns 1 if
 * added, 0 if v had no component outside the span. */
static int proj_add(orc_proj *Q, const double *v, const double *Av) {
  orc_level *L = Q->L;
  int64_t n = L->nl;
  int k = Q->nvec;
  double *alpha = malloc(sizeof(double) * (k + 1));
  for (int i = 0; i < k; ++i) alpha[i] = orc_level_dot(L, Q->AP + (size_t)i * n, v);
  double vav = orc_level_dot(L, v, Av);
  double nrm2 = vav;
  for (int i = 0; i < k; ++i) nrm2 -= alpha[i] * alpha[i];
  int added = 0;
  if (nrm2 > 1e-24 * vav && nrm2 > 0.0) {
    double s = 1.0 / sqrt(nrm2);
    double *p = Q->P + (size_t)k * n, *ap = Q->AP + (size_t)k * n;
    for (int64_t l = 0; l < n; ++l) {
      double a = v[l], b = Av[l];
      for (int i = 0; i < k; ++i) {
        a -= alpha[i] * Q->P[(size_t)i * n + l];
        b -= alpha[i] * Q->AP[(size_t)i * n + l];
      }
      p[l] = a * s;
      ap[l] = b * s;
    }
    Q->nvec = k + 1;
    added = 1;
  }
  free(alpha);
  return added;
}

/* Solve A x = b to tol (relative to ||b||) with projection: x is output only
 * (the best fit is the initial guess).  solver 0: FlexCG + pMG, 1: FGMRES(m)
 * + pMG.  Reports the iterations of the correction solve and ||b - A xbar||. */
int orc_solve_projected(orc_pmg *Pm, orc_proj *Q, int solver, int m, const double *b, double *x,
                        double tol, int maxit, int *iters, double *res_proj, double *res) {
  orc_level *L = Q->L;
  int64_t n = L->nl;
  int k = Q->nvec;
  double *c = malloc(sizeof(double) * (k + 1));
  double *bp = malloc(sizeof(double) * n), *dx = calloc(n, sizeof(double)),
         *w = malloc(sizeof(double) * n);
  for (int i = 0; i < k; ++i) c[i] = orc_level_dot(L, Q->P + (size_t)i * n, b);
  for (int64_t l = 0; l < n; ++l) {
    double xb = 0.0, ab = 0.0;
    for (int i = 0; i < k; ++i) {
      xb += c[i] * Q->P[(size_t)i * n + l];
      ab += c[i] * Q->AP[(size_t)i * n + l];
    }
    x[l] = xb;
    bp[l] = b[l] - ab;
  }
  double bnorm = sqrt(orc_level_dot(L, b, b));
  double bpn = sqrt(orc_level_dot(L, bp, bp));
  *res_proj = bpn;
  double tin = bpn > 0.0 ? tol * bnorm / bpn : 0.0;
  int st = 0;
  double r0, r1;
  *iters = 0;
  if (bpn > tol * bnorm) {
    if (solver == 1) st = orc_fgmres(Pm, 1, bp, dx, tin, m, maxit, iters, &r0, &r1, NULL);
    else st = orc_flexpcg(Pm, 1, bp, dx, tin, maxit, iters, &r0, &r1);
  }
  for (int64_t l = 0; l < n; ++l) x[l] += dx[l];
  /* grow the space with the correction, or restart from the full solution */
  if (bpn > tol * bnorm) {
    if (Q->nvec == Q->Lmax) {
      Q->nvec = 0;
      orc_level_ax(L, x, w);
      proj_add(Q, x, w);
    } else {
      orc_level_ax(L, dx, w);
      proj_add(Q, dx, w);
    }
  }
  orc_level_ax(L, x, w);
  for (int64_t l = 0; l < n; ++l) w[l] = b[l] - w[l];
  *res = sqrt(orc_level_dot(L, w, w));
  free(c); free(bp); free(dx); free(w);
  return st;
}
