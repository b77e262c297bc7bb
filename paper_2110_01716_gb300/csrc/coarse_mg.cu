// coarse_mg.cu -- multigrid-preconditioned coarse solve on the N = 1 lattice.
//
// The paper treats its N = 1 coarse grid with algebraic multigrid (Sec. 4,
// Table 1: the coarse grid falls from 45% to 11% of the run once it is
// handled well).  Here the coarse problem is the 27-point trilinear stencil
// on the (ex+1)(ey+1)(ez+1) lattice, and plain Jacobi-PCG needs O(lattice
// size) iterations, each limited by grid-wide latency.  This mode instead
// runs flexible CG (FP64) preconditioned by one geometric multigrid V(2,2)
// cycle per iteration, inside one persistent cooperative kernel:
//  * levels: lattice coarsened by two per direction (even indices plus the
//    last), index-space trilinear prolongation P = Pz x Py x Px, restriction
//    P^T, Galerkin operators P^T A P (27-point stencils, built on the device in
//    FP64, in a fixed order);
//  * smoother: degree-2 Chebyshev-Jacobi on [lambda/10, lambda], lambda =
//    1.1 x a power-iteration estimate of lambda_max(D^-1 A);
//  * bottom: dense inverse (Neumann: of A + c 1 1^T, exact on mean-free data);
//  * Dirichlet nodes are eliminated on every level (rows and unknowns zero).
// The iterations stop at the same relative tolerance and cap as the Jacobi
// mode, which remains the default.
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "coarse.cuh"
#include "kernels.cuh"
#include "reduce.cuh"
#include "trace.cuh"

namespace cg = cooperative_groups;

namespace sem {

constexpr int kMgThreads = 256;
#ifndef SEM_MG_MAX_BOTTOM
#define SEM_MG_MAX_BOTTOM 128
#endif
constexpr int kMgMaxBottom = SEM_MG_MAX_BOTTOM;  // unknowns of the dense bottom level

template <typename T>
__device__ __forceinline__ void mg_coords(const MgLevelT<T> &L, int g, int &gx, int &gy, int &gz) {
  const uint32_t u = (uint32_t)g;
  gz = (int)L.div_nxy.div(u);
  const uint32_t rem = u - (uint32_t)gz * (uint32_t)(L.nx * L.ny);
  gy = (int)L.div_nx.div(rem);
  gx = (int)(rem - (uint32_t)gy * (uint32_t)L.nx);
}

// (A v)_g of the 27-point stencil.  The neighbour tests come first and every
// load is a select on its own test, so the loads of all 27 neighbours are in
// flight together (a load is issued only for a neighbour inside the lattice).
template <typename T>
__device__ __forceinline__ T mg_apply(const MgLevelT<T> &L, int g, const T *__restrict__ v) {
  // the keep flag is read beside the stencil's loads, not before them (every
  // node has a stencil row, so the loads are in bounds either way)
  const bool kept = L.keep[g] != 0;
  int gx, gy, gz;
  mg_coords(L, g, gx, gy, gz);
  const bool in_x[3] = {gx > 0, true, gx < L.nx - 1};
  const bool in_y[3] = {gy > 0, true, gy < L.ny - 1};
  const bool in_z[3] = {gz > 0, true, gz < L.nz - 1};
  T sv[27], vv[27];
#pragma unroll
  for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        const int d = (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1);
        const bool ok = in_x[dx + 1] && in_y[dy + 1] && in_z[dz + 1];
        sv[d] = ok ? L.S[(int64_t)d * L.n + g] : (T)0;
        vv[d] = ok ? v[g + dx + L.nx * (dy + L.ny * dz)] : (T)0;
      }
  T acc = 0;
#pragma unroll
  for (int d = 0; d < 27; ++d) acc = fma(sv[d], vv[d], acc);
  return kept ? acc : (T)0;
}

// Grid-wide sums identical in every CTA (warp 0 reduces; see coarse.cu).
template <int NS>
__device__ void mg_sum(double (&v)[NS], double *part, cg::grid_group &grid) {
  __shared__ double sh[NS][kMgThreads / 32];
  __shared__ double res[NS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    double x = v[s];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) sh[s][warp] = x;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      double x = lane < kMgThreads / 32 ? sh[s][lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      if (lane == 0) part[(size_t)blockIdx.x * NS + s] = x;
    }
  }
  grid.sync();
  if (warp == 0) {
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      double x = 0.0;
      for (int b = lane; b < (int)gridDim.x; b += 32) x += __ldcg(&part[(size_t)b * NS + s]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      if (lane == 0) res[s] = x;
    }
  }
  __syncthreads();
#pragma unroll
  for (int s = 0; s < NS; ++s) v[s] = res[s];
}

// Barriers of the two execution modes of the V-cycle: the whole grid, or one
// CTA (the small coarse levels, where a grid barrier would cost more than the
// work between barriers).
struct GridBarrier {
  cg::grid_group *g;
  __device__ void operator()() const { g->sync(); }
};
struct CtaBarrier {
  __device__ void operator()() const { __syncthreads(); }
};

// Down the cycle at level l: pre-smoothing from zero (d = Dinv b / theta,
// x = d, r = b; one more step), residual, restriction to level l + 1.  Every
// phase maps node g to the same thread, so pointwise dependencies need no
// barrier; a barrier precedes every phase that reads neighbours or another
// level.  The restriction writes node G of level l + 1 from the thread that
// starts level l + 1's smoothing at G (a pointwise step), so the barrier
// after it is needed only when level l + 1 is run another way (by another
// set of threads, or the dense bottom): `last_barrier`.
template <typename Bar>
__device__ void mg_down(const MgArgs &A, int l, Bar bar, int tid, int nth, bool last_barrier) {
  const MgLevelT<float> &L = A.V[l];
  const float *b = L.b;
  float *x = L.x;
  for (int g = tid; g < L.n; g += nth) {
    const float rg = b[g];
    L.r[g] = rg;
    const float d = L.dinv[g] * rg * L.inv_theta;
    L.da[g] = d;
    x[g] = d;
  }
  bar();
  for (int g = tid; g < L.n; g += nth) {
    const float rg = L.r[g] - mg_apply(L, g, L.da);
    L.r[g] = rg;
    const float d = L.c1 * L.da[g] + L.c2 * L.dinv[g] * rg;
    L.db[g] = d;
    x[g] += d;
  }
  bar();
  for (int g = tid; g < L.n; g += nth) L.r[g] = b[g] - mg_apply(L, g, x);
  bar();
  const MgLevelT<float> &C = A.V[l + 1];
  for (int G = tid; G < C.n; G += nth) {
    float acc = 0.f;
    const bool kept = C.keep[G] != 0;  // applied at the end, not waited for
    {
      int Gx, Gy, Gz;
      mg_coords(C, G, Gx, Gy, Gz);
      // table rows first (index -1: no fine point), then guarded loads
      int fi[3][3];
      float fw[3][3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        fi[0][c] = L.ri[0][3 * Gx + c];
        fi[1][c] = L.ri[1][3 * Gy + c];
        fi[2][c] = L.ri[2][3 * Gz + c];
        fw[0][c] = L.rw[0][3 * Gx + c];
        fw[1][c] = L.rw[1][3 * Gy + c];
        fw[2][c] = L.rw[2][3 * Gz + c];
      }
      float rv[27];
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int b2 = 0; b2 < 3; ++b2)
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            const bool ok = fi[2][c] >= 0 && fi[1][b2] >= 0 && fi[0][a] >= 0;
            rv[a + 3 * (b2 + 3 * c)] = ok ? L.r[fi[0][a] + L.nx * (fi[1][b2] + L.ny * fi[2][c])] : 0.f;
          }
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int b2 = 0; b2 < 3; ++b2) {
          const float wyz = fw[2][c] * fw[1][b2];
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            const bool ok = fi[2][c] >= 0 && fi[1][b2] >= 0 && fi[0][a] >= 0;
            if (ok) acc = fma(wyz * fw[0][a], rv[a + 3 * (b2 + 3 * c)], acc);
          }
        }
    }
    C.b[G] = kept ? acc : 0.f;
  }
  if (last_barrier) bar();
}

// The bottom: dense inverse, one row per thread.
template <typename Bar>
__device__ void mg_bottom(const MgArgs &A, Bar bar, int tid, int nth) {
  const MgLevelT<float> &B = A.V[A.nlev - 1];
  for (int i = tid; i < A.nbottom; i += nth) {
    float acc = 0.f;
    for (int j = 0; j < A.nbottom; ++j) acc = fmaf(A.bottom_inv[(size_t)i * A.nbottom + j], B.b[j], acc);
    B.x[i] = acc;
  }
  bar();
}

// Up the cycle at level l: prolongation and correction from level l + 1,
// post-smoothing (r = b - A x; d = Dinv r / theta; x += d; one more step).
// The first step's x += d waits for the second step, whose phase reads only
// d's neighbours: one barrier fewer, the same arithmetic.
template <typename Bar>
__device__ void mg_up(const MgArgs &A, int l, Bar bar, int tid, int nth) {
  const MgLevelT<float> &L = A.V[l];
  const MgLevelT<float> &C = A.V[l + 1];
  const float *b = L.b;
  float *x = L.x;
  for (int g = tid; g < L.n; g += nth) {
    const bool kept = L.keep[g] != 0;  // applied at the end, not waited for
    int gx, gy, gz;
    mg_coords(L, g, gx, gy, gz);
    int ci[3][2];
    float cw[3][2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      ci[0][c] = L.pi[0][2 * gx + c];
      ci[1][c] = L.pi[1][2 * gy + c];
      ci[2][c] = L.pi[2][2 * gz + c];
      cw[0][c] = L.pw[0][2 * gx + c];
      cw[1][c] = L.pw[1][2 * gy + c];
      cw[2][c] = L.pw[2][2 * gz + c];
    }
    float xv[8];
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int b2 = 0; b2 < 2; ++b2)
#pragma unroll
        for (int a = 0; a < 2; ++a) {
          const bool ok = ci[2][c] >= 0 && ci[1][b2] >= 0 && ci[0][a] >= 0;
          xv[a + 2 * (b2 + 2 * c)] = ok ? C.x[ci[0][a] + C.nx * (ci[1][b2] + C.ny * ci[2][c])] : 0.f;
        }
    float acc = 0.f;
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int b2 = 0; b2 < 2; ++b2) {
        const float wyz = cw[2][c] * cw[1][b2];
#pragma unroll
        for (int a = 0; a < 2; ++a) {
          const bool ok = ci[2][c] >= 0 && ci[1][b2] >= 0 && ci[0][a] >= 0;
          if (ok) acc = fma(wyz * cw[0][a], xv[a + 2 * (b2 + 2 * c)], acc);
        }
      }
    if (kept) x[g] += acc;
  }
  bar();
  for (int g = tid; g < L.n; g += nth) {
    const float rg = b[g] - mg_apply(L, g, x);
    L.r[g] = rg;
    L.da[g] = L.dinv[g] * rg * L.inv_theta;
  }
  bar();
  for (int g = tid; g < L.n; g += nth) {
    const float rg = L.r[g] - mg_apply(L, g, L.da);
    L.r[g] = rg;
    const float d = L.c1 * L.da[g] + L.c2 * L.dinv[g] * rg;
    x[g] = (x[g] + L.da[g]) + d;
  }
  bar();
}

// One V(2,2) cycle in FP32 (the preconditioner of the FP64 flexible CG):
// level-0 right-hand side b0, result x0 (both FP64 level-0 vectors, b0 read
// only; converted on the way in and out).  Levels from A.small_from down (and
// the bottom) run in CTA 0 alone with CTA barriers while the other CTAs wait
// at one grid barrier.
__device__ void mg_vcycle(const MgArgs &A, const double *__restrict__ b0, double *__restrict__ x0,
                          cg::grid_group &grid, int tid, int nth) {
  const GridBarrier gb{&grid};
  const int ls = A.small_from;  // first level handled by CTA 0 (nlev - 1: the bottom only)
  const MgLevelT<float> &V0 = A.V[0];
  for (int g = tid; g < V0.n; g += nth) V0.b[g] = (float)b0[g];
  if (ls == 0) grid.sync();  // CTA 0 reads every node of level 0
  for (int l = 0; l < ls; ++l) mg_down(A, l, gb, tid, nth, l + 1 >= ls);
  if (ls == A.nlev - 1 && A.nbottom > (int)blockDim.x) {
    mg_bottom(A, gb, tid, nth);  // a large bottom: rows across the grid
  } else {
    if (blockIdx.x == 0) {
      const CtaBarrier cb;
      const int t = threadIdx.x, n = blockDim.x;
      for (int l = ls; l < A.nlev - 1; ++l) mg_down(A, l, cb, t, n, l + 1 == A.nlev - 1);
      mg_bottom(A, cb, t, n);
      for (int l = A.nlev - 2; l >= ls; --l) mg_up(A, l, cb, t, n);
    }
    grid.sync();
  }
  for (int l = ls - 1; l >= 0; --l) mg_up(A, l, gb, tid, nth);
  for (int g = tid; g < V0.n; g += nth) x0[g] = (double)V0.x[g];
}

__global__ void __launch_bounds__(kMgThreads) coarse_mgcg_kernel(MgArgs A) {
  cg::grid_group grid = cg::this_grid();
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nth = gridDim.x * blockDim.x;
  const MgLevelT<double> &L0 = A.L0;
  // right-hand side to unique layout (owner copy), x = 0
  double v1[1] = {0.0};
  for (int g = tid; g < L0.n; g += nth) {
    int gx, gy, gz;
    mg_coords(L0, g, gx, gy, gz);
    const int ix = min(gx, A.ex - 1), iy = min(gy, A.ey - 1), iz = min(gz, A.ez - 1);
    const int64_t e = ix + (int64_t)A.ex * (iy + (int64_t)A.ey * iz);
    const int a = (gx - ix) + 2 * (gy - iy) + 4 * (gz - iz);
    const double bg = A.b_local[e * 8 + a];
    A.r[g] = bg;
    A.x[g] = 0.0;
    v1[0] += bg;
  }
  if (A.bc == SEM_NEUMANN) {
    mg_sum<1>(v1, A.partM, grid);
    const double mean = v1[0] / (double)L0.n;
    for (int g = tid; g < L0.n; g += nth) A.r[g] -= mean;
  }
  grid.sync();
  mg_vcycle(A, A.r, A.z, grid, tid, nth);
  double v2[2] = {0.0, 0.0};  // rho = (r,z), rr = (r,r)
  for (int g = tid; g < L0.n; g += nth) {
    const double rg = A.r[g];
    v2[0] = fma(rg, A.z[g], v2[0]);
    v2[1] = fma(rg, rg, v2[1]);
    A.p[g] = A.z[g];
  }
  mg_sum<2>(v2, A.partI, grid);
  const double bb = v2[1];
  double rho = v2[0];
  int it = 0;
  if (bb > 0.0 && A.maxit > 0 && rho != 0.0) {
    for (;;) {
      ++it;
      double v[1] = {0.0};
      for (int g = tid; g < L0.n; g += nth) {
        const double wg = mg_apply(L0, g, A.p);
        A.w[g] = wg;
        v[0] = fma(A.p[g], wg, v[0]);
      }
      mg_sum<1>(v, A.partA, grid);
      const double pw = v[0];
      const double alpha = rho / pw;
      // the update with (r,r): the stopping test comes before the
      // preconditioner, whose output the last iteration would not use (the
      // reduction's grid barrier is also the one the V-cycle needs first)
      double q[1] = {0.0};
      for (int g = tid; g < L0.n; g += nth) {
        A.x[g] = fma(alpha, A.p[g], A.x[g]);
        const double rg = fma(-alpha, A.w[g], A.r[g]);
        A.r[g] = rg;
        q[0] = fma(rg, rg, q[0]);
      }
      mg_sum<1>(q, A.partM, grid);
      if (!(q[0] > A.tol2 * bb) || it >= A.maxit || !(q[0] == q[0])) break;
      mg_vcycle(A, A.r, A.z, grid, tid, nth);
      double u[2] = {0.0, 0.0};  // (r,z), (z,w)
      for (int g = tid; g < L0.n; g += nth) {
        const double zg = A.z[g];
        u[0] = fma(A.r[g], zg, u[0]);
        u[1] = fma(zg, A.w[g], u[1]);
      }
      mg_sum<2>(u, A.partK, grid);
      if (u[0] == 0.0) break;
      // flexible (Polak-Ribiere) coefficient: (z_new, r_new - r_old) / rho
      const double beta = -alpha * u[1] / rho;
      rho = u[0];
      for (int g = tid; g < L0.n; g += nth) A.p[g] = fma(beta, A.p[g], A.z[g]);
      grid.sync();  // the next product reads the neighbours' p
    }
  }
  grid.sync();
  const int64_t nloc = (int64_t)A.ex * A.ey * A.ez * 8;
  for (int64_t l = tid; l < nloc; l += nth) {
    const uint32_t e = (uint32_t)(l >> 3);
    const int a = (int)(l & 7);
    const uint32_t yz = A.div_ex.div(e);
    const int ix = (int)(e - yz * (uint32_t)A.ex);
    const int iz = (int)A.div_ey.div(yz);
    const int iy = (int)(yz - (uint32_t)iz * (uint32_t)A.ey);
    const int g = (ix + (a & 1)) + L0.nx * ((iy + ((a >> 1) & 1)) + L0.ny * (iz + (a >> 2)));
    A.x_local[l] = A.x[g];
  }
  if (tid == 0) *A.iters = it;
}

// ------------------------------------------------------------------ device setup
// The hierarchy is built on the device: Galerkin stencils by a gather over
// each coarse point's fine support, keep masks and Jacobi inverses, and the
// power iterations of the Chebyshev bounds.  The host keeps the 1D transfer
// tables and inverts the dense bottom (at most kMgMaxBottom unknowns).

// 1D transfer tables of one level pair (device), per direction.
struct GalerkinTables {
  const int *pi[3];     // [2 nf]: coarse indices of fine point i (-1: none)
  const double *pw[3];  // [2 nf]: their weights
  const int *ri[3];     // [3 nc]: fine indices of coarse point k (-1: none)
  const double *rw[3];  // [3 nc]: their weights (the transposed prolongation)
};

// keep = not on the Dirichlet boundary; dinv = 1 / diagonal (0 where not
// kept or where the diagonal is zero).
__global__ void mg_finish_kernel(int nx, int ny, int nz, int dirichlet, const double *__restrict__ S,
                                 unsigned char *__restrict__ keep, double *__restrict__ dinv) {
  const int n = nx * ny * nz;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < n; g += gridDim.x * blockDim.x) {
    const int x = g % nx, y = (g / nx) % ny, z = g / (nx * ny);
    const bool bnd = dirichlet && (x == 0 || y == 0 || z == 0 || x == nx - 1 || y == ny - 1 ||
                                   z == nz - 1);
    keep[g] = bnd ? 0 : 1;
    const double dg = S[(size_t)13 * n + g];
    dinv[g] = !bnd && dg != 0.0 ? 1.0 / dg : 0.0;
  }
}

// A_c = P^T A P over the fine unknowns, one coarse point I per thread:
// A_c[I][J] = sum_f R[I][f] sum_g A[f][g] P[g][J] over kept fine f in I's
// support and kept stencil neighbours g of f.  Each term is formed as
// (w_I a) w_J with w = w_z w_y w_x, the factors in the host's order.
__global__ void mg_galerkin_kernel(int fnx, int fny, int fnz, const double *__restrict__ SF,
                                   const unsigned char *__restrict__ keepF, int cnx, int cny, int cnz,
                                   GalerkinTables T, double *__restrict__ SC, int *bad) {
  const int fn = fnx * fny * fnz, cn = cnx * cny * cnz;
  for (int I = blockIdx.x * blockDim.x + threadIdx.x; I < cn; I += gridDim.x * blockDim.x) {
    const int Ix = I % cnx, Iy = (I / cnx) % cny, Iz = I / (cnx * cny);
    double acc[27];
    for (int q = 0; q < 27; ++q) acc[q] = 0.0;
    for (int c1 = 0; c1 < 3; ++c1) {
      const int fz = T.ri[2][3 * Iz + c1];
      if (fz < 0) continue;
      for (int b1 = 0; b1 < 3; ++b1) {
        const int fy = T.ri[1][3 * Iy + b1];
        if (fy < 0) continue;
        for (int a1 = 0; a1 < 3; ++a1) {
          const int fx = T.ri[0][3 * Ix + a1];
          if (fx < 0) continue;
          const int f = fx + fnx * (fy + fny * fz);
          if (!keepF[f]) continue;
          const double wI = T.rw[2][3 * Iz + c1] * T.rw[1][3 * Iy + b1] * T.rw[0][3 * Ix + a1];
          for (int d = 0; d < 27; ++d) {
            const int gx = fx + d % 3 - 1, gy = fy + (d / 3) % 3 - 1, gz = fz + d / 9 - 1;
            if (gx < 0 || gy < 0 || gz < 0 || gx >= fnx || gy >= fny || gz >= fnz) continue;
            if (!keepF[gx + fnx * (gy + fny * gz)]) continue;
            const double a = SF[(size_t)d * fn + f];
            if (a == 0.0) continue;
            const double wa = wI * a;
            for (int c2 = 0; c2 < 2; ++c2) {
              const int Jz = T.pi[2][2 * gz + c2];
              if (Jz < 0) continue;
              for (int b2 = 0; b2 < 2; ++b2) {
                const int Jy = T.pi[1][2 * gy + b2];
                if (Jy < 0) continue;
                for (int a2 = 0; a2 < 2; ++a2) {
                  const int Jx = T.pi[0][2 * gx + a2];
                  if (Jx < 0) continue;
                  const int ox = Jx - Ix, oy = Jy - Iy, oz = Jz - Iz;
                  if (ox < -1 || ox > 1 || oy < -1 || oy > 1 || oz < -1 || oz > 1) {
                    atomicExch(bad, 1);
                    continue;
                  }
                  const double wJ = T.pw[2][2 * gz + c2] * T.pw[1][2 * gy + b2] * T.pw[0][2 * gx + a2];
                  acc[(ox + 1) + 3 * (oy + 1) + 9 * (oz + 1)] += wa * wJ;
                }
              }
            }
          }
        }
      }
    }
    for (int q = 0; q < 27; ++q) SC[(size_t)q * cn + I] = acc[q];
  }
}

// Start vector of the power iterations: 1 + sin(0.7 g + 0.3) / 2 on kept nodes.
__global__ void mg_power_start_kernel(int n, const unsigned char *__restrict__ keep,
                                      double *__restrict__ v) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < n; g += gridDim.x * blockDim.x)
    v[g] = keep[g] ? 1.0 + 0.5 * sin(0.7 * g + 0.3) : 0.0;
}

// One power step: w = D^-1 A v over kept nodes, and <v, v>, <v, w> (the
// Rayleigh quotient of v is the second over the first).
__global__ void __launch_bounds__(kVecThreads)
    mg_power_step_kernel(int nx, int ny, int nz, const double *__restrict__ S,
                         const unsigned char *__restrict__ keep, const double *__restrict__ dinv,
                         const double *__restrict__ v, double *__restrict__ w, double *partials,
                         unsigned int *counter, OutPtrs<2> out) {
  const int n = nx * ny * nz;
  double acc[2] = {0.0, 0.0};
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < n; g += gridDim.x * blockDim.x) {
    double a = 0.0;
    if (keep[g]) {
      const int gx = g % nx, gy = (g / nx) % ny, gz = g / (nx * ny);
      for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            const int x = gx + dx, y = gy + dy, z = gz + dz;
            if (x < 0 || y < 0 || z < 0 || x >= nx || y >= ny || z >= nz) continue;
            const int nb = x + nx * (y + ny * z);
            if (!keep[nb]) continue;
            a += S[(size_t)((dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)) * n + g] * v[nb];
          }
    }
    const double wg = dinv[g] * a;
    w[g] = wg;
    acc[0] = fma(v[g], v[g], acc[0]);
    acc[1] = fma(v[g], wg, acc[1]);
  }
  grid_reduce<2>(acc, partials, counter, out.p);
}

// FP64 -> FP32, rounded to nearest (the V-cycle's copies of the operators).
__global__ void mg_narrow_kernel(size_t n, const double *__restrict__ a, float *__restrict__ b) {
  for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (size_t)gridDim.x * blockDim.x)
    b[q] = (float)a[q];
}

// ------------------------------------------------------------------ host setup
namespace {

// The dense bottom level on the host.
struct HostLevel {
  int nx, ny, nz, n;
  std::vector<double> S;            // [27][n]
  std::vector<unsigned char> keep;  // unknowns
};

// Coarse points of a 1D lattice of n points: the even indices and the last.
std::vector<int> coarse_points(int n) {
  std::vector<int> c;
  for (int i = 0; i < n; i += 2) c.push_back(i);
  if (c.back() != n - 1) c.push_back(n - 1);
  return c;
}

// Prolongation rows (fine index -> up to two (coarse index, weight)).
void prolong_1d(int n, std::vector<int> &pi, std::vector<double> &pw, std::vector<int> &ri,
                std::vector<double> &rw, int &nc) {
  const std::vector<int> c = coarse_points(n);
  nc = (int)c.size();
  std::vector<int> cidx(n, -1);
  for (int k = 0; k < nc; ++k) cidx[c[k]] = k;
  pi.assign(2 * n, -1);
  pw.assign(2 * n, 0.0);
  for (int i = 0; i < n; ++i) {
    if (cidx[i] >= 0) {
      pi[2 * i] = cidx[i];
      pw[2 * i] = 1.0;
    } else {
      pi[2 * i] = cidx[i - 1];
      pw[2 * i] = 0.5;
      pi[2 * i + 1] = cidx[i + 1];
      pw[2 * i + 1] = 0.5;
    }
  }
  ri.assign(3 * nc, -1);
  rw.assign(3 * nc, 0.0);
  std::vector<int> cnt(nc, 0);
  for (int i = 0; i < n; ++i)
    for (int q = 0; q < 2; ++q)
      if (pi[2 * i + q] >= 0) {
        const int k = pi[2 * i + q];
        ri[3 * k + cnt[k]] = i;
        rw[3 * k + cnt[k]] = pw[2 * i + q];
        ++cnt[k];
      }
}

double apply_host(const HostLevel &L, int g, const std::vector<double> &v) {
  if (!L.keep[g]) return 0.0;
  const int gx = g % L.nx, gy = (g / L.nx) % L.ny, gz = g / (L.nx * L.ny);
  double acc = 0.0;
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        const int x = gx + dx, y = gy + dy, z = gz + dz;
        if (x < 0 || y < 0 || z < 0 || x >= L.nx || y >= L.ny || z >= L.nz) continue;
        const int nb = x + L.nx * (y + L.ny * z);
        if (!L.keep[nb]) continue;
        acc += L.S[(size_t)((dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)) * L.n + g] * v[nb];
      }
  return acc;
}

}  // namespace

void coarse_mg_setup(CoarseSolver &C, const Level &Lv, cudaStream_t st, int max_ctas) {
  const int nx0 = Lv.t.ex + 1, ny0 = Lv.t.ey + 1, nz0 = Lv.t.ez + 1;
  const int n0 = nx0 * ny0 * nz0;
  std::unique_ptr<CoarseMg> M(new CoarseMg());
  const bool dir = Lv.t.bc == SEM_DIRICHLET;
  // FP64 operators of the levels, on the device: level 0 is the coarse
  // solver's own stencil; the others are Galerkin products of their finer
  // level.  Every level gets its keep mask and Jacobi inverse.
  struct DevLevel {
    int nx = 0, ny = 0, nz = 0, n = 0;
    const double *S = nullptr;
    DevBuf<double> Sbuf, dinv;
    DevBuf<unsigned char> keep;
    double lam_hi = 0.0;
  };
  std::vector<std::unique_ptr<DevLevel>> H;
  auto finish = [&](DevLevel &L) {
    L.keep.alloc(L.n);
    L.dinv.alloc(L.n);
    const int g = (int)std::min<int64_t>((L.n + 255) / 256, 152 * 8);
    mg_finish_kernel<<<g, 256, 0, st>>>(L.nx, L.ny, L.nz, dir ? 1 : 0, L.S, L.keep.p, L.dinv.p);
    SEM_CHECK_CUDA(cudaGetLastError());
  };
  H.emplace_back(new DevLevel());
  H[0]->nx = nx0; H[0]->ny = ny0; H[0]->nz = nz0; H[0]->n = n0;
  H[0]->S = C.S.p;
  finish(*H[0]);
  // transfer tables (host) and Galerkin operators (device)
  std::vector<std::vector<int>> PI[3], RI[3];
  std::vector<std::vector<double>> PW[3], RW[3];
  DevBuf<int> bad;
  bad.alloc(1);
  SEM_CHECK_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), st));
  std::vector<std::unique_ptr<DevBuf<int>>> tab_i;
  std::vector<std::unique_ptr<DevBuf<double>>> tab_d;
  auto to_dev_i = [&](const std::vector<int> &v) {
    tab_i.emplace_back(new DevBuf<int>());
    tab_i.back()->alloc(v.size());
    SEM_CHECK_CUDA(cudaMemcpyAsync(tab_i.back()->p, v.data(), v.size() * sizeof(int),
                                   cudaMemcpyHostToDevice, st));
    return (const int *)tab_i.back()->p;
  };
  auto to_dev_d = [&](const std::vector<double> &v) {
    tab_d.emplace_back(new DevBuf<double>());
    tab_d.back()->alloc(v.size());
    SEM_CHECK_CUDA(cudaMemcpyAsync(tab_d.back()->p, v.data(), v.size() * sizeof(double),
                                   cudaMemcpyHostToDevice, st));
    return (const double *)tab_d.back()->p;
  };
  while ((int)H.size() < kMgMaxLevels && H.back()->n > kMgMaxBottom &&
         std::min({H.back()->nx, H.back()->ny, H.back()->nz}) > 3) {
    const DevLevel &F = *H.back();
    int ncd[3];
    std::vector<int> pi[3], ri[3];
    std::vector<double> pw[3], rw[3];
    const int nf[3] = {F.nx, F.ny, F.nz};
    GalerkinTables T;
    for (int d = 0; d < 3; ++d) {
      prolong_1d(nf[d], pi[d], pw[d], ri[d], rw[d], ncd[d]);
      T.pi[d] = to_dev_i(pi[d]);
      T.pw[d] = to_dev_d(pw[d]);
      T.ri[d] = to_dev_i(ri[d]);
      T.rw[d] = to_dev_d(rw[d]);
    }
    std::unique_ptr<DevLevel> Cl(new DevLevel());
    Cl->nx = ncd[0]; Cl->ny = ncd[1]; Cl->nz = ncd[2];
    Cl->n = Cl->nx * Cl->ny * Cl->nz;
    Cl->Sbuf.alloc((size_t)27 * Cl->n);
    Cl->S = Cl->Sbuf.p;
    const int g = (int)std::min<int64_t>((Cl->n + 127) / 128, 152 * 8);
    mg_galerkin_kernel<<<g, 128, 0, st>>>(F.nx, F.ny, F.nz, F.S, F.keep.p, Cl->nx, Cl->ny, Cl->nz,
                                          T, Cl->Sbuf.p, bad.p);
    SEM_CHECK_CUDA(cudaGetLastError());
    finish(*Cl);
    for (int d = 0; d < 3; ++d) {
      PI[d].push_back(pi[d]); PW[d].push_back(pw[d]);
      RI[d].push_back(ri[d]); RW[d].push_back(rw[d]);
    }
    H.push_back(std::move(Cl));
  }
  SEM_REQUIRE(H.back()->n <= kMgMaxBottom, "coarse lattice too elongated for the multigrid mode");
  // Chebyshev bounds (smoothed levels): 30 power steps each on the device
  {
    Reducer R;
    R.init(kVecMaxBlocks, 2);
    DevBuf<double> pv, slots;
    size_t nmax = 0;
    for (size_t l = 0; l + 1 < H.size(); ++l) nmax = std::max(nmax, (size_t)H[l]->n);
    pv.alloc(2 * std::max<size_t>(nmax, 1));
    slots.alloc(2 * std::max<size_t>(H.size(), 1));
    for (size_t l = 0; l + 1 < H.size(); ++l) {
      const DevLevel &L = *H[l];
      double *v = pv.p, *w = pv.p + nmax;
      const int g = vec_grid(L.n);
      mg_power_start_kernel<<<g, kVecThreads, 0, st>>>(L.n, L.keep.p, v);
      SEM_CHECK_CUDA(cudaGetLastError());
      OutPtrs<2> o{{slots.p + 2 * l, slots.p + 2 * l + 1}};
      for (int it = 0; it < 30; ++it) {
        mg_power_step_kernel<<<g, kVecThreads, 0, st>>>(L.nx, L.ny, L.nz, L.S, L.keep.p, L.dinv.p, v,
                                                         w, R.partials.p, R.counter.p, o);
        SEM_CHECK_CUDA(cudaGetLastError());
        std::swap(v, w);
      }
    }
    std::vector<double> hs(2 * H.size(), 0.0);
    SEM_CHECK_CUDA(cudaMemcpyAsync(hs.data(), slots.p, hs.size() * sizeof(double),
                                   cudaMemcpyDeviceToHost, st));
    int hbad = 0;
    SEM_CHECK_CUDA(cudaMemcpyAsync(&hbad, bad.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    SEM_CHECK_CUDA(cudaStreamSynchronize(st));
    SEM_REQUIRE(hbad == 0, "coarse stencil exceeds 27 points");
    for (size_t l = 0; l + 1 < H.size(); ++l)
      H[l]->lam_hi = 1.1 * (hs[2 * l] > 0.0 ? hs[2 * l + 1] / hs[2 * l] : 1.0);
  }
  // bottom: dense (Dirichlet rows -> identity; Neumann: + c 1 1^T), from the
  // last level's stencil and mask brought to the host
  HostLevel B;
  {
    const DevLevel &D = *H.back();
    B.nx = D.nx; B.ny = D.ny; B.nz = D.nz; B.n = D.n;
    B.S.resize((size_t)27 * D.n);
    B.keep.resize(D.n);
    SEM_CHECK_CUDA(cudaMemcpyAsync(B.S.data(), D.S, B.S.size() * sizeof(double),
                                   cudaMemcpyDeviceToHost, st));
    SEM_CHECK_CUDA(cudaMemcpyAsync(B.keep.data(), D.keep.p, B.keep.size(), cudaMemcpyDeviceToHost,
                                   st));
    SEM_CHECK_CUDA(cudaStreamSynchronize(st));
  }
  const int nb = B.n;
  std::vector<double> Ad((size_t)nb * nb, 0.0), inv((size_t)nb * nb, 0.0);
  {
    std::vector<double> e(nb, 0.0);
    for (int j = 0; j < nb; ++j) {
      std::fill(e.begin(), e.end(), 0.0);
      e[j] = 1.0;
      for (int i = 0; i < nb; ++i) Ad[(size_t)i * nb + j] = apply_host(B, i, e);
    }
    double dmean = 0.0;
    for (int i = 0; i < nb; ++i) dmean += Ad[(size_t)i * nb + i];
    dmean /= nb;
    for (int i = 0; i < nb; ++i)
      if (!B.keep[i]) {
        for (int j = 0; j < nb; ++j) Ad[(size_t)i * nb + j] = Ad[(size_t)j * nb + i] = 0.0;
        Ad[(size_t)i * nb + i] = 1.0;
      }
    if (!dir)
      for (size_t q = 0; q < Ad.size(); ++q) Ad[q] += dmean / nb;
    // Gauss-Jordan with partial pivoting
    std::vector<double> a = Ad;
    for (int i = 0; i < nb; ++i) inv[(size_t)i * nb + i] = 1.0;
    for (int col = 0; col < nb; ++col) {
      int piv = col;
      for (int r = col + 1; r < nb; ++r)
        if (std::fabs(a[(size_t)r * nb + col]) > std::fabs(a[(size_t)piv * nb + col])) piv = r;
      SEM_REQUIRE(a[(size_t)piv * nb + col] != 0.0, "singular bottom-level operator");
      if (piv != col)
        for (int k = 0; k < nb; ++k) {
          std::swap(a[(size_t)piv * nb + k], a[(size_t)col * nb + k]);
          std::swap(inv[(size_t)piv * nb + k], inv[(size_t)col * nb + k]);
        }
      const double d = 1.0 / a[(size_t)col * nb + col];
      for (int k = 0; k < nb; ++k) {
        a[(size_t)col * nb + k] *= d;
        inv[(size_t)col * nb + k] *= d;
      }
      for (int r = 0; r < nb; ++r) {
        if (r == col) continue;
        const double f = a[(size_t)r * nb + col];
        if (f == 0.0) continue;
        for (int k = 0; k < nb; ++k) {
          a[(size_t)r * nb + k] -= f * a[(size_t)col * nb + k];
          inv[(size_t)r * nb + k] -= f * inv[(size_t)col * nb + k];
        }
      }
    }
    for (int i = 0; i < nb; ++i)
      if (!B.keep[i])
        for (int j = 0; j < nb; ++j) inv[(size_t)i * nb + j] = 0.0;
  }
  // Device buffers of the FP32 V-cycle.  Every array carved out of the three
  // buffers starts on a 256-byte boundary: the unrolled gathers read
  // neighbouring table entries, which the compiler may merge into vector
  // loads that need that alignment.
  auto up = [](size_t n, size_t q) { return (n + q - 1) / q * q; };
  const int nlev = (int)H.size();
  size_t flt = up((size_t)nb * nb, 64), ints = 0;
  for (int l = 0; l < nlev; ++l) {
    flt += up((size_t)27 * H[l]->n, 64) + 6 * up(H[l]->n, 64);
    if (l + 1 < nlev)
      for (int d = 0; d < 3; ++d) {
        flt += up(PW[d][l].size(), 64) + up(RW[d][l].size(), 64);
        ints += up(PI[d][l].size(), 64) + up(RI[d][l].size(), 64);
      }
  }
  size_t keeps = 0;
  for (int l = 0; l < nlev; ++l) keeps += up(H[l]->n, 256);
  M->fbuf.alloc(flt);
  M->ibuf.alloc(ints > 0 ? ints : 1);
  M->kbuf.alloc(keeps);
  std::vector<float> hf(flt, 0.f);
  std::vector<int> hi(ints > 0 ? ints : 1, -1);
  std::vector<unsigned char> hk(keeps, 0);
  size_t of = 0, oi = 0, ok = 0;
  auto put = [&](const std::vector<double> &v) {  // FP32 copy (rounded to nearest)
    for (size_t q = 0; q < v.size(); ++q) hf[of + q] = (float)v[q];
    const float *dst = M->fbuf.p + of;
    of += up(v.size(), 64);
    return dst;
  };
  auto vec = [&](size_t n) {
    float *dst = M->fbuf.p + of;
    of += up(n, 64);
    return dst;
  };
  // FP32 copies of the levels' operators made on the device once the host
  // part of the buffers has been copied (dst, FP64 src, count), and the keep
  // masks copied likewise
  struct Narrow {
    float *dst;
    const double *src;
    size_t n;
  };
  struct KeepCopy {
    unsigned char *dst;
    const unsigned char *src;
    size_t n;
  };
  std::vector<Narrow> narrows;
  std::vector<KeepCopy> keepcopies;
  MgArgs &A = M->args;
  std::memset(&A, 0, sizeof(A));
  A.nlev = nlev;
  for (int l = 0; l < nlev; ++l) {
    const DevLevel &L = *H[l];
    MgLevelT<float> &D = A.V[l];
    D.nx = L.nx; D.ny = L.ny; D.nz = L.nz; D.n = L.n;
    D.div_nx = FastDiv((uint32_t)L.nx);
    D.div_nxy = FastDiv((uint32_t)(L.nx * L.ny));
    {
      float *dS = vec((size_t)27 * L.n);
      narrows.push_back({dS, L.S, (size_t)27 * L.n});
      D.S = dS;
      float *dD = vec(L.n);
      narrows.push_back({dD, L.dinv.p, (size_t)L.n});
      D.dinv = dD;
    }
    keepcopies.push_back({M->kbuf.p + ok, L.keep.p, (size_t)L.n});
    D.keep = M->kbuf.p + ok; ok += up(L.n, 256);
    D.x = vec(L.n);
    D.b = vec(L.n);
    D.r = vec(L.n);
    D.da = vec(L.n);
    D.db = vec(L.n);
    if (l + 1 < nlev) {
      const double theta = 0.5 * (L.lam_hi + L.lam_hi / 10.0);
      const double delta = 0.5 * (L.lam_hi - L.lam_hi / 10.0);
      const double sigma = theta / delta, rho0 = 1.0 / sigma;
      const double rho1 = 1.0 / (2.0 * sigma - rho0);
      D.inv_theta = (float)(1.0 / theta);
      D.c1 = (float)(rho1 * rho0);
      D.c2 = (float)(2.0 * rho1 / delta);
      for (int d = 0; d < 3; ++d) {
        std::copy(PI[d][l].begin(), PI[d][l].end(), hi.begin() + oi);
        D.pi[d] = M->ibuf.p + oi; oi += up(PI[d][l].size(), 64);
        std::copy(RI[d][l].begin(), RI[d][l].end(), hi.begin() + oi);
        D.ri[d] = M->ibuf.p + oi; oi += up(RI[d][l].size(), 64);
        D.pw[d] = put(PW[d][l]);
        D.rw[d] = put(RW[d][l]);
      }
    }
  }
  A.bottom_inv = put(inv);
  A.nbottom = nb;
  // level 0 of the flexible CG in FP64: the coarse solver's own stencil and
  // Jacobi inverse, the keep mask of the hierarchy
  A.L0.nx = nx0; A.L0.ny = ny0; A.L0.nz = nz0; A.L0.n = n0;
  A.L0.div_nx = A.V[0].div_nx;
  A.L0.div_nxy = A.V[0].div_nxy;
  A.L0.S = C.S.p;
  A.L0.dinv = C.dinv.p;
  A.L0.keep = A.V[0].keep;
#ifndef SEM_MG_SMALL
#define SEM_MG_SMALL 0
#endif
  // levels of at most SEM_MG_SMALL unknowns run in one CTA
  A.small_from = nlev - 1;
  for (int l = 0; l < nlev - 1; ++l)
    if (A.V[l].n <= SEM_MG_SMALL) {
      A.small_from = l;
      break;
    }
  SEM_REQUIRE(of <= flt && oi <= hi.size() && ok <= keeps, "multigrid buffer layout overflow");
  // guard: every device array of the hierarchy is 256-byte aligned
  auto aligned = [](const void *p) { return ((uintptr_t)p & 255u) == 0; };
  for (int l = 0; l < nlev; ++l) {
    const MgLevelT<float> &D = A.V[l];
    bool ok_al = aligned(D.S) && aligned(D.dinv) && aligned(D.keep) && aligned(D.r) &&
                 aligned(D.da) && aligned(D.db) && aligned(D.x) && aligned(D.b);
    if (l + 1 < nlev)
      for (int d = 0; d < 3; ++d)
        ok_al = ok_al && aligned(D.pi[d]) && aligned(D.pw[d]) && aligned(D.ri[d]) &&
                aligned(D.rw[d]);
    SEM_REQUIRE(ok_al, "multigrid arrays are not 256-byte aligned");
  }
  SEM_REQUIRE(aligned(A.bottom_inv), "multigrid arrays are not 256-byte aligned");
  SEM_CHECK_CUDA(cudaMemcpyAsync(M->fbuf.p, hf.data(), hf.size() * sizeof(float),
                                 cudaMemcpyHostToDevice, st));
  SEM_CHECK_CUDA(cudaMemcpyAsync(M->ibuf.p, hi.data(), hi.size() * sizeof(int),
                                 cudaMemcpyHostToDevice, st));
  SEM_CHECK_CUDA(cudaMemcpyAsync(M->kbuf.p, hk.data(), hk.size(), cudaMemcpyHostToDevice, st));
  for (const Narrow &q : narrows) {
    const int g = (int)std::min<size_t>((q.n + 255) / 256, 152 * 8);
    mg_narrow_kernel<<<g, 256, 0, st>>>(q.n, q.src, q.dst);
    SEM_CHECK_CUDA(cudaGetLastError());
  }
  for (const KeepCopy &q : keepcopies)
    SEM_CHECK_CUDA(cudaMemcpyAsync(q.dst, q.src, q.n, cudaMemcpyDeviceToDevice, st));
  A.ex = Lv.t.ex; A.ey = Lv.t.ey; A.ez = Lv.t.ez; A.bc = Lv.t.bc;
  A.div_ex = FastDiv((uint32_t)Lv.t.ex);
  A.div_ey = FastDiv((uint32_t)Lv.t.ey);
  const size_t s0 = C.vec_stride;
  A.x = C.vec.p; A.r = A.x + s0; A.z = A.r + s0; A.p = A.z + s0; A.w = A.p + s0;
  // grid: two CTAs per SM (more warps hide the stencil loads' latency; each
  // grid barrier costs a little more)
  int dev = 0, sms = 0, per_sm = 0;
  SEM_CHECK_CUDA(cudaGetDevice(&dev));
  SEM_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  SEM_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, coarse_mgcg_kernel,
                                                               kMgThreads, 0));
  SEM_REQUIRE(per_sm >= 1, "multigrid coarse kernel cannot be resident");
#ifndef SEM_MG_CTAS_PER_SM
#define SEM_MG_CTAS_PER_SM 2  // 1 / 2 / 4 measured 0.47 / 0.44 / 0.44 ms per coarse solve at 48^3
#endif
  M->grid = std::max(1, std::min(sms * std::min(per_sm, SEM_MG_CTAS_PER_SM),
                                 (n0 + kMgThreads - 1) / kMgThreads));
  if (max_ctas > 0 && M->grid > max_ctas) M->grid = max_ctas;
  const size_t ps = up((size_t)M->grid * 4, 32);
  M->part.alloc(4 * ps);
  A.partM = M->part.p;
  A.partI = A.partM + ps;
  A.partA = A.partI + ps;
  A.partK = A.partA + ps;
  A.iters = C.iters.p;
  M->levels = nlev;
  SEM_CHECK_CUDA(cudaStreamSynchronize(st));
  C.mg = std::move(M);
}

void coarse_mg_solve(CoarseSolver &C, const double *b_local, double *x_local, double tol,
                     int maxit, cudaStream_t st) {
  MgArgs A = C.mg->args;
  A.b_local = b_local;
  A.x_local = x_local;
  A.tol2 = tol > 0 ? tol * tol : 0.0;
  A.maxit = maxit;
  void *args[] = {&A};
  TraceScope ts("coarse_mgcg", 1, st);
  SEM_CHECK_CUDA(cudaLaunchCooperativeKernel((const void *)coarse_mgcg_kernel, dim3(C.mg->grid),
                                             dim3(kMgThreads), args, 0, st));
}

}  // namespace sem
