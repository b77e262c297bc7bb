// coarse.cu -- coarsest p-multigrid level (N = 1): FP64 Jacobi-PCG in one
// persistent cooperative kernel.
//
// The paper solves its N = 1 coarse grid with algebraic multigrid on the host
// (Sec. 4, Table 1 discussion).  On one GPU the coarse problem is small
// (about one unique node per element) and latency bound, so the whole CG
// iteration runs inside one launch: vectors live in unique-node layout
// (no duplicated copies), the operator is applied node by node from
// precomputed 8x8 element matrices (each node sums the rows of the at most 8
// elements that contain it, in a fixed order, so no atomics are needed), and
// the inner products use a two-stage grid reduction in which every CTA adds
// the per-CTA partials in the same order -- all CTAs obtain bit-identical
// scalars and take the same stopping decision.  Three grid barriers per
// iteration.
#include <cooperative_groups.h>

#include <algorithm>

#include "coarse.cuh"
#include "kernels.cuh"
#include "trace.cuh"

namespace cg = cooperative_groups;

namespace sem {

constexpr int kCoarseThreads = 256;

struct CoarseArgs {
  int ex, ey, ez;
  int nx, ny;  // lattice points along x and y
  int64_t ng;
  int bc;
  const double *Ae;    // [E][64]
  const double *dinv;  // [ng]
  const double *b_local;
  double *x_local;
  double *x, *r, *z, *p, *w;
  // Four partial-sum regions of grid*4 doubles: the mean, the initial sums,
  // <p,w> and (rr, rz).  Consecutive reductions use different regions, so a
  // CTA that races ahead never overwrites partials another CTA still reads.
  double *partM, *partI, *partA, *partB;
  int *iters;
  double tol2;
  int maxit;
};

__device__ __forceinline__ void node_coords(int64_t g, int nx, int ny, int &gx, int &gy, int &gz) {
  int64_t nxy = (int64_t)nx * ny;
  gz = (int)(g / nxy);
  int64_t rem = g - (int64_t)gz * nxy;
  gy = (int)(rem / nx);
  gx = (int)(rem - (int64_t)gy * nx);
}

// Block sum of NS values, then grid-wide sum identical in every CTA.
template <int NS>
__device__ void coop_sum(double (&v)[NS], double *part, cg::grid_group &grid) {
  __shared__ double sh[NS][kCoarseThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    double x = v[s];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) sh[s][warp] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      double x = 0.0;
      for (int q = 0; q < kCoarseThreads / 32; ++q) x += sh[s][q];
      part[(size_t)blockIdx.x * NS + s] = x;
    }
  }
  grid.sync();
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    double x = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
      x += __ldcg(&part[(size_t)b * NS + s]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    __syncthreads();
    if (lane == 0) sh[s][warp] = x;
    __syncthreads();
    double t = 0.0;
    for (int q = 0; q < kCoarseThreads / 32; ++q) t += sh[s][q];
    v[s] = t;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kCoarseThreads) coarse_cg_kernel(CoarseArgs A) {
  cg::grid_group grid = cg::this_grid();
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  const int ex = A.ex, ey = A.ey, ez = A.ez;
  // ---- right-hand side to unique layout (owner copy), x = 0
  double v1[1] = {0.0};
  for (int64_t g = tid; g < A.ng; g += nth) {
    int gx, gy, gz;
    node_coords(g, A.nx, A.ny, gx, gy, gz);
    int ix = min(gx, ex - 1), iy = min(gy, ey - 1), iz = min(gz, ez - 1);
    int64_t e = ix + (int64_t)ex * (iy + (int64_t)ey * iz);
    int a = (gx - ix) + 2 * (gy - iy) + 4 * (gz - iz);
    double bg = A.b_local[e * 8 + a];
    A.r[g] = bg;
    A.x[g] = 0.0;
    v1[0] += bg;
  }
  if (A.bc == SEM_NEUMANN) {
    // project onto the range: subtract the unique-node mean
    coop_sum<1>(v1, A.partM, grid);
    const double mean = v1[0] / (double)A.ng;
    for (int64_t g = tid; g < A.ng; g += nth) A.r[g] -= mean;
  }
  double v3[3] = {0.0, 0.0, 0.0};  // bb, rr, rz
  for (int64_t g = tid; g < A.ng; g += nth) {
    double rg = A.r[g];
    double zg = A.dinv[g] * rg;
    A.z[g] = zg;
    A.p[g] = zg;
    v3[0] = fma(rg, rg, v3[0]);
    v3[2] = fma(rg, zg, v3[2]);
  }
  v3[1] = v3[0];
  coop_sum<3>(v3, A.partI, grid);  // also orders the p writes before the first product
  const double bb = v3[0];
  double rr = v3[1], rho = v3[2];
  int it = 0;
  bool done = !(rr > A.tol2 * bb) || A.maxit <= 0;
  while (!done) {
    ++it;
    // ---- w = A p, node by node; pw = <p, w>
    double v[1] = {0.0};
    for (int64_t g = tid; g < A.ng; g += nth) {
      int gx, gy, gz;
      node_coords(g, A.nx, A.ny, gx, gy, gz);
      double acc = 0.0;
      const bool bnd = A.bc == SEM_DIRICHLET &&
                       (gx == 0 || gy == 0 || gz == 0 || gx == ex || gy == ey || gz == ez);
      if (!bnd) {
        for (int iz = max(gz - 1, 0); iz <= min(gz, ez - 1); ++iz)
          for (int iy = max(gy - 1, 0); iy <= min(gy, ey - 1); ++iy)
            for (int ix = max(gx - 1, 0); ix <= min(gx, ex - 1); ++ix) {
              const int64_t e = ix + (int64_t)ex * (iy + (int64_t)ey * iz);
              const int a = (gx - ix) + 2 * (gy - iy) + 4 * (gz - iz);
              const double *row = A.Ae + e * 64 + a * 8;
              const int64_t base = ix + (int64_t)A.nx * (iy + (int64_t)A.ny * iz);
#pragma unroll
              for (int b = 0; b < 8; ++b) {
                const int64_t nb = base + (b & 1) + (int64_t)A.nx * (((b >> 1) & 1) +
                                                                    (int64_t)A.ny * (b >> 2));
                acc = fma(row[b], A.p[nb], acc);
              }
            }
      }
      A.w[g] = acc;
      v[0] = fma(A.p[g], acc, v[0]);
    }
    coop_sum<1>(v, A.partA, grid);
    const double alpha = rho / v[0];
    // ---- x += alpha p, r -= alpha w, z = Dinv r;  rr, rz
    double u[2] = {0.0, 0.0};
    for (int64_t g = tid; g < A.ng; g += nth) {
      A.x[g] = fma(alpha, A.p[g], A.x[g]);
      double rg = fma(-alpha, A.w[g], A.r[g]);
      A.r[g] = rg;
      double zg = A.dinv[g] * rg;
      A.z[g] = zg;
      u[0] = fma(rg, rg, u[0]);
      u[1] = fma(rg, zg, u[1]);
    }
    coop_sum<2>(u, A.partB, grid);
    rr = u[0];
    if (!(rr > A.tol2 * bb) || it >= A.maxit || !(rr == rr)) break;
    const double beta = u[1] / rho;
    rho = u[1];
    for (int64_t g = tid; g < A.ng; g += nth) A.p[g] = fma(beta, A.p[g], A.z[g]);
    grid.sync();
  }
  grid.sync();
  // ---- solution back to E-layout
  const int64_t nloc = (int64_t)ex * ey * ez * 8;
  for (int64_t l = tid; l < nloc; l += nth) {
    const int64_t e = l >> 3;
    const int a = (int)(l & 7);
    const int64_t ix = e % ex, iy = (e / ex) % ey, iz = e / ((int64_t)ex * ey);
    const int64_t g = (ix + (a & 1)) + (int64_t)A.nx * ((iy + ((a >> 1) & 1)) +
                                                       (int64_t)A.ny * (iz + (a >> 2)));
    A.x_local[l] = A.x[g];
  }
  if (tid == 0) *A.iters = it;
}

// Element matrices of the N = 1 operator from its geometric factors:
// A_e[a][b] = sum_p sum_{d,f} (d_d phi_a)(p) G_df(p) (d_f phi_b)(p), where the
// reference derivative of basis (ai,aj,ak) along r at point (pi,pj,pk) is
// D[pi][ai] when pj = aj and pk = ak (and likewise along s and t).
__global__ void coarse_element_matrices(int64_t E, Basis bs, const double *__restrict__ G,
                                        double *__restrict__ Ae) {
  const double *D = bs.D;  // 2x2
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < E * 64;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = q >> 6;
    const int a = (int)((q >> 3) & 7), b = (int)(q & 7);
    const int ai = a & 1, aj = (a >> 1) & 1, ak = a >> 2;
    const int bi = b & 1, bj = (b >> 1) & 1, bk = b >> 2;
    double acc = 0.0;
    for (int p = 0; p < 8; ++p) {
      const int pi = p & 1, pj = (p >> 1) & 1, pk = p >> 2;
      double ga[3] = {(pj == aj && pk == ak) ? D[pi * 2 + ai] : 0.0,
                      (pi == ai && pk == ak) ? D[pj * 2 + aj] : 0.0,
                      (pi == ai && pj == aj) ? D[pk * 2 + ak] : 0.0};
      double gb[3] = {(pj == bj && pk == bk) ? D[pi * 2 + bi] : 0.0,
                      (pi == bi && pk == bk) ? D[pj * 2 + bj] : 0.0,
                      (pi == bi && pj == bj) ? D[pk * 2 + bk] : 0.0};
      const double *g = G + e * 48 + p;
      const double Grr = g[0], Grs = g[8], Grt = g[16], Gss = g[24], Gst = g[32], Gtt = g[40];
      acc += ga[0] * (Grr * gb[0] + Grs * gb[1] + Grt * gb[2]) +
             ga[1] * (Grs * gb[0] + Gss * gb[1] + Gst * gb[2]) +
             ga[2] * (Grt * gb[0] + Gst * gb[1] + Gtt * gb[2]);
    }
    Ae[q] = acc;
  }
}

// Unique-layout Jacobi inverse from the E-layout one (owner copy).
__global__ void coarse_unique_dinv(CoarseArgs A, const double *__restrict__ dinv_local,
                                   double *__restrict__ out) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < A.ng;
       g += (int64_t)gridDim.x * blockDim.x) {
    int gx, gy, gz;
    node_coords(g, A.nx, A.ny, gx, gy, gz);
    int ix = min(gx, A.ex - 1), iy = min(gy, A.ey - 1), iz = min(gz, A.ez - 1);
    int64_t e = ix + (int64_t)A.ex * (iy + (int64_t)A.ey * iz);
    int a = (gx - ix) + 2 * (gy - iy) + 4 * (gz - iz);
    out[g] = dinv_local[e * 8 + a];
  }
}

static CoarseArgs base_args(const CoarseSolver &C, const Level &L) {
  CoarseArgs A{};
  A.ex = L.t.ex; A.ey = L.t.ey; A.ez = L.t.ez;
  A.nx = L.t.ex + 1; A.ny = L.t.ey + 1;
  A.ng = L.t.ng;
  A.bc = L.t.bc;
  A.Ae = C.Ae.p;
  A.dinv = C.dinv.p;
  A.x = C.vec.p; A.r = A.x + A.ng; A.z = A.r + A.ng; A.p = A.z + A.ng; A.w = A.p + A.ng;
  A.partM = C.part.p;
  A.partI = A.partM + (size_t)C.grid * 4;
  A.partA = A.partI + (size_t)C.grid * 4;
  A.partB = A.partA + (size_t)C.grid * 4;
  A.iters = C.iters.p;
  return A;
}

void coarse_setup(CoarseSolver &C, const Level &L, cudaStream_t st) {
  SEM_REQUIRE(L.t.N == 1, "the persistent coarse solver needs N = 1");
  SEM_REQUIRE(L.G64.p != nullptr, "coarse level needs stored FP64 factors");
  const int64_t E = L.t.E, ng = L.t.ng;
  C.Ae.alloc((size_t)E * 64);
  C.dinv.alloc(ng);
  C.vec.alloc((size_t)5 * ng);
  C.iters.alloc(1);
  int dev = 0, sms = 0, per_sm = 0;
  SEM_CHECK_CUDA(cudaGetDevice(&dev));
  SEM_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  int coop = 0;
  SEM_CHECK_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  SEM_REQUIRE(coop != 0, "device does not support cooperative launches");
  SEM_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, coarse_cg_kernel,
                                                               kCoarseThreads, 0));
  SEM_REQUIRE(per_sm >= 1, "coarse kernel cannot be resident");
  const int64_t want = (ng + kCoarseThreads - 1) / kCoarseThreads;
  C.grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms * per_sm));
  C.part.alloc((size_t)C.grid * 16);
  {
    TraceScope ts("coarse_setup", 1, st);
    int blocks = (int)std::min<int64_t>((E * 64 + 255) / 256, 152 * 16);
    coarse_element_matrices<<<blocks, 256, 0, st>>>(E, L.basis, L.G64.p, C.Ae.p);
    SEM_CHECK_CUDA(cudaGetLastError());
    CoarseArgs A = base_args(C, L);
    coarse_unique_dinv<<<(int)std::min<int64_t>((ng + 255) / 256, 152 * 16), 256, 0, st>>>(
        A, L.dinv64.p, C.dinv.p);
    SEM_CHECK_CUDA(cudaGetLastError());
  }
}

void coarse_solve_persistent(CoarseSolver &C, const Level &L, const double *b_local,
                             double *x_local, double tol, int maxit, cudaStream_t st) {
  CoarseArgs A = base_args(C, L);
  A.b_local = b_local;
  A.x_local = x_local;
  A.tol2 = tol > 0 ? tol * tol : 0.0;
  A.maxit = maxit;
  void *args[] = {&A};
  TraceScope ts("coarse_cg", 1, st);
  SEM_CHECK_CUDA(cudaLaunchCooperativeKernel((const void *)coarse_cg_kernel, dim3(C.grid),
                                             dim3(kCoarseThreads), args, 0, st));
}

}  // namespace sem
