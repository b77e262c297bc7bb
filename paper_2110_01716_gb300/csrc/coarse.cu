// coarse.cu -- coarsest p-multigrid level (N = 1): FP64 Jacobi-PCG in one
// persistent cooperative kernel.
//
// The paper solves its N = 1 coarse grid with algebraic multigrid on the host
// (Sec. 4, Table 1 discussion).  On one GPU the coarse problem is small
// (about one unique node per element) and latency bound, so the whole CG
// iteration runs inside one launch:
//  * vectors live in unique-node layout (no duplicated copies);
//  * the operator is the assembled 27-point stencil of the trilinear N = 1
//    discretisation, stored structure-of-arrays [27][nodes] in FP64 and built
//    once from the 8x8 element matrices in a fixed order (no atomics);
//  * the Krylov method is Jacobi-preconditioned CG in the Chronopoulos-Gear
//    arrangement (one fused reduction of (r,z), (Az,z), (r,r) per iteration,
//    s = A p carried by recurrence), so an iteration needs two grid barriers;
//  * reductions are two-stage: per-CTA partials, then every CTA adds all
//    partials in the same order, so all CTAs hold bit-identical scalars and
//    take the same stopping decision.
#include <cooperative_groups.h>

#include <algorithm>

#include "coarse.cuh"
#include "kernels.cuh"
#include "trace.cuh"

namespace cg = cooperative_groups;

namespace sem {

// CTA size and the number of CTAs per SM of the persistent coarse kernel
// (grid barriers cost more with more CTAs; more CTAs hide more latency).
#ifndef SEM_COARSE_THREADS
#define SEM_COARSE_THREADS 256
#endif
#ifndef SEM_COARSE_CTAS_PER_SM
#define SEM_COARSE_CTAS_PER_SM 1
#endif
constexpr int kCoarseThreads = SEM_COARSE_THREADS;

// All index arithmetic is 32-bit with multiplicative division: 64-bit
// integer division is emulated and would compete for the scarce FP64 pipe.
struct CoarseArgs {
  int ex, ey, ez;
  int nx, ny, nz;  // lattice points per direction
  FastDiv div_nx, div_nxy, div_ex, div_ey;
  int64_t ng;
  int bc;
  const double *S;     // [27][ng] assembled stencil
  const double *dinv;  // [ng]
  const double *b_local;
  double *x_local;
  double *x, *r, *z, *p, *s, *w;
  // Three partial-sum regions of grid*4 doubles (mean, start, iteration);
  // every reduction write is separated by a grid barrier from the reads of
  // the previous reduction in the same region.
  double *partM, *partI, *partK;
  int *iters;
  double tol2;
  int maxit;
};

__device__ __forceinline__ void node_coords(const CoarseArgs &A, int64_t g, int &gx, int &gy,
                                            int &gz) {
  const uint32_t u = (uint32_t)g;
  gz = (int)A.div_nxy.div(u);
  const uint32_t rem = u - (uint32_t)gz * (uint32_t)(A.nx * A.ny);
  gy = (int)A.div_nx.div(rem);
  gx = (int)(rem - (uint32_t)gy * (uint32_t)A.nx);
}

// Block sum of NS values, then grid-wide sum identical in every CTA.  FP64
// additions are scarce on this part, so only warp 0 of each CTA reduces the
// per-warp partials and, after the grid barrier, the per-CTA partials (in
// CTA order, lane-strided, then a fixed shuffle tree); the result is
// broadcast through shared memory.
template <int NS>
__device__ void coop_sum(double (&v)[NS], double *part, cg::grid_group &grid) {
  __shared__ double sh[NS][kCoarseThreads / 32];
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
      double x = lane < kCoarseThreads / 32 ? sh[s][lane] : 0.0;
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

// (A v)_g from the 27-point stencil; Dirichlet boundary rows are zero.
__device__ __forceinline__ double stencil_apply(const CoarseArgs &A, int64_t g,
                                                const double *__restrict__ v) {
  int gx, gy, gz;
  node_coords(A, g, gx, gy, gz);
  if (A.bc == SEM_DIRICHLET &&
      (gx == 0 || gy == 0 || gz == 0 || gx == A.nx - 1 || gy == A.ny - 1 || gz == A.nz - 1))
    return 0.0;
  // neighbour tests first, then one guarded load pair per neighbour, so that
  // all the loads are in flight together
  const bool in_x[3] = {gx > 0, true, gx < A.nx - 1};
  const bool in_y[3] = {gy > 0, true, gy < A.ny - 1};
  const bool in_z[3] = {gz > 0, true, gz < A.nz - 1};
  double sv[27], vv[27];
#pragma unroll
  for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        const int d = (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1);
        const bool ok = in_x[dx + 1] && in_y[dy + 1] && in_z[dz + 1];
        sv[d] = ok ? A.S[(int64_t)d * A.ng + g] : 0.0;
        vv[d] = ok ? v[g + dx + (int64_t)A.nx * (dy + (int64_t)A.ny * dz)] : 0.0;
      }
  double acc = 0.0;
#pragma unroll
  for (int d = 0; d < 27; ++d) acc = fma(sv[d], vv[d], acc);
  return acc;
}

__global__ void __launch_bounds__(kCoarseThreads) coarse_cg_kernel(CoarseArgs A) {
  cg::grid_group grid = cg::this_grid();
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  const int ex = A.ex, ey = A.ey;
  // ---- right-hand side to unique layout (owner copy), x = 0
  double v1[1] = {0.0};
  for (int64_t g = tid; g < A.ng; g += nth) {
    int gx, gy, gz;
    node_coords(A, g, gx, gy, gz);
    int ix = min(gx, ex - 1), iy = min(gy, ey - 1), iz = min(gz, A.ez - 1);
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
  for (int64_t g = tid; g < A.ng; g += nth) A.z[g] = A.dinv[g] * A.r[g];
  grid.sync();
  // ---- w = A z;  rho = (r,z), mu = (w,z), rr = (r,r)
  double v3[3] = {0.0, 0.0, 0.0};
  for (int64_t g = tid; g < A.ng; g += nth) {
    const double wg = stencil_apply(A, g, A.z);
    A.w[g] = wg;
    const double rg = A.r[g], zg = A.z[g];
    v3[0] = fma(rg, zg, v3[0]);
    v3[1] = fma(wg, zg, v3[1]);
    v3[2] = fma(rg, rg, v3[2]);
  }
  coop_sum<3>(v3, A.partI, grid);
  const double bb = v3[2];
  double rho = v3[0], alpha = v3[0] / v3[1];
  int it = 0;
  if (v3[2] > A.tol2 * bb && A.maxit > 0 && rho != 0.0) {
    for (int64_t g = tid; g < A.ng; g += nth) {
      A.p[g] = A.z[g];
      A.s[g] = A.w[g];
    }
    for (;;) {
      ++it;
      // x += alpha p, r -= alpha s, z = Dinv r   (own nodes only)
      for (int64_t g = tid; g < A.ng; g += nth) {
        A.x[g] = fma(alpha, A.p[g], A.x[g]);
        const double rg = fma(-alpha, A.s[g], A.r[g]);
        A.r[g] = rg;
        A.z[g] = A.dinv[g] * rg;
      }
      grid.sync();
      double v[3] = {0.0, 0.0, 0.0};
      for (int64_t g = tid; g < A.ng; g += nth) {
        const double wg = stencil_apply(A, g, A.z);
        A.w[g] = wg;
        const double rg = A.r[g], zg = A.z[g];
        v[0] = fma(rg, zg, v[0]);
        v[1] = fma(wg, zg, v[1]);
        v[2] = fma(rg, rg, v[2]);
      }
      coop_sum<3>(v, A.partK, grid);
      const double rr = v[2];
      if (!(rr > A.tol2 * bb) || it >= A.maxit || !(rr == rr) || v[0] == 0.0) break;
      const double beta = v[0] / rho;
      alpha = v[0] / (v[1] - beta * v[0] / alpha);
      rho = v[0];
      for (int64_t g = tid; g < A.ng; g += nth) {
        A.p[g] = fma(beta, A.p[g], A.z[g]);
        A.s[g] = fma(beta, A.s[g], A.w[g]);
      }
    }
  }
  grid.sync();
  // ---- solution back to E-layout
  const int64_t nloc = (int64_t)ex * ey * A.ez * 8;
  for (int64_t l = tid; l < nloc; l += nth) {
    const uint32_t e = (uint32_t)(l >> 3);
    const int a = (int)(l & 7);
    const uint32_t yz = A.div_ex.div(e);
    const int64_t ix = e - yz * (uint32_t)ex;
    const int64_t iz = A.div_ey.div(yz);
    const int64_t iy = yz - (uint32_t)iz * (uint32_t)ey;
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

// Assembled stencil S[d][g] = sum over elements e containing g of
// A_e[a(g)][b] for the node b of e at offset d from g; elements in a fixed
// order, so the assembly is deterministic.
__global__ void coarse_stencil_assemble(CoarseArgs A, const double *__restrict__ Ae,
                                        double *__restrict__ S) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < A.ng;
       g += (int64_t)gridDim.x * blockDim.x) {
    int gx, gy, gz;
    node_coords(A, g, gx, gy, gz);
    for (int d = 0; d < 27; ++d) S[(int64_t)d * A.ng + g] = 0.0;
    for (int iz = max(gz - 1, 0); iz <= min(gz, A.ez - 1); ++iz)
      for (int iy = max(gy - 1, 0); iy <= min(gy, A.ey - 1); ++iy)
        for (int ix = max(gx - 1, 0); ix <= min(gx, A.ex - 1); ++ix) {
          const int64_t e = ix + (int64_t)A.ex * (iy + (int64_t)A.ey * iz);
          const int a = (gx - ix) + 2 * (gy - iy) + 4 * (gz - iz);
          for (int b = 0; b < 8; ++b) {
            const int dx = ix + (b & 1) - gx, dy = iy + ((b >> 1) & 1) - gy, dz = iz + (b >> 2) - gz;
            const int d = (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1);
            S[(int64_t)d * A.ng + g] += Ae[e * 64 + a * 8 + b];
          }
        }
  }
}

// Unique-layout Jacobi inverse from the E-layout one (owner copy).
__global__ void coarse_unique_dinv(CoarseArgs A, const double *__restrict__ dinv_local,
                                   double *__restrict__ out) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < A.ng;
       g += (int64_t)gridDim.x * blockDim.x) {
    int gx, gy, gz;
    node_coords(A, g, gx, gy, gz);
    int ix = min(gx, A.ex - 1), iy = min(gy, A.ey - 1), iz = min(gz, A.ez - 1);
    int64_t e = ix + (int64_t)A.ex * (iy + (int64_t)A.ey * iz);
    int a = (gx - ix) + 2 * (gy - iy) + 4 * (gz - iz);
    out[g] = dinv_local[e * 8 + a];
  }
}

static CoarseArgs base_args(const CoarseSolver &C, const Level &L) {
  CoarseArgs A{};
  A.ex = L.t.ex; A.ey = L.t.ey; A.ez = L.t.ez;
  A.nx = L.t.ex + 1; A.ny = L.t.ey + 1; A.nz = L.t.ez + 1;
  A.div_nx = FastDiv((uint32_t)A.nx);
  A.div_nxy = FastDiv((uint32_t)(A.nx * A.ny));
  A.div_ex = FastDiv((uint32_t)A.ex);
  A.div_ey = FastDiv((uint32_t)A.ey);
  A.ng = L.t.ng;
  A.bc = L.t.bc;
  A.S = C.S.p;
  A.dinv = C.dinv.p;
  const size_t vs = C.vec_stride;
  A.x = C.vec.p; A.r = A.x + vs; A.z = A.r + vs; A.p = A.z + vs; A.s = A.p + vs; A.w = A.s + vs;
  const size_t ps = (size_t)((C.grid * 4 + 31) / 32 * 32);
  A.partM = C.part.p;
  A.partI = A.partM + ps;
  A.partK = A.partI + ps;
  A.iters = C.iters.p;
  return A;
}

void coarse_setup(CoarseSolver &C, const Level &L, cudaStream_t st, int max_ctas) {
  SEM_REQUIRE(L.t.N == 1, "the persistent coarse solver needs N = 1");
  DevBuf<double> Gtmp;
  const double *G = L.G64.p;
  if (!G) {
    level_fp64_factors(L, Gtmp, st);
    G = Gtmp.p;
  }
  const int64_t E = L.t.E, ng = L.t.ng;
  DevBuf<double> Ae;
  Ae.alloc((size_t)E * 64);
  C.S.alloc((size_t)27 * ng);
  C.dinv.alloc(ng);
  // vectors start on 256-byte boundaries (see coarse_mg.cu)
  C.vec_stride = (size_t)((ng + 31) / 32 * 32);
  C.vec.alloc(6 * C.vec_stride);
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
  per_sm = std::min(per_sm, SEM_COARSE_CTAS_PER_SM);
  C.grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms * per_sm));
  if (max_ctas > 0 && C.grid > max_ctas) C.grid = max_ctas;
  C.part.alloc(3 * (size_t)((C.grid * 4 + 31) / 32 * 32));
  {
    TraceScope ts("coarse_setup", 1, st, 3);
    int blocks = (int)std::min<int64_t>((E * 64 + 255) / 256, 152 * 16);
    coarse_element_matrices<<<blocks, 256, 0, st>>>(E, L.basis, G, Ae.p);
    SEM_CHECK_CUDA(cudaGetLastError());
    CoarseArgs A = base_args(C, L);
    coarse_stencil_assemble<<<(int)std::min<int64_t>((ng + 255) / 256, 152 * 16), 256, 0, st>>>(
        A, Ae.p, C.S.p);
    SEM_CHECK_CUDA(cudaGetLastError());
    coarse_unique_dinv<<<(int)std::min<int64_t>((ng + 255) / 256, 152 * 16), 256, 0, st>>>(
        A, L.dinv64.p, C.dinv.p);
    SEM_CHECK_CUDA(cudaGetLastError());
    SEM_CHECK_CUDA(cudaStreamSynchronize(st));  // before the element matrices are freed
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
