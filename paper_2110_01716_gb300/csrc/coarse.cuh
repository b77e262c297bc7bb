// coarse.cuh -- the N = 1 coarsest level: persistent FP64 Jacobi-PCG, and FP64 CG
// preconditioned by a geometric lattice multigrid V-cycle in FP32 (coarse_mg.cu).
#pragma once

#include <memory>

#include "common.cuh"

namespace sem {

constexpr int kMgMaxLevels = 8;

// One level of the coarse-lattice multigrid, in the arithmetic T.
template <typename T>
struct MgLevelT {
  int nx, ny, nz, n;
  FastDiv div_nx, div_nxy;
  const T *S;     // [27][n] stencil (Dirichlet rows/unknowns eliminated via dinv/mask)
  const T *dinv;  // [n] 0 on Dirichlet nodes
  const unsigned char *keep;  // [n] 1 for unknowns, 0 for Dirichlet nodes
  T *x, *b, *r, *da, *db;
  T inv_theta, c1, c2;  // Chebyshev degree-2 coefficients
  // 1D transfer tables (this level -> next coarser): prolongation rows of the
  // fine indices (2 entries, index -1 = none), restriction rows of the coarse
  // indices (3 entries).
  const int *pi[3];
  const T *pw[3];
  const int *ri[3];
  const T *rw[3];
};

struct MgArgs {
  int nlev;
  int small_from;  // first level run by one CTA (nlev - 1: the bottom only)
  MgLevelT<double> L0;              // level 0 in FP64: the flexible CG's operator
  MgLevelT<float> V[kMgMaxLevels];  // the V-cycle (the preconditioner) in FP32
  const float *bottom_inv;
  int nbottom;
  int ex, ey, ez, bc;
  FastDiv div_ex, div_ey;
  const double *b_local;
  double *x_local;
  double *x, *r, *z, *p, *w;  // CG vectors on level 0
  double *partM, *partI, *partA, *partK;
  int *iters;
  double tol2;
  int maxit;
};

// Multigrid hierarchy of the coarse lattice (coarse_mg.cu).
struct CoarseMg {
  MgArgs args{};
  DevBuf<float> fbuf;
  DevBuf<int> ibuf;
  DevBuf<unsigned char> kbuf;
  DevBuf<double> part;
  int grid = 0, levels = 0;
};

struct CoarseSolver {
  DevBuf<double> S;     // [27][ng] assembled stencil
  DevBuf<double> dinv;  // [ng] Jacobi inverse, unique layout (0 on Dirichlet nodes)
  DevBuf<double> vec;   // x, r, z, p, s, w in unique layout
  size_t vec_stride = 0; // doubles between consecutive vectors (multiple of 32)
  DevBuf<double> part;  // grid reduction partials
  DevBuf<int> iters;    // iterations of the last solve
  int grid = 0;
  std::unique_ptr<CoarseMg> mg;  // multigrid-preconditioned mode
};

// max_ctas > 0 caps the persistent kernel's grid (sem_pmg_desc.coarse_ctas).
void coarse_setup(CoarseSolver &C, const Level &L, cudaStream_t st, int max_ctas = 0);
void coarse_solve_persistent(CoarseSolver &C, const Level &L, const double *b_local,
                             double *x_local, double tol, int maxit, cudaStream_t st);
void coarse_mg_setup(CoarseSolver &C, const Level &L, cudaStream_t st, int max_ctas = 0);
void coarse_mg_solve(CoarseSolver &C, const double *b_local, double *x_local, double tol,
                     int maxit, cudaStream_t st);

}  // namespace sem
