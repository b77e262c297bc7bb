// coarse.cuh -- persistent FP64 Jacobi-PCG of the N = 1 coarsest level.
#pragma once

#include "common.cuh"

namespace sem {

struct CoarseSolver {
  DevBuf<double> S;     // [27][ng] assembled stencil
  DevBuf<double> dinv;  // [ng] Jacobi inverse, unique layout (0 on Dirichlet nodes)
  DevBuf<double> vec;   // x, r, z, p, s, w in unique layout
  DevBuf<double> part;  // grid reduction partials
  DevBuf<int> iters;    // iterations of the last solve
  int grid = 0;
};

void coarse_setup(CoarseSolver &C, const Level &L, cudaStream_t st);
void coarse_solve_persistent(CoarseSolver &C, const Level &L, const double *b_local,
                             double *x_local, double tol, int maxit, cudaStream_t st);

}  // namespace sem
