// schwarz.cuh -- data of the overlapping Schwarz preconditioner (internal).
#pragma once

#include "common.cuh"

namespace sem {

struct AsmData {
  int n = 0;                     // points per direction of an extended element (N + 3)
  DevBuf<double> S64, lam64;     // [E][3][n][n] eigenvectors (point, mode), [E][3][n]
  DevBuf<float> S32, lam32;      // FP32 copies for FP32 smoothing
  DevBuf<double> ext64;          // [E][6][Np^2] face layers of the local solutions
  DevBuf<float> ext32;
  DevBuf<double> mr64;           // M r of the Chebyshev recurrence
  DevBuf<float> mr32;
  int tc = 0;                     // FP32 local solves on the tensor cores: 1 with the
                                 // head + remainder split, 2 in plain TF32
};

// Eigendecompositions of every element's 1D pencils (FP64; FP32 copies if
// want_f32) and the layer buffers.
void asm_setup(AsmData &A, const Level &L, bool want_f32, cudaStream_t st);
// The FP32 local solves on the tensor cores (schwarz_tc.cu): own points of
// every extended element's solution to z, its face layers to ext.
void launch_asm_solve_tc(const AsmData &A, const Level &L, const float *r, float *z, float *ext,
                         bool split, cudaStream_t st);
// z = mask sum_e R_e^T K_e^{-1} R_e r (r continuous; z assembled).
template <typename T>
void launch_asm(const AsmData &A, const Level &L, const T *r, T *z, cudaStream_t st);

}  // namespace sem
