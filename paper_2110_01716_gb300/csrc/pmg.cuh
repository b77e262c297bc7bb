// pmg.cuh -- p-multigrid hierarchy (internal).
#pragma once

#include <memory>
#include <vector>

#include "coarse.cuh"
#include "common.cuh"
#include "schwarz.cuh"

namespace sem {

struct PmgLevel {
  Level *L = nullptr;          // level 0 is the mesh's own fine level
  std::unique_ptr<Level> own;  // coarser levels are owned here
  int dtype = SEM_F64;         // arithmetic of the level's smoother (F64 or F32)
  int g16 = 0;                 // SEM_F16 / SEM_BF16: FP32 smoother on 16-bit factors
  double lam_lo = 0.0, lam_hi = 0.0;
  DevBuf<double> v64[5];       // b, x, r, d, w in FP64 ...
  DevBuf<float> v32[5];        // ... or FP32
  std::vector<double> J;       // (N_l+1) x (N_{l+1}+1) interpolation to this level
  std::unique_ptr<AsmData> asmd;  // Schwarz smoother data (SEM_SMOOTH_ASM)
};

void pmg_build(sem_pmg *P, sem_mesh *mesh, const sem_pmg_desc &d, cudaStream_t st);
void pmg_vcycle(sem_pmg *P, const double *r, double *z, cudaStream_t st);

// The fine level's V-cycle buffers in the level's arithmetic: the input
// (residual) and the output (correction); one of each pair is set.
struct VcycleIO {
  float *in32 = nullptr;
  double *in64 = nullptr;
  const float *out32 = nullptr;
  const double *out64 = nullptr;
};
VcycleIO pmg_io(sem_pmg *P);
// One V-cycle from the input buffer to the output buffer.
void pmg_vcycle_core(sem_pmg *P, cudaStream_t st);
// Device bytes held by the hierarchy (not the mesh's).
size_t pmg_device_bytes(const sem_pmg *P);
// The coarsest-level solve alone (b, x: E-layout vectors of that level).
void pmg_coarse_solve(sem_pmg *P, const double *b, double *x, cudaStream_t st);

}  // namespace sem

struct sem_pmg {
  sem_mesh *mesh = nullptr;
  sem_pmg_desc desc{};
  std::vector<std::unique_ptr<sem::PmgLevel>> levp;
  sem::Reducer red;
  sem::DevBuf<double> scal;
  sem::DevBuf<int> flags;
  sem::DevBuf<double> cz, cp, cw, z64;
  sem::CoarseSolver coarse;   // persistent solver when the coarsest order is 1
  bool persistent_coarse = false;
  uint64_t serial = 0;        // distinct for every hierarchy created
};
