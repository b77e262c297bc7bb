// kernels.cuh -- launchers of the vector, smoother and transfer kernels.
#pragma once

#include "common.cuh"

namespace sem {

constexpr int kVecThreads = 256;
constexpr int kVecMaxBlocks = 152 * 8;  // grid of every reduction (fixed per size)

int vec_grid(int64_t n);

void launch_dot(const Topo &t, Reducer &R, const double *u, const double *v, double *out,
                cudaStream_t st);
void launch_dot(const Topo &t, Reducer &R, const float *u, const double *v, double *out,
                cudaStream_t st);
void launch_dot_skip(const Topo &t, Reducer &R, const double *u, const double *v, double *out,
                     const int *skip, cudaStream_t st);
void launch_dot_local(const Topo &t, Reducer &R, const double *u, const double *v, double *out,
                      const int *skip, cudaStream_t st);
void launch_sum(const Topo &t, Reducer &R, const double *u, double *out, cudaStream_t st);
void launch_remove_mean(const Topo &t, Reducer &R, double *u, double *scratch, cudaStream_t st);
void launch_cg_start(const Topo &t, Reducer &R, const double *b, const double *w,
                     const double *dinv, double *r, double *z, double *p, double *bb, double *rr,
                     double *rz, cudaStream_t st);
void launch_cg_update(const Topo &t, Reducer &R, const double *rho, const double *pw,
                      const double *p, const double *w, const double *dinv, double *x, double *r,
                      double *z, double *rr, double *rz, const int *skip, cudaStream_t st,
                      float *rc32 = nullptr, double *rc64 = nullptr);
template <typename Tz>
void launch_cg_direction(int64_t n, const double *num, const double *den, double sign,
                         const Tz *z, double *p, const int *skip, cudaStream_t st);
template <typename Tz>
void launch_flex_dots(const Topo &t, Reducer &R, const Tz *z, const double *r, const double *w,
                      double *zr, double *zw, cudaStream_t st);
void launch_stop_test(const double *rr, const double *bb, double tol2, int it, int maxit,
                      int *skip, int *iters, cudaStream_t st);
// Reduction target of the FP64 pair operator's fused form: pw = <u, A_L u>.
struct PairFuse {
  double *partials = nullptr;
  unsigned int *counter = nullptr;
  double *pw = nullptr;
};

// Hint: bring [p, p + bytes) into L2 (bulk prefetch; the range is shrunk to
// whole 16-byte units inside it, so nothing outside it is touched).
__device__ __forceinline__ void prefetch_l2(const void *p, int64_t bytes) {
  uintptr_t a = reinterpret_cast<uintptr_t>(p);
  const uintptr_t b = (a + (uintptr_t)bytes) & ~(uintptr_t)15;
  a = (a + 15) & ~(uintptr_t)15;
  while (a + 16 <= b) {
    const uint32_t n = (uint32_t)((b - a) < (1u << 20) ? (b - a) : (1u << 20));
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"(n) : "memory");
    a += n;
  }
}

// Exact widening of a float to double through its bit pattern (zero and
// subnormal floats give 0, Inf/NaN stay Inf/NaN).
__device__ __forceinline__ double widen_f32(float f) {
  const unsigned int u = __float_as_uint(f);
  const unsigned int e = (u >> 23) & 0xFFu;
  if (e == 0) return 0.0;
  const unsigned long long s = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned long long ex = (unsigned long long)(e == 255 ? 2047u : e + 896u) << 52;
  const unsigned long long m = (unsigned long long)(u & 0x7FFFFFu) << 29;
  return __longlong_as_double((long long)(s | ex | m));
}

// The FP64 pair operator w = A_L u (local, unassembled) with <u, A_L u>
// written to *pw (ax_pair_fused.cu).
void launch_ax_pair_dot(const Level &L, const double *u, double *w, double *pw, Reducer &R,
                        cudaStream_t st);

void launch_graph_stop(const double *rr, double *g, cudaGraphConditionalHandle h,
                       cudaStream_t st);
void launch_graph_arm(double *g, double tol2, int maxit, int done, cudaStream_t st);
void launch_graph_arm_full(const double *bb, const double *rr, double *g, double tol, int maxit,
                           cudaGraphConditionalHandle h, cudaStream_t st);
template <typename A, typename B>
void launch_convert(int64_t n, const A *a, B *b, cudaStream_t st);

// b = mask gs(B f), f = 3 pi^2 sin(pi x) sin(pi y) sin(pi z) on the level's
// points (tmp: 4 n_local doubles of scratch) -- serve.cu.
void build_manufactured_rhs(const Level &L, double *b, double *tmp, cudaStream_t st);

// Flexible GMRES (krylov.cu).  Basis vectors i < c at V + i * stride.
constexpr int kMaxKrylov = 32;  // restart length limit
void launch_multi_dot(const Topo &t, Reducer &R, const double *w, const double *V, size_t stride,
                      int c, double *h, cudaStream_t st);
void launch_orth_update(const Topo &t, Reducer &R, const double *w, const double *V,
                        size_t stride, int c, const double *h, double *v, double *nrm2,
                        cudaStream_t st);
void launch_scale(int64_t n, double a, double *v, cudaStream_t st);
void launch_mul(int64_t n, const double *a, const double *b, double *out, cudaStream_t st);
void launch_combine(int64_t n, const double *Z, size_t stride, int c, const double *y, double *x,
                    cudaStream_t st);

// Assembled operator on a level: w = mask * gs(A_L u).
// FP32 on stored factors takes the fused operator (x-face sums in the operator
// kernel, plane passes for y and z).
template <typename T>
inline void apply_assembled(const Level &L, const T *u, T *w, cudaStream_t st) {
  if constexpr (sizeof(T) == 4) {
    if (L.geom == SEM_GEOM_STORED) {
      launch_ax32(L, SEM_F32, u, w, true, st);
      return;
    }
  }
  launch_ax<T>(L, u, w, st);
#ifndef SEM_GS_NODES
  // the copies of shared nodes summed by x, y and z face passes (whole
  // sectors in y and z), the Dirichlet mask with them
  launch_planes_assemble<T>(L, w, st);
#else
  launch_gs<T>(L, w, st);
  launch_mask<T>(L, w, st);
#endif
}

}  // namespace sem
