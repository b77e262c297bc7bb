// krylov.cu -- vector kernels of the flexible GMRES outer solver (Sec. 3:
// GMRES as the alternative to FlexCG; Sec. 5: classical Gram-Schmidt, so one
// reduction gives every orthogonalisation coefficient of a step).
//
// The Krylov basis V and the preconditioned vectors Z are E-layout FP64
// vectors stored back to back with a fixed stride.  Inner products are the
// unique-dof product sum_l u_l v_l / mult_l, reduced deterministically (fixed
// grid, partials summed in order).
#include "common.cuh"
#include "kernels.cuh"
#include "reduce.cuh"
#include "trace.cuh"

namespace sem {

// h_i = <w, V_i> for i < c, in one pass over w.
template <int NS>
__global__ void __launch_bounds__(kVecThreads)
    multi_dot_kernel(Topo t, const double *__restrict__ w, const double *__restrict__ V,
                     size_t stride, int c, double *partials, unsigned int *counter,
                     OutPtrs<NS> out) {
  double acc[NS];
#pragma unroll
  for (int i = 0; i < NS; ++i) acc[i] = 0.0;
  for (uint32_t l = blockIdx.x * blockDim.x + threadIdx.x; l < (uint32_t)t.nl;
       l += gridDim.x * blockDim.x) {
    const PointInfo q = point_info(l, t);
    const double ws = scale_pow2_down(w[l], q.log2_mult);
#pragma unroll
    for (int i = 0; i < NS; ++i)
      if (i < c) acc[i] = fma(ws, V[(size_t)i * stride + l], acc[i]);
  }
  grid_reduce<NS>(acc, partials, counter, out.p);
}

// v = w - sum_{i<c} h_i V_i and nrm2 = <v, v>.
__global__ void __launch_bounds__(kVecThreads)
    orth_update_kernel(Topo t, const double *__restrict__ w, const double *__restrict__ V,
                       size_t stride, int c, const double *__restrict__ h,
                       double *__restrict__ v, double *partials, unsigned int *counter,
                       OutPtrs<1> out) {
  double acc[1] = {0.0};
  for (uint32_t l = blockIdx.x * blockDim.x + threadIdx.x; l < (uint32_t)t.nl;
       l += gridDim.x * blockDim.x) {
    const PointInfo q = point_info(l, t);
    double s = w[l];
    for (int i = 0; i < c; ++i) s = fma(-__ldg(h + i), V[(size_t)i * stride + l], s);
    v[l] = s;
    acc[0] = fma(scale_pow2_down(s, q.log2_mult), s, acc[0]);
  }
  grid_reduce<1>(acc, partials, counter, out.p);
}

__global__ void scale_kernel(int64_t n, double a, double *__restrict__ v) {
  for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < n;
       l += (int64_t)gridDim.x * blockDim.x)
    v[l] *= a;
}

__global__ void mul_kernel(int64_t n, const double *__restrict__ a, const double *__restrict__ b,
                           double *__restrict__ out) {
  for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < n;
       l += (int64_t)gridDim.x * blockDim.x)
    out[l] = a[l] * b[l];
}

struct Coefs {
  double y[kMaxKrylov];
};

// x += sum_{i<c} y_i Z_i
__global__ void combine_kernel(int64_t n, const double *__restrict__ Z, size_t stride, int c,
                               Coefs y, double *__restrict__ x) {
  for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < n;
       l += (int64_t)gridDim.x * blockDim.x) {
    double s = x[l];
    for (int i = 0; i < c; ++i) s = fma(y.y[i], Z[(size_t)i * stride + l], s);
    x[l] = s;
  }
}

template <int NS>
static void multi_dot_ns(const Topo &t, Reducer &R, const double *w, const double *V,
                         size_t stride, int c, double *h, cudaStream_t st) {
  OutPtrs<NS> o;
  for (int i = 0; i < NS; ++i) o.p[i] = h + i;  // h has room for kMaxKrylov + 1 values
  multi_dot_kernel<NS><<<vec_grid(t.nl), kVecThreads, 0, st>>>(t, w, V, stride, c, R.partials.p,
                                                               R.counter.p, o);
}

void launch_multi_dot(const Topo &t, Reducer &R, const double *w, const double *V, size_t stride,
                      int c, double *h, cudaStream_t st) {
  SEM_REQUIRE(c >= 1 && c <= kMaxKrylov + 1, "multi_dot: %d vectors", c);
  TraceScope ts("multi_dot", t.N, st);
  if (c <= 4) multi_dot_ns<4>(t, R, w, V, stride, c, h, st);
  else if (c <= 8) multi_dot_ns<8>(t, R, w, V, stride, c, h, st);
  else if (c <= 16) multi_dot_ns<16>(t, R, w, V, stride, c, h, st);
  else multi_dot_ns<kMaxKrylov + 1>(t, R, w, V, stride, c, h, st);
  SEM_CHECK_CUDA(cudaGetLastError());
}

void launch_orth_update(const Topo &t, Reducer &R, const double *w, const double *V,
                        size_t stride, int c, const double *h, double *v, double *nrm2,
                        cudaStream_t st) {
  OutPtrs<1> o{{nrm2}};
  TraceScope ts("orth_update", t.N, st);
  orth_update_kernel<<<vec_grid(t.nl), kVecThreads, 0, st>>>(t, w, V, stride, c, h, v,
                                                             R.partials.p, R.counter.p, o);
  SEM_CHECK_CUDA(cudaGetLastError());
}

void launch_scale(int64_t n, double a, double *v, cudaStream_t st) {
  TraceScope ts("scale", 0, st);
  scale_kernel<<<vec_grid(n), kVecThreads, 0, st>>>(n, a, v);
  SEM_CHECK_CUDA(cudaGetLastError());
}

void launch_mul(int64_t n, const double *a, const double *b, double *out, cudaStream_t st) {
  TraceScope ts("jacobi", 0, st);
  mul_kernel<<<vec_grid(n), kVecThreads, 0, st>>>(n, a, b, out);
  SEM_CHECK_CUDA(cudaGetLastError());
}

void launch_combine(int64_t n, const double *Z, size_t stride, int c, const double *y, double *x,
                    cudaStream_t st) {
  SEM_REQUIRE(c >= 0 && c <= kMaxKrylov, "combine: %d vectors", c);
  if (c == 0) return;
  Coefs cf;
  for (int i = 0; i < kMaxKrylov; ++i) cf.y[i] = i < c ? y[i] : 0.0;
  TraceScope ts("combine", 0, st);
  combine_kernel<<<vec_grid(n), kVecThreads, 0, st>>>(n, Z, stride, c, cf, x);
  SEM_CHECK_CUDA(cudaGetLastError());
}

}  // namespace sem
