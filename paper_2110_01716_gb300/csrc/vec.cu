// vec.cu -- fused vector updates and deterministic reductions of the Krylov
// solvers (Sec. 3: Jacobi-PCG for the Stokes substep, flexible CG for the
// pMG-preconditioned pressure solve).
//
// Inner products are over unique nodes: sum_l u_l v_l / mult_l, with the
// multiplicity computed from the point's position (no stored weights).
// Reductions are deterministic: each CTA of a fixed-size grid reduces its
// share in a fixed order (warp shuffles, then warps in order), writes one
// partial per sum, and the last CTA to finish (ticket counter) adds the
// partials in CTA order.  The same n gives the same bits on every run.
// Scalars live in device memory, so an iteration needs no host round trip.
#include "common.cuh"
#include "kernels.cuh"
#include "reduce.cuh"
#include "trace.cuh"

namespace sem {

void Reducer::init(int blocks, int max_sums) {
  nblocks = blocks;
  capacity = (size_t)blocks * max_sums;
  partials.alloc(capacity);
  counter.alloc(1);
  SEM_CHECK_CUDA(cudaMemset(counter.p, 0, sizeof(unsigned int)));
  // the memset runs on the legacy stream, which kernels on non-blocking
  // streams (server workers, batch captures) do not wait for: finish it here
  SEM_CHECK_CUDA(cudaStreamSynchronize(0));
}

int vec_grid(int64_t n) {
  int64_t b = (n + kVecThreads - 1) / kVecThreads;
  return (int)(b < 1 ? 1 : (b > kVecMaxBlocks ? kVecMaxBlocks : b));
}

// ------------------------------------------------------------------ dots
__device__ __forceinline__ double as_f64(double v) { return v; }
__device__ __forceinline__ double as_f64(float v) { return widen_f32(v); }

// out = sum u v / mult; u in FP64 or FP32 (widened exactly)
template <typename Tu>
__global__ void __launch_bounds__(kVecThreads)
    dot_kernel(Topo t, const Tu *__restrict__ u, const double *__restrict__ v,
               double *partials, unsigned int *counter, OutPtrs<1> out) {
  double acc[1] = {0.0};
  for (uint32_t l = blockIdx.x * blockDim.x + threadIdx.x; l < (uint32_t)t.nl;
       l += gridDim.x * blockDim.x) {
    PointInfo q = point_info(l, t);
    acc[0] = fma(scale_pow2_down(as_f64(u[l]), q.log2_mult), v[l], acc[0]);
  }
  grid_reduce<1>(acc, partials, counter, out.p);
}

template <typename Tu>
static void dot_any(const Topo &t, Reducer &R, const Tu *u, const double *v, double *out,
                    cudaStream_t st) {
  OutPtrs<1> o{{out}};
  TraceScope ts("dot", t.N, st);
  dot_kernel<Tu><<<vec_grid(t.nl), kVecThreads, 0, st>>>(t, u, v, R.partials.p, R.counter.p, o);
  SEM_CHECK_CUDA(cudaGetLastError());
}

void launch_dot(const Topo &t, Reducer &R, const double *u, const double *v, double *out,
                cudaStream_t st) {
  dot_any(t, R, u, v, out, st);
}

void launch_dot(const Topo &t, Reducer &R, const float *u, const double *v, double *out,
                cudaStream_t st) {
  dot_any(t, R, u, v, out, st);
}

// ------------------------------------------------------------------ CG start
// r = b - w (w = A x assembled and masked, or r = b when w == null),
// z = dinv r (Jacobi) or z untouched (flexible: z comes from the V-cycle),
// p = z;  sums: bb = <b,b>, rr = <r,r>, rz = <r,z>.
__global__ void __launch_bounds__(kVecThreads)
    cg_start_kernel(Topo t, const double *__restrict__ b, const double *__restrict__ w,
                    const double *__restrict__ dinv, double *__restrict__ r,
                    double *__restrict__ z, double *__restrict__ p, double *partials,
                    unsigned int *counter, OutPtrs<3> out) {
  double acc[3] = {0.0, 0.0, 0.0};
  for (uint32_t l = blockIdx.x * blockDim.x + threadIdx.x; l < (uint32_t)t.nl;
       l += gridDim.x * blockDim.x) {
    PointInfo q = point_info(l, t);
    double bl = b[l];
    double rl = w ? bl - w[l] : bl;
    r[l] = rl;
    double rs = scale_pow2_down(rl, q.log2_mult);
    acc[0] = fma(scale_pow2_down(bl, q.log2_mult), bl, acc[0]);
    acc[1] = fma(rs, rl, acc[1]);
    if (dinv) {
      double zl = dinv[l] * rl;
      z[l] = zl;
      p[l] = zl;
      acc[2] = fma(rs, zl, acc[2]);
    }
  }
  grid_reduce<3>(acc, partials, counter, out.p);
}

void launch_cg_start(const Topo &t, Reducer &R, const double *b, const double *w,
                     const double *dinv, double *r, double *z, double *p, double *bb, double *rr,
                     double *rz, cudaStream_t st) {
  OutPtrs<3> o{{bb, rr, rz}};
  TraceScope ts("cg_start", t.N, st);
  cg_start_kernel<<<vec_grid(t.nl), kVecThreads, 0, st>>>(t, b, w, dinv, r, z, p, R.partials.p,
                                                          R.counter.p, o);
  SEM_CHECK_CUDA(cudaGetLastError());
}

// ------------------------------------------------------------------ CG iteration
// alpha = rho / pw;  x += alpha p;  r -= alpha w (w = A p assembled, masked);  rr = <r,r>;
// Jacobi: z = dinv r and rz = <r,z>.  rc32 / rc64: a copy of the new r (the
// V-cycle's input, FP32 rounded to nearest or FP64).  skip != null: the whole kernel is a
// no-op once *skip is set (device-side stop of the coarse solve).
__global__ void __launch_bounds__(kVecThreads)
    cg_update_kernel(Topo t, const double *__restrict__ rho, const double *__restrict__ pw,
                     const double *__restrict__ p, const double *__restrict__ w,
                     const double *__restrict__ dinv, double *__restrict__ x,
                     double *__restrict__ r, double *__restrict__ z, double *partials,
                     unsigned int *counter, OutPtrs<2> out, const int *__restrict__ skip,
                     float *__restrict__ rc32, double *__restrict__ rc64) {
  if (skip && *skip) return;
  const double alpha = *rho / *pw;
  double acc[2] = {0.0, 0.0};
  for (uint32_t l = blockIdx.x * blockDim.x + threadIdx.x; l < (uint32_t)t.nl;
       l += gridDim.x * blockDim.x) {
    PointInfo q = point_info(l, t);
    x[l] = fma(alpha, p[l], x[l]);
    double rl = fma(-alpha, w[l], r[l]);
    r[l] = rl;
    if (rc32) rc32[l] = (float)rl;
    if (rc64) rc64[l] = rl;
    double rs = scale_pow2_down(rl, q.log2_mult);
    acc[0] = fma(rs, rl, acc[0]);
    if (dinv) {
      double zl = dinv[l] * rl;
      z[l] = zl;
      acc[1] = fma(rs, zl, acc[1]);
    }
  }
  grid_reduce<2>(acc, partials, counter, out.p);
}

void launch_cg_update(const Topo &t, Reducer &R, const double *rho, const double *pw,
                      const double *p, const double *w, const double *dinv, double *x, double *r,
                      double *z, double *rr, double *rz, const int *skip, cudaStream_t st,
                      float *rc32, double *rc64) {
  OutPtrs<2> o{{rr, rz}};
  TraceScope ts("cg_update", t.N, st);
  cg_update_kernel<<<vec_grid(t.nl), kVecThreads, 0, st>>>(t, rho, pw, p, w, dinv, x, r, z,
                                                           R.partials.p, R.counter.p, o, skip,
                                                           rc32, rc64);
  SEM_CHECK_CUDA(cudaGetLastError());
}

// p = z + beta p with beta = num / den (Fletcher-Reeves: rz_new / rz_old) or
// beta = -num / den (flexible: -<z,w> / <p,w>); z in FP64 or FP32.
template <typename Tz>
__global__ void __launch_bounds__(kVecThreads)
    cg_direction_kernel(int64_t n, const double *__restrict__ num, const double *__restrict__ den,
                        double sign, const Tz *__restrict__ z, double *__restrict__ p,
                        const int *__restrict__ skip) {
  if (skip && *skip) return;
  const double beta = sign * *num / *den;
  for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < n;
       l += (int64_t)gridDim.x * blockDim.x)
    p[l] = as_f64(z[l]) + beta * p[l];
}

template <typename Tz>
void launch_cg_direction(int64_t n, const double *num, const double *den, double sign,
                         const Tz *z, double *p, const int *skip, cudaStream_t st) {
  TraceScope ts("cg_direction", 0, st);
  cg_direction_kernel<Tz><<<vec_grid(n), kVecThreads, 0, st>>>(n, num, den, sign, z, p, skip);
  SEM_CHECK_CUDA(cudaGetLastError());
}
template void launch_cg_direction<double>(int64_t, const double *, const double *, double,
                                          const double *, double *, const int *, cudaStream_t);
template void launch_cg_direction<float>(int64_t, const double *, const double *, double,
                                         const float *, double *, const int *, cudaStream_t);

// Flexible CG after the preconditioner: zr = <z, r>, zw = <z, w> (w masked);
// z in FP64, or the FP32 output of the V-cycle (widened exactly).
template <typename Tz>
__global__ void __launch_bounds__(kVecThreads)
    flex_dots_kernel(Topo t, const Tz *__restrict__ z, const double *__restrict__ r,
                     const double *__restrict__ w, double *partials, unsigned int *counter,
                     OutPtrs<2> out) {
  double acc[2] = {0.0, 0.0};
  for (uint32_t l = blockIdx.x * blockDim.x + threadIdx.x; l < (uint32_t)t.nl;
       l += gridDim.x * blockDim.x) {
    PointInfo q = point_info(l, t);
    const double zl = scale_pow2_down(as_f64(z[l]), q.log2_mult);
    acc[0] = fma(zl, r[l], acc[0]);
    acc[1] = fma(zl, w[l], acc[1]);
  }
  grid_reduce<2>(acc, partials, counter, out.p);
}

// The same two sums for an FP32 z whose element rows are whole float4s
// (Np % 4 == 0): four points per iteration, one index decode for the four
// (they share an element, j and k), and 16-byte loads of z, r and w.
__global__ void __launch_bounds__(kVecThreads)
    flex_dots4_kernel(Topo t, const float4 *__restrict__ z, const double2 *__restrict__ r,
                      const double2 *__restrict__ w, double *partials, unsigned int *counter,
                      OutPtrs<2> out) {
  double acc[2] = {0.0, 0.0};
  const uint32_t n4 = (uint32_t)t.nl / 4;
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < n4; q += gridDim.x * blockDim.x) {
    const float4 zv = z[q];
    const double2 r0 = r[2 * q], r1 = r[2 * q + 1], w0 = w[2 * q], w1 = w[2 * q + 1];
    const uint32_t l = q * 4;
    const uint32_t e = t.div_np3.div(l);
    const uint32_t jk = t.div_np.div(l - e * (uint32_t)t.Np3);
    const int i0 = (int)(l - e * (uint32_t)t.Np3 - jk * (uint32_t)t.Np);
    const int k = (int)t.div_np.div(jk);
    const int j = (int)(jk - (uint32_t)k * t.Np);
    const uint32_t yz = t.div_ex.div(e);
    const int ix = (int)(e - yz * (uint32_t)t.ex);
    const int iz = (int)t.div_ey.div(yz);
    const int iy = (int)(yz - (uint32_t)iz * t.ey);
    const uint32_t ef = elem_face_bits(ix, iy, iz, t);
    const float zc[4] = {zv.x, zv.y, zv.z, zv.w};
    const double rc[4] = {r0.x, r0.y, r1.x, r1.y}, wc[4] = {w0.x, w0.y, w1.x, w1.y};
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int lm = __popc(point_face_bits(i0 + c, j, k, t.N) & ~ef);
      const double zl = scale_pow2_down(widen_f32(zc[c]), lm);
      acc[0] = fma(zl, rc[c], acc[0]);
      acc[1] = fma(zl, wc[c], acc[1]);
    }
  }
  grid_reduce<2>(acc, partials, counter, out.p);
}

template <typename Tz>
void launch_flex_dots(const Topo &t, Reducer &R, const Tz *z, const double *r, const double *w,
                      double *zr, double *zw, cudaStream_t st) {
  OutPtrs<2> o{{zr, zw}};
  TraceScope ts("flex_dots", t.N, st);
  auto a16 = [](const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
  if constexpr (sizeof(Tz) == 4) {
    if (t.Np % 4 == 0 && (uint64_t)t.nl < (1ull << 32) && a16(z) && a16(r) && a16(w)) {
      flex_dots4_kernel<<<vec_grid(t.nl / 4), kVecThreads, 0, st>>>(
          t, reinterpret_cast<const float4 *>(z), reinterpret_cast<const double2 *>(r),
          reinterpret_cast<const double2 *>(w), R.partials.p, R.counter.p, o);
      SEM_CHECK_CUDA(cudaGetLastError());
      return;
    }
  }
  flex_dots_kernel<Tz><<<vec_grid(t.nl), kVecThreads, 0, st>>>(t, z, r, w, R.partials.p,
                                                               R.counter.p, o);
  SEM_CHECK_CUDA(cudaGetLastError());
}
template void launch_flex_dots<double>(const Topo &, Reducer &, const double *, const double *,
                                       const double *, double *, double *, cudaStream_t);
template void launch_flex_dots<float>(const Topo &, Reducer &, const float *, const double *,
                                      const double *, double *, double *, cudaStream_t);

// <p, mask gs(w)> for a continuous masked p and w = A_L p unassembled: the
// plain sum over local points (no weights, no gather); optional skip flag.
__global__ void __launch_bounds__(kVecThreads)
    dot_local_kernel(Topo t, const double *__restrict__ u, const double *__restrict__ v,
                     double *partials, unsigned int *counter, OutPtrs<1> out,
                     const int *__restrict__ skip) {
  if (skip && *skip) return;
  double acc[1] = {0.0};
  for (uint32_t l = blockIdx.x * blockDim.x + threadIdx.x; l < (uint32_t)t.nl;
       l += gridDim.x * blockDim.x)
    acc[0] = fma(u[l], v[l], acc[0]);
  grid_reduce<1>(acc, partials, counter, out.p);
}

void launch_dot_local(const Topo &t, Reducer &R, const double *u, const double *v, double *out,
                      const int *skip, cudaStream_t st) {
  OutPtrs<1> o{{out}};
  TraceScope ts("dot_local", t.N, st);
  dot_local_kernel<<<vec_grid(t.nl), kVecThreads, 0, st>>>(t, u, v, R.partials.p, R.counter.p, o,
                                                           skip);
  SEM_CHECK_CUDA(cudaGetLastError());
}

// <p, w> with a device-side skip flag (coarse solve).
__global__ void __launch_bounds__(kVecThreads)
    dot_skip_kernel(Topo t, const double *__restrict__ u, const double *__restrict__ v,
                    double *partials, unsigned int *counter, OutPtrs<1> out,
                    const int *__restrict__ skip) {
  if (skip && *skip) return;
  double acc[1] = {0.0};
  for (uint32_t l = blockIdx.x * blockDim.x + threadIdx.x; l < (uint32_t)t.nl;
       l += gridDim.x * blockDim.x) {
    PointInfo q = point_info(l, t);
    acc[0] = fma(scale_pow2_down(u[l], q.log2_mult), v[l], acc[0]);
  }
  grid_reduce<1>(acc, partials, counter, out.p);
}

void launch_dot_skip(const Topo &t, Reducer &R, const double *u, const double *v, double *out,
                     const int *skip, cudaStream_t st) {
  OutPtrs<1> o{{out}};
  TraceScope ts("dot", t.N, st);
  dot_skip_kernel<<<vec_grid(t.nl), kVecThreads, 0, st>>>(t, u, v, R.partials.p, R.counter.p, o,
                                                          skip);
  SEM_CHECK_CUDA(cudaGetLastError());
}

// Device-side stopping test of the coarse solve: skip = (rr <= tol^2 bb) or
// (iteration count reached).  One thread.
__global__ void stop_test_kernel(const double *__restrict__ rr, const double *__restrict__ bb,
                                 double tol2, int it, int maxit, int *skip, int *iters) {
  if (*skip) return;
  *iters = it;
  if (it >= maxit || !(*rr > tol2 * *bb)) *skip = 1;
}

void launch_stop_test(const double *rr, const double *bb, double tol2, int it, int maxit,
                      int *skip, int *iters, cudaStream_t st) {
  TraceScope ts("stop_test", 0, st);
  stop_test_kernel<<<1, 1, 0, st>>>(rr, bb, tol2, it, maxit, skip, iters);
  SEM_CHECK_CUDA(cudaGetLastError());
}

// Stopping test inside the device-driven FlexCG loop (a CUDA-graph while
// node).  g: 0 squared absolute tolerance on (r, r), 1 max_iter, 2 iterations done, 3 state (0 running,
// 1 stopped, 2 NaN/Inf residual).  Counts the iteration, stops at the
// tolerance, at max_iter or on a non-finite residual, and sets the loop's
// condition to "continue" only while running.
__global__ void graph_stop_kernel(const double *__restrict__ rr, double *g,
                                  cudaGraphConditionalHandle h) {
  const double it = g[2] + 1.0;
  g[2] = it;
  const double v = *rr;
  double state = 0.0;
  if (!(v == v) || isinf(v)) state = 2.0;
  else if (!(v > g[0]) || it >= g[1]) state = 1.0;
  g[3] = state;
  cudaGraphSetConditional(h, state == 0.0 ? 1u : 0u);
}

__global__ void graph_arm_kernel(double *g, double tol2, double maxit, double done) {
  g[0] = tol2;
  g[1] = maxit;
  g[2] = done;
  g[3] = 0.0;
}

// Start of a solve run wholly on the device: the stopping state from the
// start kernel's <b, b> and <r, r> (the host loop's tests, in the same
// arithmetic), g[4] = the initial <r, r>, and the condition of the node that
// runs the iterations (1 while iterations are due).
__global__ void graph_arm_full_kernel(const double *__restrict__ bb, const double *__restrict__ rr,
                                      double *g, double tol, double maxit,
                                      cudaGraphConditionalHandle h) {
  const double b = *bb, r = *rr;
  const double tol2 = tol * tol * b;
  g[0] = tol2;
  g[1] = maxit;
  g[2] = 0.0;
  g[4] = r;
  double state = 0.0;
  if (!(r == r) || !(b == b)) state = 2.0;
  else if (r <= tol2 || maxit < 1.0) state = 1.0;
  g[3] = state;
  cudaGraphSetConditional(h, state == 0.0 ? 1u : 0u);
}

void launch_graph_arm_full(const double *bb, const double *rr, double *g, double tol, int maxit,
                           cudaGraphConditionalHandle h, cudaStream_t st) {
  TraceScope ts("graph_ctl", 0, st);
  graph_arm_full_kernel<<<1, 1, 0, st>>>(bb, rr, g, tol, (double)maxit, h);
  SEM_CHECK_CUDA(cudaGetLastError());
}

void launch_graph_stop(const double *rr, double *g, cudaGraphConditionalHandle h,
                       cudaStream_t st) {
  TraceScope ts("graph_ctl", 0, st);
  graph_stop_kernel<<<1, 1, 0, st>>>(rr, g, h);
  SEM_CHECK_CUDA(cudaGetLastError());
}

void launch_graph_arm(double *g, double tol2, int maxit, int done, cudaStream_t st) {
  TraceScope ts("graph_ctl", 0, st);
  graph_arm_kernel<<<1, 1, 0, st>>>(g, tol2, (double)maxit, (double)done);
  SEM_CHECK_CUDA(cudaGetLastError());
}

// ------------------------------------------------------------------ conversions
template <typename A, typename B>
__global__ void convert_kernel(int64_t n, const A *__restrict__ a, B *__restrict__ b) {
  for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < n;
       l += (int64_t)gridDim.x * blockDim.x)
    b[l] = (B)a[l];
}

template <typename A, typename B>
void launch_convert(int64_t n, const A *a, B *b, cudaStream_t st) {
  TraceScope ts("convert", 0, st);
  convert_kernel<A, B><<<vec_grid(n), kVecThreads, 0, st>>>(n, a, b);
  SEM_CHECK_CUDA(cudaGetLastError());
}
template void launch_convert<double, float>(int64_t, const double *, float *, cudaStream_t);
template void launch_convert<float, double>(int64_t, const float *, double *, cudaStream_t);
template void launch_convert<double, double>(int64_t, const double *, double *, cudaStream_t);
template void launch_convert<float, float>(int64_t, const float *, float *, cudaStream_t);

// Neumann: subtract the unique-dof mean, u -= (sum u/mult) / (sum 1/mult).
__global__ void sub_mean_kernel(Topo t, const double *__restrict__ sum, double *__restrict__ u) {
  const double mean = *sum / (double)t.ng;
  for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < t.nl;
       l += (int64_t)gridDim.x * blockDim.x)
    u[l] -= mean;
}

__global__ void __launch_bounds__(kVecThreads)
    sum_kernel(Topo t, const double *__restrict__ u, double *partials, unsigned int *counter,
               OutPtrs<1> out) {
  double acc[1] = {0.0};
  for (uint32_t l = blockIdx.x * blockDim.x + threadIdx.x; l < (uint32_t)t.nl;
       l += gridDim.x * blockDim.x) {
    PointInfo q = point_info(l, t);
    acc[0] += scale_pow2_down(u[l], q.log2_mult);
  }
  grid_reduce<1>(acc, partials, counter, out.p);
}

void launch_remove_mean(const Topo &t, Reducer &R, double *u, double *scratch, cudaStream_t st) {
  OutPtrs<1> o{{scratch}};
  TraceScope ts("mean", t.N, st, 2);
  sum_kernel<<<vec_grid(t.nl), kVecThreads, 0, st>>>(t, u, R.partials.p, R.counter.p, o);
  SEM_CHECK_CUDA(cudaGetLastError());
  sub_mean_kernel<<<vec_grid(t.nl), kVecThreads, 0, st>>>(t, scratch, u);
  SEM_CHECK_CUDA(cudaGetLastError());
}

void launch_sum(const Topo &t, Reducer &R, const double *u, double *out, cudaStream_t st) {
  OutPtrs<1> o{{out}};
  TraceScope ts("sum", t.N, st);
  sum_kernel<<<vec_grid(t.nl), kVecThreads, 0, st>>>(t, u, R.partials.p, R.counter.p, o);
  SEM_CHECK_CUDA(cudaGetLastError());
}

}  // namespace sem
