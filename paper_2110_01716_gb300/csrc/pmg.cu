// pmg.cu -- p-multigrid preconditioner (Sec. 3, pMG paragraph).
//
// Levels of decreasing polynomial order on the same trilinear geometry;
// coarse-to-fine interpolation u_f = (J x J x J) u_c with one 1D matrix J per
// level pair; restriction is its transpose on unique dofs,
// r_c = mask_c gs_c((J^T x J^T x J^T)(r_f / mult_f)); Chebyshev-accelerated
// point-Jacobi smoothing in FP64 or FP32 (the paper runs all of pMG in 32-bit);
// the coarsest level is solved by FP64 Jacobi-PCG on the device (the paper
// used an algebraic multigrid on the host there).  One V-cycle: pre-smooth
// from zero, residual, restrict, recurse, prolong and correct, post-smooth.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <type_traits>

#include "common.cuh"
#include "kernels.cuh"
#include "pmg.cuh"
#include "trace.cuh"

namespace sem {

// ------------------------------------------------------------------ Chebyshev
// Start of a Chebyshev smoothing: r = b - w (w = A x assembled and masked, or
// r = b when w is null and x = 0), d = dinv r / theta, x = d (x_zero) or x += d.
template <typename T>
__global__ void cheb_start_kernel(Topo t, const T *__restrict__ b, const T *__restrict__ w,
                                  const T *__restrict__ dinv, T *__restrict__ r, T *__restrict__ d,
                                  T *__restrict__ x, T inv_theta, int x_zero) {
  for (uint32_t l = blockIdx.x * blockDim.x + threadIdx.x; l < (uint32_t)t.nl;
       l += gridDim.x * blockDim.x) {
    T rl = w ? b[l] - w[l] : b[l];
    r[l] = rl;
    T dl = dinv[l] * rl * inv_theta;
    d[l] = dl;
    x[l] = x_zero ? dl : x[l] + dl;
  }
}

// One Chebyshev step after w = A d (assembled and masked):
// r -= w;  d = c1 d + c2 dinv r;  x += d.  The last step of a smoothing
// (last) does not store r: the V-cycle recomputes the residual from x.
template <typename T>
__global__ void cheb_step_kernel(Topo t, const T *__restrict__ w, const T *__restrict__ dinv,
                                 T *__restrict__ r, T *__restrict__ d, T *__restrict__ x, T c1,
                                 T c2, int last) {
  for (uint32_t l = blockIdx.x * blockDim.x + threadIdx.x; l < (uint32_t)t.nl;
       l += gridDim.x * blockDim.x) {
    T rl = r[l] - w[l];
    if (!last) r[l] = rl;
    T dl = c1 * d[l] + c2 * dinv[l] * rl;
    d[l] = dl;
    x[l] += dl;
  }
}

// FP32 forms of the two kernels above on float4 (nl a multiple of 4): fewer
// instructions and four independent loads per stream in flight per thread.
__device__ __forceinline__ float4 f4fma(float a, float4 x, float4 y) {
  return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
}
// x_zero with only_d: r (= b) and x (= d) are not written; the first step
// reads b and d in their place.
__global__ void cheb_start4_kernel(int64_t n4, const float4 *__restrict__ b,
                                   const float4 *__restrict__ w, const float4 *__restrict__ dinv,
                                   float4 *__restrict__ r, float4 *__restrict__ d,
                                   float4 *__restrict__ x, float inv_theta, int x_zero,
                                   int only_d) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n4;
       q += (int64_t)gridDim.x * blockDim.x) {
    float4 rl = b[q];
    if (w) {
      const float4 wl = w[q];
      rl = make_float4(rl.x - wl.x, rl.y - wl.y, rl.z - wl.z, rl.w - wl.w);
    }
    const float4 di = dinv[q];
    const float4 dl = make_float4(di.x * rl.x * inv_theta, di.y * rl.y * inv_theta,
                                  di.z * rl.z * inv_theta, di.w * rl.w * inv_theta);
    d[q] = dl;
    if (only_d) continue;
    r[q] = rl;
    if (x_zero) {
      x[q] = dl;
    } else {
      const float4 xl = x[q];
      x[q] = make_float4(xl.x + dl.x, xl.y + dl.y, xl.z + dl.z, xl.w + dl.w);
    }
  }
}

// first: the step after a start that wrote d only (r = b, x = d there);
// last: the smoothing's last step, whose r is not stored.
__global__ void cheb_step4_kernel(int64_t n4, const float4 *__restrict__ w,
                                  const float4 *__restrict__ dinv, const float4 *__restrict__ b,
                                  float4 *__restrict__ r, float4 *__restrict__ d,
                                  float4 *__restrict__ x, float c1, float c2, int first,
                                  int last) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n4;
       q += (int64_t)gridDim.x * blockDim.x) {
    const float4 wl = w[q], di = dinv[q], d0 = d[q];
    const float4 r0 = first ? b[q] : r[q];
    const float4 x0 = first ? d0 : x[q];
    const float4 rl = make_float4(r0.x - wl.x, r0.y - wl.y, r0.z - wl.z, r0.w - wl.w);
    const float4 dl = make_float4(c1 * d0.x + c2 * di.x * rl.x, c1 * d0.y + c2 * di.y * rl.y,
                                  c1 * d0.z + c2 * di.z * rl.z, c1 * d0.w + c2 * di.w * rl.w);
    if (!last) r[q] = rl;
    d[q] = dl;
    x[q] = make_float4(x0.x + dl.x, x0.y + dl.y, x0.z + dl.z, x0.w + dl.w);
  }
}

// Chebyshev with a general preconditioner M (the Schwarz smoother): the
// residual update r = b - w (b given) or r -= w, and the direction update
// d = c1 d + c2 (M r) (c1 = 0: start), x = d (x_zero) or x += d.
template <typename T>
__global__ void resid_kernel(int64_t n, const T *__restrict__ b, const T *__restrict__ w,
                             T *__restrict__ r) {
  for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < n;
       l += (int64_t)gridDim.x * blockDim.x)
    r[l] = (b ? b[l] : r[l]) - w[l];
}

template <typename T>
__global__ void cheb_m_kernel(int64_t n, const T *__restrict__ mr, T *__restrict__ d,
                              T *__restrict__ x, T c1, T c2, int start, int x_zero) {
  for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < n;
       l += (int64_t)gridDim.x * blockDim.x) {
    const T dl = start ? c2 * mr[l] : c1 * d[l] + c2 * mr[l];
    d[l] = dl;
    x[l] = x_zero ? dl : x[l] + dl;
  }
}

// ------------------------------------------------------------------ transfers
struct TransferParams {
  Topo tf;      // fine level
  int npf, npc; // points per direction
  double J[kMaxNp * kMaxNp];  // J[i*npc + a]: coarse basis a at fine node i
};

// Arithmetic of a transfer: FP32 when either level smooths in FP32 (the data
// carries single precision then), FP64 otherwise.
template <typename A, typename B>
struct TransferCompute {
  using type = double;
};
template <>
struct TransferCompute<float, float> {
  using type = float;
};
template <>
struct TransferCompute<float, double> {
  using type = float;
};
template <>
struct TransferCompute<double, float> {
  using type = float;
};

// Restriction of the fine residual b - w (w = A x assembled and masked),
// weighted by 1/mult, to unassembled coarse values:
// out_e = (J^T x J^T x J^T) ((b - w)/mult)_e.  One CTA per element.
template <typename Tf, typename Tc>
__global__ void restrict_kernel(TransferParams tp, const Tf *__restrict__ b,
                                const Tf *__restrict__ w, Tc *__restrict__ out) {
  using R = typename TransferCompute<Tf, Tc>::type;
  extern __shared__ double sm_raw[];
  R *sm = reinterpret_cast<R *>(sm_raw);
  __shared__ R sJ[kMaxNp * kMaxNp];
  const int nf = tp.npf, nc = tp.npc;
  const int nf3 = nf * nf * nf;
  R *s0 = sm;                    // nf^3
  R *s1 = s0 + nf3;              // nc nf nf
  R *s2 = s1 + nc * nf * nf;     // nc nc nf
  for (int q = threadIdx.x; q < nf * nc; q += blockDim.x) sJ[q] = (R)tp.J[q];
  for (int64_t e = blockIdx.x; e < tp.tf.E; e += gridDim.x) {
    for (int q = threadIdx.x; q < nf3; q += blockDim.x) {
      uint32_t l = (uint32_t)(e * nf3 + q);
      PointInfo pi = point_info(l, tp.tf);
      s0[q] = ((R)b[l] - (R)w[l]) * (R)pi.inv_mult;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < nc * nf * nf; q += blockDim.x) {
      int a = q % nc, jk = q / nc;
      R s = 0;
      for (int i = 0; i < nf; ++i) s += sJ[i * nc + a] * s0[i + nf * jk];
      s1[q] = s;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < nc * nc * nf; q += blockDim.x) {
      int a = q % nc, bk = q / nc, bb = bk % nc, k = bk / nc;
      R s = 0;
      for (int j = 0; j < nf; ++j) s += sJ[j * nc + bb] * s1[a + nc * (j + nf * k)];
      s2[q] = s;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < nc * nc * nc; q += blockDim.x) {
      int ab = q % (nc * nc), c = q / (nc * nc);
      R s = 0;
      for (int k = 0; k < nf; ++k) s += sJ[k * nc + c] * s2[ab + nc * nc * k];
      out[e * nc * nc * nc + q] = (Tc)s;
    }
    __syncthreads();
  }
}

// Prolongation and correction: x_f += (J x J x J) x_c.  One CTA per element.
template <typename Tc, typename Tf>
__global__ void prolong_kernel(TransferParams tp, const Tc *__restrict__ xc, Tf *__restrict__ xf) {
  using R = typename TransferCompute<Tf, Tc>::type;
  extern __shared__ double sm_raw[];
  R *sm = reinterpret_cast<R *>(sm_raw);
  __shared__ R sJ[kMaxNp * kMaxNp];
  const int nf = tp.npf, nc = tp.npc;
  const int nc3 = nc * nc * nc, nf3 = nf * nf * nf;
  R *s0 = sm;                // nc^3
  R *s1 = s0 + nc3;          // nf nc nc
  R *s2 = s1 + nf * nc * nc; // nf nf nc
  for (int q = threadIdx.x; q < nf * nc; q += blockDim.x) sJ[q] = (R)tp.J[q];
  for (int64_t e = blockIdx.x; e < tp.tf.E; e += gridDim.x) {
    for (int q = threadIdx.x; q < nc3; q += blockDim.x) s0[q] = (R)xc[e * nc3 + q];
    __syncthreads();
    for (int q = threadIdx.x; q < nf * nc * nc; q += blockDim.x) {
      int i = q % nf, bc = q / nf;
      R s = 0;
      for (int a = 0; a < nc; ++a) s += sJ[i * nc + a] * s0[a + nc * bc];
      s1[q] = s;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < nf * nf * nc; q += blockDim.x) {
      int i = q % nf, jc = q / nf, j = jc % nf, c = jc / nf;
      R s = 0;
      for (int b = 0; b < nc; ++b) s += sJ[j * nc + b] * s1[i + nf * (b + nc * c)];
      s2[q] = s;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < nf3; q += blockDim.x) {
      int ij = q % (nf * nf), k = q / (nf * nf);
      R s = 0;
      for (int c = 0; c < nc; ++c) s += sJ[k * nc + c] * s2[ij + nf * nf * c];
      xf[e * nf3 + q] = (Tf)((R)xf[e * nf3 + q] + s);
    }
    __syncthreads();
  }
}

// Transfers with compile-time orders: NE elements per CTA, one thread per
// (i, j) column of a fine element.  The contraction along t is thread-local;
// r and s pass through shared memory; two barriers per chunk of elements.
template <int NF>
struct TrShape {
  static constexpr int NF2 = NF * NF;
  static constexpr int NE = (256 / NF2) < 1 ? 1 : (256 / NF2);
  static constexpr int THREADS = NE * NF2;
  // six CTAs per SM (40 registers): at 48^3 the transfers between N = 7 and
  // N = 4 took 0.176 -> 0.141 ms (restriction) and 0.146 -> 0.130 ms
  // (prolongation) against the compiler's choice of four; eight spilled
  // and lost
#ifndef SEM_TR_MIN_CTAS
#define SEM_TR_MIN_CTAS 6
#endif
  static constexpr int MIN_CTAS = SEM_TR_MIN_CTAS;
};

// 2^-(number of elements sharing fine point (i, j, k) besides its own) as the
// box topology fixes it: each direction in which the point lies on a face
// between two elements doubles the copies.
__device__ __forceinline__ int shared_dirs(int i, int j, int k, int N, int ix, int iy, int iz,
                                           const Topo &t) {
  return ((i == 0 && ix > 0) || (i == N && ix < t.ex - 1)) +
         ((j == 0 && iy > 0) || (j == N && iy < t.ey - 1)) +
         ((k == 0 && iz > 0) || (k == N && iz < t.ez - 1));
}

template <int NF, int NC, typename Tf, typename Tc>
__global__ void __launch_bounds__(TrShape<NF>::THREADS, TrShape<NF>::MIN_CTAS)
    restrict_fast_kernel(TransferParams tp, const Tf *__restrict__ b, const Tf *__restrict__ w,
                         Tc *__restrict__ out) {
  using R = typename TransferCompute<Tf, Tc>::type;
  constexpr int NF2 = NF * NF, NF3 = NF2 * NF, NC2 = NC * NC, NC3 = NC2 * NC;
  constexpr int NE = TrShape<NF>::NE, N = NF - 1;
  __shared__ R sJ[NF * NC];
  __shared__ R s1[NE][NC * NF2];  // y(i, j, c) = sum_k J[k][c] v(i, j, k)
  __shared__ R s2[NE][NC2 * NF];  // z(i, b, c) = sum_j J[j][b] y(i, j, c)
  const Topo &t = tp.tf;
  const int le = threadIdx.x / NF2, ij = threadIdx.x - le * NF2;
  const int i = ij % NF, j = ij / NF;
  for (int q = threadIdx.x; q < NF * NC; q += blockDim.x) sJ[q] = (R)tp.J[q];
  __syncthreads();
  // the inputs of this thread's next batch are loaded into registers while
  // the current batch is contracted (the loads' latency overlaps the barriers)
  Tf bn[NF], wn[NF];
  auto load = [&](int64_t e) {
    if (e < t.E) {
#pragma unroll
      for (int k = 0; k < NF; ++k) {
        const int64_t l = e * NF3 + k * NF2 + ij;
        bn[k] = b[l];
        wn[k] = w[l];
      }
    }
  };
  load((int64_t)blockIdx.x * NE + le);
  for (int64_t e0 = (int64_t)blockIdx.x * NE; e0 < t.E; e0 += (int64_t)gridDim.x * NE) {
    const int64_t e = e0 + le;
    const bool active = e < t.E;
    if (active) {
      const uint32_t e32 = (uint32_t)e, r1 = t.div_ex.div(e32);
      const int ix = (int)(e32 - r1 * t.ex), iz = (int)t.div_ey.div(r1);
      const int iy = (int)(r1 - (uint32_t)iz * t.ey);
      R v[NF];
#pragma unroll
      for (int k = 0; k < NF; ++k) {
        const int sd = shared_dirs(i, j, k, N, ix, iy, iz, t);
        v[k] = ((R)bn[k] - (R)wn[k]) * (R)(1.0f / (float)(1 << sd));
      }
      load(e + (int64_t)gridDim.x * NE);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        R y = 0;
#pragma unroll
        for (int k = 0; k < NF; ++k) y += sJ[k * NC + c] * v[k];
        s1[le][c * NF2 + ij] = y;
      }
    }
    __syncthreads();
    // the j and i contractions one line per thread: a line is read once for
    // its NC outputs, and J is read at warp-uniform addresses (broadcast)
    if (active) {
      for (int q = ij; q < NF * NC; q += NF2) {
        const int ii = q % NF, c = q / NF;  // line (ii, ., c) of y
        R yl[NF];
#pragma unroll
        for (int jj = 0; jj < NF; ++jj) yl[jj] = s1[le][c * NF2 + jj * NF + ii];
#pragma unroll
        for (int bb = 0; bb < NC; ++bb) {
          R z = 0;
#pragma unroll
          for (int jj = 0; jj < NF; ++jj) z += sJ[jj * NC + bb] * yl[jj];
          s2[le][(c * NC + bb) * NF + ii] = z;
        }
      }
    }
    __syncthreads();
    if (active) {
      for (int bc = ij; bc < NC2; bc += NF2) {  // line (., b, c) of z
        R zl[NF];
#pragma unroll
        for (int ii = 0; ii < NF; ++ii) zl[ii] = s2[le][bc * NF + ii];
#pragma unroll
        for (int a = 0; a < NC; ++a) {
          R o = 0;
#pragma unroll
          for (int ii = 0; ii < NF; ++ii) o += sJ[ii * NC + a] * zl[ii];
          out[e * NC3 + bc * NC + a] = (Tc)o;
        }
      }
    }
  }
}

template <int NF, int NC, typename Tc, typename Tf>
__global__ void __launch_bounds__(TrShape<NF>::THREADS, TrShape<NF>::MIN_CTAS)
    prolong_fast_kernel(TransferParams tp, const Tc *__restrict__ xc, Tf *__restrict__ xf) {
  using R = typename TransferCompute<Tf, Tc>::type;
  constexpr int NF2 = NF * NF, NF3 = NF2 * NF, NC2 = NC * NC, NC3 = NC2 * NC;
  constexpr int NE = TrShape<NF>::NE;
  __shared__ R sJ[NF * NC];
  __shared__ R s0[NE][NC3];       // coarse element
  __shared__ R s1[NE][NF * NC2];  // z(i, b, c) = sum_a J[i][a] x(a, b, c)
  const Topo &t = tp.tf;
  const int le = threadIdx.x / NF2, ij = threadIdx.x - le * NF2;
  const int i = ij % NF, j = ij / NF;
  for (int q = threadIdx.x; q < NF * NC; q += blockDim.x) sJ[q] = (R)tp.J[q];
  // the coarse values and the fine column of this thread's next batch are
  // loaded into registers while the current batch is interpolated (the
  // loads' latency overlaps the barriers; the fine values were read only
  // after them before, which left the kernel waiting on memory)
  constexpr int QC = (NC3 + NF2 - 1) / NF2;
  Tc cn[QC];
  Tf fn[NF];
  auto load = [&](int64_t e) {
    if (e < t.E) {
#pragma unroll
      for (int r = 0; r < QC; ++r)
        if (ij + r * NF2 < NC3) cn[r] = xc[e * NC3 + ij + r * NF2];
#pragma unroll
      for (int k = 0; k < NF; ++k) fn[k] = xf[e * NF3 + k * NF2 + ij];
    }
  };
  load((int64_t)blockIdx.x * NE + le);
  for (int64_t e0 = (int64_t)blockIdx.x * NE; e0 < t.E; e0 += (int64_t)gridDim.x * NE) {
    const int64_t e = e0 + le;
    const bool active = e < t.E;
    R fc[NF];
    if (active) {
#pragma unroll
      for (int r = 0; r < QC; ++r)
        if (ij + r * NF2 < NC3) s0[le][ij + r * NF2] = (R)cn[r];
#pragma unroll
      for (int k = 0; k < NF; ++k) fc[k] = (R)fn[k];
      load(e + (int64_t)gridDim.x * NE);
    }
    __syncthreads();
    if (active) {
      for (int q = ij; q < NF * NC2; q += NF2) {
        const int ii = q % NF, bc = q / NF;
        R z = 0;
#pragma unroll
        for (int a = 0; a < NC; ++a) z += sJ[ii * NC + a] * s0[le][a + NC * bc];
        s1[le][q] = z;
      }
    }
    __syncthreads();
    if (active) {
      R z2[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        R z = 0;
#pragma unroll
        for (int bb = 0; bb < NC; ++bb) z += sJ[j * NC + bb] * s1[le][(c * NC + bb) * NF + i];
        z2[c] = z;
      }
#pragma unroll
      for (int k = 0; k < NF; ++k) {
        R s = 0;
#pragma unroll
        for (int c = 0; c < NC; ++c) s += sJ[k * NC + c] * z2[c];
        xf[e * NF3 + k * NF2 + ij] = (Tf)(fc[k] + s);
      }
    }
  }
}

// ------------------------------------------------------------------ Lanczos start vector
// splitmix64 (Steele, Lea and Flood 2014) keyed by the node's unique id:
// v = 2 u - 1 with u the top 53 bits times 2^-53; masked.
__global__ void random_start_kernel(Topo t, uint64_t seed, double *__restrict__ v) {
  const uint64_t nx = (uint64_t)t.ex * t.N + 1, ny = (uint64_t)t.ey * t.N + 1;
  for (uint32_t l = blockIdx.x * blockDim.x + threadIdx.x; l < (uint32_t)t.nl;
       l += gridDim.x * blockDim.x) {
    PointInfo q = point_info(l, t);
    uint64_t gx = (uint64_t)q.ix * t.N + q.i, gy = (uint64_t)q.iy * t.N + q.j,
             gz = (uint64_t)q.iz * t.N + q.k;
    uint64_t id = gx + nx * (gy + ny * gz);
    uint64_t z = seed + (id + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
    v[l] = (2.0 * u - 1.0) * (double)q.mask;
  }
}

// Largest eigenvalue of the symmetric tridiagonal (diag a, off-diagonal b) by
// bisection: the number of negative pivots of the LDL^T factorisation of
// T - mu I counts the eigenvalues below mu (Sylvester's law of inertia).
static double tridiag_lambda_max(const std::vector<double> &a, const std::vector<double> &b) {
  const int m = (int)a.size();
  double lo = a[0], hi = a[0];
  for (int i = 0; i < m; ++i) {
    double rad = 0.0;
    if (i > 0) rad += std::fabs(b[i - 1]);
    if (i + 1 < m) rad += std::fabs(b[i]);
    lo = std::min(lo, a[i] - rad);
    hi = std::max(hi, a[i] + rad);
  }
  auto below = [&](double mu) {
    int neg = 0;
    double piv = a[0] - mu;
    if (piv < 0) ++neg;
    for (int i = 1; i < m; ++i) {
      if (piv == 0.0) piv = 1e-300;
      piv = (a[i] - mu) - b[i - 1] * b[i - 1] / piv;
      if (piv < 0) ++neg;
    }
    return neg;
  };
  for (int it = 0; it < 300 && hi - lo > 1e-15 * std::fabs(hi); ++it) {
    double mid = 0.5 * (lo + hi);
    if (below(mid) == m) hi = mid; else lo = mid;
  }
  return hi;
}

// lambda_max(D^-1 A) from the Lanczos tridiagonal of m steps of Jacobi-PCG on
// A y = v (alpha_j, beta_j give T_jj = 1/alpha_j + beta_{j-1}/alpha_{j-1},
// T_j,j+1 = sqrt(beta_j)/alpha_j).
static double lanczos_lambda_max(Level &L, Reducer &R, int m, uint64_t seed, cudaStream_t st,
                                 const AsmData *asmd = nullptr) {
  const Topo &t = L.t;
  DevBuf<double> v, r, z, p, w, x, sc;
  v.alloc(t.nl); r.alloc(t.nl); z.alloc(t.nl); p.alloc(t.nl); w.alloc(t.nl); x.alloc(t.nl);
  sc.alloc(8);
  {
  TraceScope ts("lanczos_start", t.N, st);
  random_start_kernel<<<vec_grid(t.nl), kVecThreads, 0, st>>>(t, seed, v.p);
  SEM_CHECK_CUDA(cudaGetLastError());
  }
  if (t.bc == SEM_NEUMANN) launch_remove_mean(t, R, v.p, sc.p + 7, st);
  SEM_CHECK_CUDA(cudaMemsetAsync(x.p, 0, t.nl * sizeof(double), st));
  // slots: 0 bb, 1 rr, 2 rho_a, 3 rho_b, 4 pw.  With the Schwarz preconditioner
  // z = M r is applied apart and rho = <r, z> taken by a dot.
  if (asmd) {
    launch_cg_start(t, R, v.p, nullptr, nullptr, r.p, nullptr, nullptr, sc.p + 0, sc.p + 1,
                    sc.p + 2, st);
    launch_asm<double>(*asmd, L, r.p, z.p, st);
    launch_dot(t, R, r.p, z.p, sc.p + 2, st);
    launch_convert<double, double>(t.nl, z.p, p.p, st);
  } else {
    launch_cg_start(t, R, v.p, nullptr, L.dinv64.p, r.p, z.p, p.p, sc.p + 0, sc.p + 1, sc.p + 2,
                    st);
  }
  std::vector<double> alpha, beta;
  double h[8];
  SEM_CHECK_CUDA(cudaMemcpyAsync(h, sc.p, 8 * sizeof(double), cudaMemcpyDeviceToHost, st));
  SEM_CHECK_CUDA(cudaStreamSynchronize(st));
  double rho0 = h[2], rho = h[2];
  for (int j = 0; j < m; ++j) {
    int cur = 2 + (j & 1), nxt = 2 + ((j + 1) & 1);
    apply_assembled<double>(L, p.p, w.p, st);
    launch_dot(t, R, p.p, w.p, sc.p + 4, st);
    launch_cg_update(t, R, sc.p + cur, sc.p + 4, p.p, w.p, asmd ? nullptr : L.dinv64.p, x.p, r.p,
                     z.p, sc.p + 1, sc.p + nxt, nullptr, st);
    if (asmd) {
      launch_asm<double>(*asmd, L, r.p, z.p, st);
      launch_dot(t, R, r.p, z.p, sc.p + nxt, st);
    }
    SEM_CHECK_CUDA(cudaMemcpyAsync(h, sc.p, 8 * sizeof(double), cudaMemcpyDeviceToHost, st));
    SEM_CHECK_CUDA(cudaStreamSynchronize(st));
    double pw = h[4], rho1 = h[nxt];
    double a = rho / pw, bta = rho1 / rho;
    alpha.push_back(a);
    beta.push_back(bta);
    rho = rho1;
    if (!(rho1 > 1e-28 * rho0)) break;
    launch_cg_direction(t.nl, sc.p + nxt, sc.p + cur, 1.0, z.p, p.p, nullptr, st);
  }
  const int k = (int)alpha.size();
  std::vector<double> ta(k), tb(k > 1 ? k - 1 : 0);
  for (int j = 0; j < k; ++j) {
    ta[j] = 1.0 / alpha[j] + (j > 0 ? beta[j - 1] / alpha[j - 1] : 0.0);
    if (j + 1 < k) tb[j] = std::sqrt(beta[j]) / alpha[j];
  }
  return tridiag_lambda_max(ta, tb);
}

// ------------------------------------------------------------------ setup
static int grid_elems(int64_t E) { return (int)std::min<int64_t>(E, 152 * 16); }

template <typename T>
static T *vec_of(PmgLevel &P, int which) {
  if constexpr (sizeof(T) == 8) return P.v64[which].p;
  else return P.v32[which].p;
}

void pmg_build(sem_pmg *P, sem_mesh *mesh, const sem_pmg_desc &d, cudaStream_t st) {
  SEM_REQUIRE(d.nlevels >= 1 && d.nlevels <= 8, "nlevels=%d outside [1,8]", d.nlevels);
  SEM_REQUIRE(d.orders[0] == mesh->fine.t.N, "orders[0]=%d differs from the mesh order %d",
              d.orders[0], mesh->fine.t.N);
  for (int l = 1; l < d.nlevels; ++l)
    SEM_REQUIRE(d.orders[l] >= 1 && d.orders[l] < d.orders[l - 1],
                "orders must be strictly decreasing and >= 1");
  SEM_REQUIRE(d.cheb_degree >= 1 && d.cheb_degree <= 16, "cheb_degree=%d outside [1,16]",
              d.cheb_degree);
  SEM_REQUIRE(d.lanczos_steps >= 2 && d.lanczos_steps <= 200, "lanczos_steps outside [2,200]");
  SEM_REQUIRE(d.smoother_dtype >= SEM_F64 && d.smoother_dtype <= SEM_BF16,
              "smoother_dtype must be SEM_F64, SEM_F32, SEM_F16 or SEM_BF16");
  SEM_REQUIRE(d.coarse_maxit >= 0 && d.coarse_maxit <= 100000, "coarse_maxit out of range");
  SEM_REQUIRE(d.smoother == SEM_SMOOTH_JACOBI || d.smoother == SEM_SMOOTH_ASM ||
                  d.smoother == SEM_SMOOTH_ASM_TC || d.smoother == SEM_SMOOTH_ASM_TF32,
              "unknown smoother %d", d.smoother);
  SEM_REQUIRE((d.smoother != SEM_SMOOTH_ASM_TC && d.smoother != SEM_SMOOTH_ASM_TF32) ||
                  d.smoother_dtype != SEM_F64,
              "the tensor-core Schwarz smoothers smooth in FP32 (smoother_dtype F32, F16 or BF16)");
  P->mesh = mesh;
  P->desc = d;
  const Level &F = mesh->fine;
  P->red.init(kVecMaxBlocks, 4);
  P->scal.alloc(32);
  P->flags.alloc(4);
  P->levp.clear();
  for (int l = 0; l < d.nlevels; ++l) P->levp.emplace_back(new PmgLevel());
  for (int l = 0; l < d.nlevels; ++l) {
    PmgLevel &Q = *P->levp[l];
    const bool coarsest = (l == d.nlevels - 1);
    const bool half = d.smoother_dtype == SEM_F16 || d.smoother_dtype == SEM_BF16;
    Q.dtype = coarsest ? SEM_F64 : (half ? SEM_F32 : d.smoother_dtype);
    Q.g16 = (!coarsest && half) ? d.smoother_dtype : 0;
    if (l == 0) {
      Q.L = &mesh->fine;
    } else {
      Q.own.reset(new Level());
      // the N = 1 coarsest level keeps FP64 factors for its element matrices
      const int arith = (coarsest && d.orders[l] == 1) ? SEM_ARITH_NATIVE : F.arith;
      build_level(*Q.own, F.t.ex, F.t.ey, F.t.ez, d.orders[l], F.t.bc, SEM_GEOM_STORED, arith,
                  F.verts_host.data(), Q.dtype == SEM_F32 && !Q.g16, st);
      Q.L = Q.own.get();
    }
    if (Q.g16) level_ensure_g16(*Q.L, Q.g16, st);
    else if (Q.dtype == SEM_F32) level_ensure_f32(*Q.L, st);
    const int64_t n = Q.L->t.nl;
    // vectors: 0 b, 1 x, 2 r, 3 d, 4 w
    for (int v = 0; v < 5; ++v) {
      if (Q.dtype == SEM_F32) Q.v32[v].alloc(n);
      else Q.v64[v].alloc(n);
    }
    if (!coarsest) {
      if (d.smoother == SEM_SMOOTH_ASM || d.smoother == SEM_SMOOTH_ASM_TC ||
          d.smoother == SEM_SMOOTH_ASM_TF32) {
        SEM_REQUIRE(Q.L->t.N <= 9, "the Schwarz smoother supports orders up to 9");
        Q.asmd.reset(new AsmData());
        asm_setup(*Q.asmd, *Q.L, Q.dtype == SEM_F32, st);
        if (Q.dtype == SEM_F32)
          Q.asmd->tc = d.smoother == SEM_SMOOTH_ASM_TC ? 1 : d.smoother == SEM_SMOOTH_ASM_TF32 ? 2 : 0;
        if (Q.dtype == SEM_F32) Q.asmd->mr32.alloc(n);
        else Q.asmd->mr64.alloc(n);
      }
      double est = lanczos_lambda_max(*Q.L, P->red, d.lanczos_steps, d.seed, st,
                                      Q.asmd.get());
      Q.lam_hi = 1.1 * est;
      Q.lam_lo = Q.lam_hi / 10.0;
      Q.J.resize((size_t)(d.orders[l] + 1) * (d.orders[l + 1] + 1));
      interpolation_matrix(d.orders[l], d.orders[l + 1], Q.J.data());
    }
  }
  // coarse solve: one persistent kernel at N = 1, launch-based Jacobi-PCG otherwise
  PmgLevel &Cl = *P->levp.back();
  P->persistent_coarse = Cl.L->t.N == 1 && Cl.L->geom == SEM_GEOM_STORED;
  SEM_REQUIRE(d.coarse_mode == SEM_COARSE_JACOBI || d.coarse_mode == SEM_COARSE_MG,
              "unknown coarse_mode %d", d.coarse_mode);
  SEM_REQUIRE(d.coarse_mode == SEM_COARSE_JACOBI || P->persistent_coarse,
              "SEM_COARSE_MG needs a coarsest level of order 1");
  SEM_REQUIRE(d.coarse_ctas >= 0, "coarse_ctas must be >= 0");
  if (P->persistent_coarse) {
    coarse_setup(P->coarse, *Cl.L, st, d.coarse_ctas);
    if (d.coarse_mode == SEM_COARSE_MG) coarse_mg_setup(P->coarse, *Cl.L, st, d.coarse_ctas);
  } else {
    const int64_t nc = Cl.L->t.nl;
    P->cz.alloc(nc); P->cp.alloc(nc); P->cw.alloc(nc);
  }
  P->z64.alloc(F.t.nl);
  SEM_CHECK_CUDA(cudaStreamSynchronize(st));
}

// ------------------------------------------------------------------ V-cycle
// Assembled operator of a smoothed level in its own precision.
template <typename T>
static void level_apply(const PmgLevel &Q, const T *u, T *w, cudaStream_t st) {
  if constexpr (sizeof(T) == 4) {
    if (Q.g16) {
      launch_ax32(*Q.L, Q.g16, u, w, true, st);
      return;
    }
  }
  apply_assembled<T>(*Q.L, u, w, st);
}

// Chebyshev-accelerated Schwarz smoothing (Saad Alg. 12.1 with M in place
// of the Jacobi diagonal; the interval comes from the Lanczos estimate of
// lambda_max(M A)).
template <typename T>
static void smooth_asm(sem_pmg *P, int l, bool x_zero, cudaStream_t st) {
  PmgLevel &Q = (*P->levp[l]);
  const Level &L = *Q.L;
  const int64_t n = L.t.nl;
  T *b = vec_of<T>(Q, 0), *x = vec_of<T>(Q, 1), *r = vec_of<T>(Q, 2), *d = vec_of<T>(Q, 3),
    *w = vec_of<T>(Q, 4);
  T *mr;
  if constexpr (sizeof(T) == 8) mr = Q.asmd->mr64.p;
  else mr = Q.asmd->mr32.p;
  const double theta = 0.5 * (Q.lam_hi + Q.lam_lo), delta = 0.5 * (Q.lam_hi - Q.lam_lo);
  const double sigma = theta / delta;
  double rho = 1.0 / sigma;
  const char *nm = sizeof(T) == 8 ? "cheb_m_f64" : "cheb_m_f32";
  if (x_zero) {
    launch_convert<T, T>(n, b, r, st);
  } else {
    level_apply<T>(Q, x, w, st);
    TraceScope ts(nm, L.t.N, st);
    resid_kernel<T><<<vec_grid(n), kVecThreads, 0, st>>>(n, b, w, r);
    SEM_CHECK_CUDA(cudaGetLastError());
  }
  launch_asm<T>(*Q.asmd, L, r, mr, st);
  {
    TraceScope ts(nm, L.t.N, st);
    cheb_m_kernel<T><<<vec_grid(n), kVecThreads, 0, st>>>(n, mr, d, x, (T)0, (T)(1.0 / theta), 1,
                                                          x_zero);
    SEM_CHECK_CUDA(cudaGetLastError());
  }
  for (int it = 2; it <= P->desc.cheb_degree; ++it) {
    level_apply<T>(Q, d, w, st);
    {
      TraceScope ts(nm, L.t.N, st);
      resid_kernel<T><<<vec_grid(n), kVecThreads, 0, st>>>(n, nullptr, w, r);
      SEM_CHECK_CUDA(cudaGetLastError());
    }
    launch_asm<T>(*Q.asmd, L, r, mr, st);
    const double rho1 = 1.0 / (2.0 * sigma - rho);
    TraceScope ts(nm, L.t.N, st);
    cheb_m_kernel<T><<<vec_grid(n), kVecThreads, 0, st>>>(n, mr, d, x, (T)(rho1 * rho),
                                                          (T)(2.0 * rho1 / delta), 0, 0);
    SEM_CHECK_CUDA(cudaGetLastError());
    rho = rho1;
  }
}

template <typename T>
static void smooth(sem_pmg *P, int l, bool x_zero, cudaStream_t st) {
  PmgLevel &Q = (*P->levp[l]);
  const Level &L = *Q.L;
  if (Q.asmd) {
    smooth_asm<T>(P, l, x_zero, st);
    return;
  }
  const int64_t n = L.t.nl;
  T *b = vec_of<T>(Q, 0), *x = vec_of<T>(Q, 1), *r = vec_of<T>(Q, 2), *d = vec_of<T>(Q, 3),
    *w = vec_of<T>(Q, 4);
  const T *dinv;
  if constexpr (sizeof(T) == 8) dinv = L.dinv64.p;
  else dinv = L.dinv32.p;
  const double theta = 0.5 * (Q.lam_hi + Q.lam_lo), delta = 0.5 * (Q.lam_hi - Q.lam_lo);
  const double sigma = theta / delta;
  double rho = 1.0 / sigma;
  if (!x_zero) level_apply<T>(Q, x, w, st);
  const bool f64 = sizeof(T) == 8;
  const bool v4 = !f64 && n % 4 == 0;
  // from x = 0 with later steps: the start writes d only
  const bool only_d = v4 && x_zero && P->desc.cheb_degree >= 2;
  {
  TraceScope ts(f64 ? "cheb_start_f64" : "cheb_start_f32", L.t.N, st);
  if constexpr (sizeof(T) == 4) {
    if (v4)
      cheb_start4_kernel<<<vec_grid(n / 4), kVecThreads, 0, st>>>(
          n / 4, (const float4 *)b, x_zero ? nullptr : (const float4 *)w, (const float4 *)dinv,
          (float4 *)r, (float4 *)d, (float4 *)x, (float)(1.0 / theta), x_zero, (int)only_d);
  }
  if (!v4)
    cheb_start_kernel<T><<<vec_grid(n), kVecThreads, 0, st>>>(L.t, b, x_zero ? nullptr : w, dinv,
                                                              r, d, x, (T)(1.0 / theta), x_zero);
  SEM_CHECK_CUDA(cudaGetLastError());
  }
  for (int it = 2; it <= P->desc.cheb_degree; ++it) {
    level_apply<T>(Q, d, w, st);
    double rho1 = 1.0 / (2.0 * sigma - rho);
    // r after the last step is dead: the V-cycle forms b - A x for the
    // restriction, and the post-smoothing starts again from b - A x
    const int last = it == P->desc.cheb_degree;
    TraceScope ts(f64 ? "cheb_step_f64" : "cheb_step_f32", L.t.N, st);
    if constexpr (sizeof(T) == 4) {
      if (v4)
        cheb_step4_kernel<<<vec_grid(n / 4), kVecThreads, 0, st>>>(
            n / 4, (const float4 *)w, (const float4 *)dinv, (const float4 *)b, (float4 *)r,
            (float4 *)d, (float4 *)x, (float)(rho1 * rho), (float)(2.0 * rho1 / delta),
            (int)(only_d && it == 2), last);
    }
    if (!v4)
      cheb_step_kernel<T><<<vec_grid(n), kVecThreads, 0, st>>>(
          L.t, w, dinv, r, d, x, (T)(rho1 * rho), (T)(2.0 * rho1 / delta), last);
    SEM_CHECK_CUDA(cudaGetLastError());
    rho = rho1;
  }
}

static TransferParams transfer_params(const PmgLevel &F, const PmgLevel &C) {
  TransferParams tp;
  std::memset(&tp, 0, sizeof(tp));
  tp.tf = F.L->t;
  tp.npf = F.L->t.Np;
  tp.npc = C.L->t.Np;
  std::copy(F.J.begin(), F.J.end(), tp.J);
  return tp;
}

template <typename Tf, typename Tc>
static void restrict_to(sem_pmg *P, int l, cudaStream_t st) {
  PmgLevel &F = (*P->levp[l]), &C = (*P->levp[l + 1]);
  TransferParams tp = transfer_params(F, C);
  size_t shm = sizeof(double) * ((size_t)tp.npf * tp.npf * tp.npf + (size_t)tp.npc * tp.npf * tp.npf +
                                 (size_t)tp.npc * tp.npc * tp.npf);
  {
  TraceScope ts("restrict", F.L->t.N, st);
  const Tf *fb = vec_of<Tf>(F, 0), *fw = vec_of<Tf>(F, 4);
  Tc *co = vec_of<Tc>(C, 0);
  bool done = false;
  auto fast = [&](auto nf, auto nc) {
    constexpr int NF = decltype(nf)::value, NC = decltype(nc)::value;
    if (done || tp.npf != NF || tp.npc != NC) return;
    using S = TrShape<NF>;
    const int64_t g = (tp.tf.E + S::NE - 1) / S::NE;
    restrict_fast_kernel<NF, NC, Tf, Tc>
        <<<(int)std::min<int64_t>(g, 152 * 8), S::THREADS, 0, st>>>(tp, fb, fw, co);
    done = true;
  };
  fast(std::integral_constant<int, 8>(), std::integral_constant<int, 4>());
  fast(std::integral_constant<int, 8>(), std::integral_constant<int, 5>());
  fast(std::integral_constant<int, 5>(), std::integral_constant<int, 3>());
  fast(std::integral_constant<int, 4>(), std::integral_constant<int, 2>());
  fast(std::integral_constant<int, 8>(), std::integral_constant<int, 2>());
  fast(std::integral_constant<int, 6>(), std::integral_constant<int, 4>());
  fast(std::integral_constant<int, 6>(), std::integral_constant<int, 3>());
  fast(std::integral_constant<int, 4>(), std::integral_constant<int, 3>());
  fast(std::integral_constant<int, 3>(), std::integral_constant<int, 2>());
  if (!done)
    restrict_kernel<Tf, Tc><<<grid_elems(tp.tf.E), 128, shm, st>>>(tp, fb, fw, co);
  SEM_CHECK_CUDA(cudaGetLastError());
  }
  // copies summed by the x, y and z face passes, with the Dirichlet mask
  launch_planes_assemble<Tc>(*C.L, vec_of<Tc>(C, 0), st);
}

template <typename Tc, typename Tf>
static void prolong_from(sem_pmg *P, int l, cudaStream_t st) {
  PmgLevel &F = (*P->levp[l]), &C = (*P->levp[l + 1]);
  TransferParams tp = transfer_params(F, C);
  size_t shm = sizeof(double) * ((size_t)tp.npc * tp.npc * tp.npc + (size_t)tp.npf * tp.npc * tp.npc +
                                 (size_t)tp.npf * tp.npf * tp.npc);
  TraceScope ts("prolong", F.L->t.N, st);
  const Tc *cx = vec_of<Tc>(C, 1);
  Tf *fx = vec_of<Tf>(F, 1);
  bool done = false;
  auto fast = [&](auto nf, auto nc) {
    constexpr int NF = decltype(nf)::value, NC = decltype(nc)::value;
    if (done || tp.npf != NF || tp.npc != NC) return;
    using S = TrShape<NF>;
    const int64_t g = (tp.tf.E + S::NE - 1) / S::NE;
    prolong_fast_kernel<NF, NC, Tc, Tf>
        <<<(int)std::min<int64_t>(g, 152 * 8), S::THREADS, 0, st>>>(tp, cx, fx);
    done = true;
  };
  fast(std::integral_constant<int, 8>(), std::integral_constant<int, 4>());
  fast(std::integral_constant<int, 8>(), std::integral_constant<int, 5>());
  fast(std::integral_constant<int, 5>(), std::integral_constant<int, 3>());
  fast(std::integral_constant<int, 4>(), std::integral_constant<int, 2>());
  fast(std::integral_constant<int, 8>(), std::integral_constant<int, 2>());
  fast(std::integral_constant<int, 6>(), std::integral_constant<int, 4>());
  fast(std::integral_constant<int, 6>(), std::integral_constant<int, 3>());
  fast(std::integral_constant<int, 4>(), std::integral_constant<int, 3>());
  fast(std::integral_constant<int, 3>(), std::integral_constant<int, 2>());
  if (!done) prolong_kernel<Tc, Tf><<<grid_elems(tp.tf.E), 128, shm, st>>>(tp, cx, fx);
  SEM_CHECK_CUDA(cudaGetLastError());
}

// Coarsest level: FP64 Jacobi-PCG from zero with a device-side stopping test,
// so the launch sequence is fixed (capturable) and no host round trip occurs.
static void coarse_solve(sem_pmg *P, cudaStream_t st) {
  PmgLevel &Q = (*P->levp.back());
  Level &L = *Q.L;
  if (P->persistent_coarse) {
    if (P->coarse.mg)
      coarse_mg_solve(P->coarse, Q.v64[0].p, Q.v64[1].p, P->desc.coarse_tol, P->desc.coarse_maxit,
                      st);
    else
      coarse_solve_persistent(P->coarse, L, Q.v64[0].p, Q.v64[1].p, P->desc.coarse_tol,
                              P->desc.coarse_maxit, st);
    return;
  }
  const Topo &t = L.t;
  double *b = Q.v64[0].p, *x = Q.v64[1].p, *r = Q.v64[2].p;
  double *z = P->cz.p, *p = P->cp.p, *w = P->cw.p;
  double *sc = P->scal.p;  // 0 bb, 1 rr, 2/3 rho, 4 pw, 5 mean scratch
  int *skip = P->flags.p, *iters = P->flags.p + 1;
  if (t.bc == SEM_NEUMANN) launch_remove_mean(t, P->red, b, sc + 5, st);
  SEM_CHECK_CUDA(cudaMemsetAsync(x, 0, t.nl * sizeof(double), st));
  SEM_CHECK_CUDA(cudaMemsetAsync(skip, 0, 2 * sizeof(int), st));
  launch_cg_start(t, P->red, b, nullptr, L.dinv64.p, r, z, p, sc + 0, sc + 1, sc + 2, st);
  const double tol = P->desc.coarse_tol;
  const double tol2 = tol > 0 ? tol * tol : 0.0;
  const int maxit = P->desc.coarse_maxit;
  launch_stop_test(sc + 1, sc + 0, tol2, 0, maxit, skip, iters, st);
  for (int it = 1; it <= maxit; ++it) {
    const int cur = 2 + ((it - 1) & 1), nxt = 2 + (it & 1);
    launch_ax<double>(L, p, w, st);
    launch_gs<double>(L, w, st);
    launch_mask<double>(L, w, st);
    launch_dot_skip(t, P->red, p, w, sc + 4, skip, st);
    launch_cg_update(t, P->red, sc + cur, sc + 4, p, w, L.dinv64.p, x, r, z, sc + 1, sc + nxt, skip,
                     st);
    launch_stop_test(sc + 1, sc + 0, tol2, it, maxit, skip, iters, st);
    launch_cg_direction(t.nl, sc + nxt, sc + cur, 1.0, z, p, skip, st);
  }
}

// Device bytes held by the hierarchy (the levels it owns, their vectors,
// the Schwarz data, the coarse solver and the reduction buffers).
size_t pmg_device_bytes(const sem_pmg *P) {
  size_t b = P->red.partials.bytes() + P->red.counter.bytes() + P->scal.bytes() +
             P->flags.bytes() + P->cz.bytes() + P->cp.bytes() + P->cw.bytes() + P->z64.bytes();
  for (const auto &q : P->levp) {
    if (!q) continue;
    if (q->own) b += q->own->device_bytes();
    for (int v = 0; v < 5; ++v) b += q->v64[v].bytes() + q->v32[v].bytes();
    if (q->asmd) {
      const AsmData &A = *q->asmd;
      b += A.S64.bytes() + A.lam64.bytes() + A.S32.bytes() + A.lam32.bytes() + A.ext64.bytes() +
           A.ext32.bytes() + A.mr64.bytes() + A.mr32.bytes();
    }
  }
  const CoarseSolver &C = P->coarse;
  b += C.S.bytes() + C.dinv.bytes() + C.vec.bytes() + C.part.bytes() + C.iters.bytes();
  if (C.mg) b += C.mg->fbuf.bytes() + C.mg->ibuf.bytes() + C.mg->kbuf.bytes() + C.mg->part.bytes();
  return b;
}

// The coarsest-level solve alone, on a right-hand side b of that level
// (E-layout, assembled, masked) into x.
void pmg_coarse_solve(sem_pmg *P, const double *b, double *x, cudaStream_t st) {
  PmgLevel &Q = (*P->levp.back());
  const int64_t n = Q.L->t.nl;
  SEM_REQUIRE(Q.v64[0].p && Q.v64[1].p, "coarsest level has no FP64 vectors");
  SEM_CHECK_CUDA(cudaMemcpyAsync(Q.v64[0].p, b, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  coarse_solve(P, st);
  SEM_CHECK_CUDA(cudaMemcpyAsync(x, Q.v64[1].p, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
}

template <typename T, typename Tn>
static void vcycle_level(sem_pmg *P, int l, cudaStream_t st);

template <typename T>
static void vcycle_dispatch(sem_pmg *P, int l, cudaStream_t st) {
  const int last = (int)P->levp.size() - 1;
  if (l == last) {
    coarse_solve(P, st);
    return;
  }
  if ((*P->levp[l + 1]).dtype == SEM_F32) vcycle_level<T, float>(P, l, st);
  else vcycle_level<T, double>(P, l, st);
}

template <typename T, typename Tn>
static void vcycle_level(sem_pmg *P, int l, cudaStream_t st) {
  PmgLevel &Q = (*P->levp[l]);
  smooth<T>(P, l, true, st);
  // residual w = A x (assembled); the restriction forms (b - w) / mult
  level_apply<T>(Q, vec_of<T>(Q, 1), vec_of<T>(Q, 4), st);
  restrict_to<T, Tn>(P, l, st);
  vcycle_dispatch<Tn>(P, l + 1, st);
  prolong_from<Tn, T>(P, l, st);
  smooth<T>(P, l, false, st);
}

VcycleIO pmg_io(sem_pmg *P) {
  PmgLevel &Q = (*P->levp[0]);
  VcycleIO io;
  if (P->levp.size() > 1 && Q.dtype == SEM_F32) {
    io.in32 = Q.v32[0].p;
    io.out32 = Q.v32[1].p;
  } else {
    io.in64 = Q.v64[0].p;
    io.out64 = Q.v64[1].p;
  }
  return io;
}

void pmg_vcycle_core(sem_pmg *P, cudaStream_t st) {
  PmgLevel &Q = (*P->levp[0]);
  if (P->levp.size() == 1) coarse_solve(P, st);  // a single level: the coarse solver itself
  else if (Q.dtype == SEM_F32) vcycle_dispatch<float>(P, 0, st);
  else vcycle_dispatch<double>(P, 0, st);
}

void pmg_vcycle(sem_pmg *P, const double *r, double *z, cudaStream_t st) {
  const int64_t n = P->levp[0]->L->t.nl;
  const VcycleIO io = pmg_io(P);
  if (io.in32) launch_convert<double, float>(n, r, io.in32, st);
  else launch_convert<double, double>(n, r, io.in64, st);
  pmg_vcycle_core(P, st);
  if (io.out32) launch_convert<float, double>(n, io.out32, z, st);
  else launch_convert<double, double>(n, io.out64, z, st);
}

}  // namespace sem
