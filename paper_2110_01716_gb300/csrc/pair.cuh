// pair.cuh -- FP32-pair ("double-float") arithmetic and the FP64-accurate
// stiffness operator built on it (see ax_pair.cu for the method).  The kernel
// has a plain form (u -> A_L u) and a form that also reduces <u, A_L u> over
// the local points (ax_pair_fused.cu), which for a continuous (and, under
// Dirichlet, masked) u equals <u, mask gs(A_L u)> over the unique points: the
// inner product of a CG iteration without a pass of its own.
#pragma once

#include "common.cuh"
#include "kernels.cuh"

namespace sem {

// d ~= hi + lo with |d - hi - lo| <= 2^-46 |d|; values below 2^-80 in
// magnitude lose lo (they are far below anything the operator can resolve),
// values outside the float range become 0, NaN/Inf propagate through hi.
__device__ __forceinline__ float2 split_f64(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned int hw = (unsigned int)(b >> 32), lw = (unsigned int)b;
  const unsigned int sign = hw & 0x80000000u;
  const int E = (int)((hw >> 20) & 0x7FF);
  float hi = 0.0f, lo = 0.0f;
  if (E >= 897 && E <= 1150) {
    hi = __uint_as_float(sign | ((unsigned int)(E - 896) << 23) | ((hw & 0xFFFFFu) << 3) |
                         (lw >> 29));
    if (E >= 943) {
      const unsigned int R = (lw & 0x1FFFFFFFu) >> 6;              // next 23 bits
      const float fr = __fsub_rn(__uint_as_float(0x4B000000u | R), 8388608.0f);  // = R exactly
      const float sc = __uint_as_float((unsigned int)(E - 942) << 23);          // 2^(E-1069)
      lo = __uint_as_float(__float_as_uint(__fmul_rn(fr, sc)) | sign);
    }
  } else if (E == 2047) {
    hi = __uint_as_float(sign | 0x7F800000u | (hw & 0xFFFFFu ? 0x400000u : 0u));
  }
  return make_float2(hi, lo);
}

// s + c += a * b for pair values a, b.
__device__ __forceinline__ void pair_fma(float2 a, float2 b, float &s, float &c) {
  const float p = __fmul_rn(a.x, b.x);
  float e = __fmaf_rn(a.x, b.x, -p);
  e = __fmaf_rn(a.x, b.y, e);
  e = __fmaf_rn(a.y, b.x, e);
  const float t = __fadd_rn(s, p);
  const float z = __fsub_rn(t, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
  s = t;
  c = __fadd_rn(c, __fadd_rn(err, e));
}

// Renormalise (s, c) into a pair (Fast2Sum; |c| is far below |s| here).
__device__ __forceinline__ float2 pair_norm(float s, float c) {
  const float t = __fadd_rn(s, c);
  return make_float2(t, __fsub_rn(c, __fsub_rn(t, s)));
}


template <int NP>
struct PairShape {
  static constexpr int NP2 = NP * NP;
  static constexpr int NP3 = NP2 * NP;
  static constexpr int NE = (256 / NP2) < 1 ? 1 : (256 / NP2);
  static constexpr int THREADS = NE * NP2;
  // two CTAs per SM when the register budget allows (16 warps hide latency)
  static constexpr int MIN_CTAS = THREADS >= 128 ? 2 : 4;
};

// Three phases per element, with one barrier before the last:
//  A: u_r, u_s (shared) and u_t (registers) for the whole (i,j) column;
//  B: pointwise geometric mix in place (each thread reads and writes only its
//     own points), G streamed from HBM;
//  C: transposed contractions reading the fluxes of the whole element.
// Keeping the fluxes in shared memory instead of registers lets two CTAs
// share an SM.
template <int NP, bool FUSED>
__global__ void __launch_bounds__(PairShape<NP>::THREADS, PairShape<NP>::MIN_CTAS)
    ax_pair_kernel(int64_t E, Basis bs, const double *__restrict__ u, double *__restrict__ w,
                   const float2 *__restrict__ G2, PairFuse f) {
  using S = PairShape<NP>;
  constexpr int NP2 = S::NP2, NP3 = S::NP3, NE = S::NE;
  extern __shared__ float2 smem_pair[];
  float2(*sD)[NP + 1] = reinterpret_cast<float2(*)[NP + 1]>(smem_pair);
  float2(*sU)[NP3] = reinterpret_cast<float2(*)[NP3]>(smem_pair + NP * (NP + 1));
  float2(*sR)[NP3] = sU + NE;
  float2(*sS)[NP3] = sR + NE;

  const int le = threadIdx.x / NP2;
  const int ij = threadIdx.x - le * NP2;
  const int i = ij % NP, j = ij / NP;
  for (int q = threadIdx.x; q < NP * NP; q += blockDim.x) {
    const double d = bs.D[q];
    const float hi = (float)d;
    sD[q / NP][q % NP] = make_float2(hi, (float)(d - (double)hi));
  }
  float ds = 0.f, dc = 0.f;  // <u, A_L u> of this thread's points (fused form)
  for (int64_t e0 = (int64_t)blockIdx.x * NE; e0 < E; e0 += (int64_t)gridDim.x * NE) {
    const int64_t e = e0 + le;
    const bool active = e < E;
    {
      // the next batch of this CTA towards L2 while this one computes
      const int64_t n0 = e0 + (int64_t)gridDim.x * NE;
      if (threadIdx.x == 0 && n0 < E) {
        const int64_t nn = E - n0 < NE ? E - n0 : NE;
        prefetch_l2(G2 + n0 * 6 * NP3, nn * 6 * NP3 * (int64_t)sizeof(float2));
        prefetch_l2(u + n0 * NP3, nn * NP3 * (int64_t)sizeof(double));
      }
    }
    float2 rt[NP];
    if (active) {
      const double *ue = u + e * NP3;
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        rt[k] = split_f64(ue[ij + k * NP2]);
        sU[le][ij + k * NP2] = rt[k];
      }
    }
    __syncthreads();
    if (active) {
      // A: reference gradients; u_t overwrites the column of u in registers
      float ts[NP], tc[NP];
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        ts[k] = 0.f;
        tc[k] = 0.f;
#pragma unroll
        for (int l = 0; l < NP; ++l) pair_fma(sD[k][l], rt[l], ts[k], tc[k]);
      }
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        float rs = 0.f, rc = 0.f, ss = 0.f, sc = 0.f;
#pragma unroll
        for (int l = 0; l < NP; ++l) {
          pair_fma(sD[i][l], sU[le][l + j * NP + k * NP2], rs, rc);
          pair_fma(sD[j][l], sU[le][i + l * NP + k * NP2], ss, sc);
        }
        sR[le][ij + k * NP2] = pair_norm(rs, rc);
        sS[le][ij + k * NP2] = pair_norm(ss, sc);
        rt[k] = pair_norm(ts[k], tc[k]);
      }
      // B: W = G (u_r, u_s, u_t), in place
      const float2 *Ge = G2 + e * 6 * NP3 + ij;
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        float2 g[6];
#pragma unroll
        for (int f = 0; f < 6; ++f) g[f] = __ldg(&Ge[f * NP3 + k * NP2]);
        const float2 ur = sR[le][ij + k * NP2], us = sS[le][ij + k * NP2], ut = rt[k];
        float a = 0.f, b = 0.f;
        pair_fma(g[0], ur, a, b); pair_fma(g[1], us, a, b); pair_fma(g[2], ut, a, b);
        sR[le][ij + k * NP2] = pair_norm(a, b);
        a = 0.f; b = 0.f;
        pair_fma(g[1], ur, a, b); pair_fma(g[3], us, a, b); pair_fma(g[4], ut, a, b);
        sS[le][ij + k * NP2] = pair_norm(a, b);
        a = 0.f; b = 0.f;
        pair_fma(g[2], ur, a, b); pair_fma(g[4], us, a, b); pair_fma(g[5], ut, a, b);
        rt[k] = pair_norm(a, b);
      }
    }
    __syncthreads();
    if (active) {
      // C: w = D^T W_r + D^T W_s + D^T W_t
      double *we = w + e * NP3;
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        float s = 0.f, c = 0.f;
#pragma unroll
        for (int l = 0; l < NP; ++l) {
          pair_fma(sD[l][i], sR[le][l + j * NP + k * NP2], s, c);
          pair_fma(sD[l][j], sS[le][i + l * NP + k * NP2], s, c);
          pair_fma(sD[l][k], rt[l], s, c);
        }
        const float2 r = pair_norm(s, c);
        we[ij + k * NP2] = widen_f32(r.x) + widen_f32(r.y);
        if constexpr (FUSED) pair_fma(sU[le][ij + k * NP2], r, ds, dc);
      }
    }
    __syncthreads();
  }
  if constexpr (FUSED) {
    // deterministic reduction: a fixed-order tree in the CTA, one partial per
    // CTA, and the last CTA (ticket) sums the partials in CTA order
    constexpr int T = S::THREADS;
    constexpr int P2 = T > 128 ? 256 : T > 64 ? 128 : T > 32 ? 64 : 32;
    double *red = reinterpret_cast<double *>(smem_pair);
    __shared__ bool last;
    const int tid = threadIdx.x;
    red[tid] = widen_f32(ds) + widen_f32(dc);
    __syncthreads();
#pragma unroll
    for (int h = P2 / 2; h > 0; h >>= 1) {
      if (tid < h && tid + h < T) red[tid] += red[tid + h];
      __syncthreads();
    }
    if (tid == 0) {
      f.partials[blockIdx.x] = red[0];
      __threadfence();
      last = atomicAdd(f.counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double x = 0.0;
    for (int b = tid; b < (int)gridDim.x; b += T) x += __ldcg(&f.partials[b]);
    red[tid] = x;
    __syncthreads();
#pragma unroll
    for (int h = P2 / 2; h > 0; h >>= 1) {
      if (tid < h && tid + h < T) red[tid] += red[tid + h];
      __syncthreads();
    }
    if (tid == 0) {
      *f.pw = red[0];
      *f.counter = 0u;
    }
  }
}

}  // namespace sem
