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

// (s, c) = a * b for pair values a, b: the first term of a sum, where the
// TwoSum of pair_fma against a zero accumulator would be exact (s = p).
__device__ __forceinline__ void pair_mul_first(float2 a, float2 b, float &s, float &c) {
  const float p = __fmul_rn(a.x, b.x);
  float e = __fmaf_rn(a.x, b.x, -p);
  e = __fmaf_rn(a.x, b.y, e);
  c = __fmaf_rn(a.y, b.x, e);
  s = p;
}

// Renormalise (s, c) into a pair (Fast2Sum; |c| is far below |s| here).
__device__ __forceinline__ float2 pair_norm(float s, float c) {
  const float t = __fadd_rn(s, c);
  return make_float2(t, __fsub_rn(c, __fsub_rn(t, s)));
}

// a + b for pairs: TwoSum of the heads, the tails and its error added, then
// renormalised.  The error is a few units of 2^-46 of |a| + |b|, the same
// scale as the rounding of the sums it feeds.
__device__ __forceinline__ float2 pair_add(float2 a, float2 b) {
  const float t = __fadd_rn(a.x, b.x);
  const float z = __fsub_rn(t, a.x);
  const float err = __fadd_rn(__fsub_rn(a.x, __fsub_rn(t, z)), __fsub_rn(b.x, z));
  return pair_norm(t, __fadd_rn(err, __fadd_rn(a.y, b.y)));
}

__device__ __forceinline__ float2 pair_neg(float2 a) { return make_float2(-a.x, -a.y); }

// v <- M v in place for a centro-antisymmetric NP x NP matrix M
// (M[NP-1-a][NP-1-b] = -M[a][b]; the GLL differentiation matrix and its
// transpose are).  With b' = NP-1-b, H = NP/2, s_b = v_b + v_b' and
// d_b = v_b - v_b' (b < H):
//   ((Mv)_a + (Mv)_a') / 2 = sum_b odd[a][b] d_b,   odd[a][b]  = (M_ab - M_ab') / 2,
//   ((Mv)_a - (Mv)_a') / 2 = sum_b even[a][b] s_b,  even[a][b] = (M_ab + M_ab') / 2,
// with, for odd NP, the extra column even[a][H] = M_a,mid taken against
// v_mid, and the middle row (Mv)_mid = sum_b odd[H][b] d_b.  The NP^2
// products become about NP^2 / 2 plus 2 NP pair additions.
// odd is (H + NP%2) x H, even is H x (H + NP%2), both row-major.
template <int NP>
__device__ __forceinline__ void pair_apply_eo(const float2 *odd, const float2 *even,
                                              float2 (&v)[NP]) {
  constexpr int H = NP / 2, HO = H + (NP & 1);
  float2 sv[HO], dv[H];
#pragma unroll
  for (int b = 0; b < H; ++b) {
    sv[b] = pair_add(v[b], v[NP - 1 - b]);
    dv[b] = pair_add(v[b], pair_neg(v[NP - 1 - b]));
  }
  if constexpr (HO > H) sv[H] = v[H];
#pragma unroll
  for (int a = 0; a < H; ++a) {
    float ps, pc, ms, mc;
    pair_mul_first(odd[a * H], dv[0], ps, pc);
#pragma unroll
    for (int b = 1; b < H; ++b) pair_fma(odd[a * H + b], dv[b], ps, pc);
    pair_mul_first(even[a * HO], sv[0], ms, mc);
#pragma unroll
    for (int b = 1; b < HO; ++b) pair_fma(even[a * HO + b], sv[b], ms, mc);
    v[a] = pair_add(make_float2(ps, pc), make_float2(ms, mc));
    v[NP - 1 - a] = pair_add(make_float2(ps, pc), make_float2(-ms, -mc));
  }
  if constexpr (HO > H) {
    float ps, pc;
    pair_mul_first(odd[H * H], dv[0], ps, pc);
#pragma unroll
    for (int b = 1; b < H; ++b) pair_fma(odd[H * H + b], dv[b], ps, pc);
    v[H] = pair_norm(ps, pc);
  }
}


// The fused form's <u, A_L u>: a deterministic reduction, a fixed-order tree
// in the CTA, one partial per CTA, and the last CTA (ticket) sums the
// partials in CTA order.  red: T doubles of shared memory no thread still
// reads.
template <int T>
__device__ __forceinline__ void pair_fused_reduce(float ds, float dc, const PairFuse &f,
                                                  double *red) {
  constexpr int P2 = T > 128 ? 256 : T > 64 ? 128 : T > 32 ? 64 : 32;
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

template <int NP>
struct PairShape {
  static constexpr int NP2 = NP * NP;
  static constexpr int NP3 = NP2 * NP;
  static constexpr int NE = (256 / NP2) < 1 ? 1 : (256 / NP2);
  static constexpr int THREADS = NE * NP2;
  // two CTAs per SM when the register budget allows (16 warps hide latency)
  static constexpr int MIN_CTAS = THREADS >= 128 ? 2 : 4;
  // even/odd halves of D and D^T (pair_apply_eo), H x (H + NP%2) pairs each
  static constexpr int NEO = (NP / 2) * (NP / 2 + (NP & 1));
  // dynamic shared memory in float2: D, the four even/odd blocks, u, W_r, W_s
  static constexpr int SMEM_PAIRS = NP * (NP + 1) + 4 * NEO + 3 * NE * NP3;
};

// Three phases per element, with one barrier before the last:
//  A: u_r, u_s (shared) and u_t (registers, by the even/odd halves of D) for
//     the whole (i,j) column;
//  B: pointwise geometric mix in place (each thread reads and writes only its
//     own points), G streamed from HBM;
//  C: transposed contractions reading the fluxes of the whole element (the
//     t-direction again by even/odd halves, of D^T, in registers).
// Keeping the fluxes in shared memory instead of registers lets two CTAs
// share an SM.
template <int NP, bool FUSED>
__global__ void __launch_bounds__(PairShape<NP>::THREADS, PairShape<NP>::MIN_CTAS)
    ax_pair_kernel(int64_t E, Basis bs, const double *__restrict__ u, double *__restrict__ w,
                   const float2 *__restrict__ G2, PairFuse f) {
  using S = PairShape<NP>;
  constexpr int NP2 = S::NP2, NP3 = S::NP3, NE = S::NE;
  extern __shared__ float2 smem_pair[];
  constexpr int H = NP / 2, HO = H + (NP & 1), NEO = S::NEO;
  float2(*sD)[NP + 1] = reinterpret_cast<float2(*)[NP + 1]>(smem_pair);
  float2 *sEO = smem_pair + NP * (NP + 1);  // D odd, D even, D^T odd, D^T even
  float2(*sU)[NP3] = reinterpret_cast<float2(*)[NP3]>(sEO + 4 * NEO);
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
  for (int q = threadIdx.x; q < 4 * NEO; q += blockDim.x) {
    const int m = q / NEO, r = q - m * NEO;
    const bool tr = m >= 2, ev = (m & 1) != 0;
    const int cols = ev ? HO : H;
    const int a = r / cols, b = r - a * cols;
    // entry (x, y) of D (tr false) or D^T (tr true)
    auto Dm = [&](int x, int y) { return tr ? bs.D[y * NP + x] : bs.D[x * NP + y]; };
    double d;
    if (!ev) d = 0.5 * (Dm(a, b) - Dm(a, NP - 1 - b));
    else d = b < H ? 0.5 * (Dm(a, b) + Dm(a, NP - 1 - b)) : Dm(a, H);
    const float hi = (float)d;
    sEO[q] = make_float2(hi, (float)(d - (double)hi));
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
      pair_apply_eo<NP>(sEO, sEO + NEO, rt);
      // not unrolled: the whole-kernel unrolling overflowed the instruction
      // cache (no_instruction stalls); this loop alone needs no register
      // array, and rolling it cut a launch by 10 %
#pragma unroll 1
      for (int k = 0; k < NP; ++k) {
        float rs, rc, ss, sc;
        pair_mul_first(sD[i][0], sU[le][j * NP + k * NP2], rs, rc);
        pair_mul_first(sD[j][0], sU[le][i + k * NP2], ss, sc);
#pragma unroll
        for (int l = 1; l < NP; ++l) {
          pair_fma(sD[i][l], sU[le][l + j * NP + k * NP2], rs, rc);
          pair_fma(sD[j][l], sU[le][i + l * NP + k * NP2], ss, sc);
        }
        sR[le][ij + k * NP2] = pair_norm(rs, rc);
        sS[le][ij + k * NP2] = pair_norm(ss, sc);
      }
      // B: W = G (u_r, u_s, u_t), in place
      const float2 *Ge = G2 + e * 6 * NP3 + ij;
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        float2 g[6];
#pragma unroll
        for (int f = 0; f < 6; ++f) g[f] = __ldg(&Ge[f * NP3 + k * NP2]);
        const float2 ur = sR[le][ij + k * NP2], us = sS[le][ij + k * NP2], ut = rt[k];
        float a, b;
        pair_mul_first(g[0], ur, a, b); pair_fma(g[1], us, a, b); pair_fma(g[2], ut, a, b);
        sR[le][ij + k * NP2] = pair_norm(a, b);
        pair_mul_first(g[1], ur, a, b); pair_fma(g[3], us, a, b); pair_fma(g[4], ut, a, b);
        sS[le][ij + k * NP2] = pair_norm(a, b);
        pair_mul_first(g[2], ur, a, b); pair_fma(g[4], us, a, b); pair_fma(g[5], ut, a, b);
        rt[k] = pair_norm(a, b);
      }
    }
    __syncthreads();
    if (active) {
      // C: w = D^T W_r + D^T W_s + D^T W_t, the last term first, in registers
      double *we = w + e * NP3;
      pair_apply_eo<NP>(sEO + 2 * NEO, sEO + 3 * NEO, rt);
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        float s = rt[k].x, c = rt[k].y;
#pragma unroll
        for (int l = 0; l < NP; ++l) {
          pair_fma(sD[l][i], sR[le][l + j * NP + k * NP2], s, c);
          pair_fma(sD[l][j], sS[le][i + l * NP + k * NP2], s, c);
        }
        const float2 r = pair_norm(s, c);
        we[ij + k * NP2] = widen_f32(r.x) + widen_f32(r.y);
        if constexpr (FUSED) pair_fma(sU[le][ij + k * NP2], r, ds, dc);
      }
    }
    __syncthreads();
  }
  if constexpr (FUSED) pair_fused_reduce<S::THREADS>(ds, dc, f, reinterpret_cast<double *>(smem_pair));
}


}  // namespace sem
