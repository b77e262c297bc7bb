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

// a + b for pairs: TwoSum of the heads, the tails and its error added,
// without renormalisation.  The error is a few units of 2^-46 of |a| + |b|,
// the same scale as the rounding of the sums it feeds.
__device__ __forceinline__ float2 pair_add_nn(float2 a, float2 b) {
  const float t = __fadd_rn(a.x, b.x);
  const float z = __fsub_rn(t, a.x);
  const float err = __fadd_rn(__fsub_rn(a.x, __fsub_rn(t, z)), __fsub_rn(b.x, z));
  return make_float2(t, __fadd_rn(err, __fadd_rn(a.y, b.y)));
}

__device__ __forceinline__ float2 pair_neg(float2 a) { return make_float2(-a.x, -a.y); }

// A coefficient read from shared memory that the compiler may not merge
// across calls: it would otherwise keep whole coefficient blocks in
// registers between the three directions' applications, and the operator
// runs faster with four CTAs per SM at 64 registers than with two at 128.
__device__ __forceinline__ float2 lds_pair(const float2 *p) {
  float2 r;
  asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];"
               : "=f"(r.x), "=f"(r.y)
               : "r"((unsigned)__cvta_generic_to_shared(p)));
  return r;
}

// v <- M v in place for a centro-antisymmetric NP x NP matrix M
// (M[NP-1-a][NP-1-b] = -M[a][b]; the GLL differentiation matrix and its
// transpose are).  With b' = NP-1-b, H = NP/2, s_b = v_b + v_b' and
// d_b = v_b - v_b' (b < H):
//   ((Mv)_a + (Mv)_a') / 2 = sum_b odd[a][b] d_b,   odd[a][b]  = (M_ab - M_ab') / 2,
//   ((Mv)_a - (Mv)_a') / 2 = sum_b even[a][b] s_b,  even[a][b] = (M_ab + M_ab') / 2,
// with, for odd NP, the extra column even[a][H] = M_a,mid taken against
// v_mid, and the middle row (Mv)_mid = sum_b odd[H][b] d_b.  The NP^2
// products become about NP^2 / 2 plus 2 NP pair additions.  Neither s_b,
// d_b nor the results are renormalised: every consumer (a product, or a
// TwoSum of heads) takes an unnormalised pair, and the tail's own rounding
// stays at the 2^-48 scale of the sums it came from.
// odd is (H + NP%2) x H, even is H x (H + NP%2), both row-major, in shared
// memory.
template <int NP>
__device__ __forceinline__ void pair_apply_eo(const float2 *odd, const float2 *even,
                                              float2 (&v)[NP]) {
  constexpr int H = NP / 2, HO = H + (NP & 1);
  float2 sv[HO], dv[H];
#pragma unroll
  for (int b = 0; b < H; ++b) {
    sv[b] = pair_add_nn(v[b], v[NP - 1 - b]);
    dv[b] = pair_add_nn(v[b], pair_neg(v[NP - 1 - b]));
  }
  if constexpr (HO > H) sv[H] = v[H];
#pragma unroll
  for (int a = 0; a < H; ++a) {
    float ps, pc, ms, mc;
    pair_mul_first(lds_pair(&odd[a * H]), dv[0], ps, pc);
#pragma unroll
    for (int b = 1; b < H; ++b) pair_fma(lds_pair(&odd[a * H + b]), dv[b], ps, pc);
    pair_mul_first(lds_pair(&even[a * HO]), sv[0], ms, mc);
#pragma unroll
    for (int b = 1; b < HO; ++b) pair_fma(lds_pair(&even[a * HO + b]), sv[b], ms, mc);
    v[a] = pair_add_nn(make_float2(ps, pc), make_float2(ms, mc));
    v[NP - 1 - a] = pair_add_nn(make_float2(ps, pc), make_float2(-ms, -mc));
  }
  if constexpr (HO > H) {
    float ps, pc;
    pair_mul_first(lds_pair(&odd[H * H]), dv[0], ps, pc);
#pragma unroll
    for (int b = 1; b < H; ++b) pair_fma(lds_pair(&odd[H * H + b]), dv[b], ps, pc);
    v[H] = make_float2(ps, pc);
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
  // four CTAs (32 warps) per SM at 64 registers up to N = 7; the larger
  // orders keep more registers (and N = 11 its 144-thread CTA alone)
  static constexpr int MIN_CTAS = NP >= 12 ? 1 : NP >= 9 ? 2 : 4;
  // even/odd halves of D and D^T (pair_apply_eo), H x (H + NP%2) pairs each
  static constexpr int NEO = (NP / 2) * (NP / 2 + (NP & 1));
  // dynamic shared memory in float2: the four even/odd blocks, u, W_r, W_s
  static constexpr int SMEM_PAIRS = 4 * NEO + 3 * NE * NP3;
};

// Element-local slot of point (i, j, k) in shared memory.  NP = 8: row
// 8k + (j ^ (k & 1)), column i ^ k, so that each half-warp reads 16
// distinct bank pairs in all three access patterns: column owners (i = 0..7
// with two j), r-line owners (k = 0..7 with two j) and s-line owners
// (i = 0..7 with two k).
template <int NP>
__device__ __forceinline__ int pair_slot(int i, int j, int k) {
  if constexpr (NP == 8) return 64 * k + 8 * (j ^ (k & 1)) + (i ^ k);
  else return i + NP * (j + NP * k);
}

// a + b + c for pairs, one renormalisation.
__device__ __forceinline__ float2 pair_add3(float2 a, float2 b, float2 c) {
  const float t = __fadd_rn(a.x, b.x);
  const float z = __fsub_rn(t, a.x);
  const float e1 = __fadd_rn(__fsub_rn(a.x, __fsub_rn(t, z)), __fsub_rn(b.x, z));
  const float u = __fadd_rn(t, c.x);
  const float y = __fsub_rn(u, t);
  const float e2 = __fadd_rn(__fsub_rn(t, __fsub_rn(u, y)), __fsub_rn(c.x, y));
  return pair_norm(u, __fadd_rn(__fadd_rn(e1, e2), __fadd_rn(__fadd_rn(a.y, b.y), c.y)));
}

// w = A_L u for NE elements per CTA, every contraction through the even/odd
// halves of D or D^T.  Each of an element's NP^2 threads owns one (i,j)
// column (the t-direction, in registers, and the pointwise geometric mix),
// one r-line (fixed j, k) and one s-line (fixed i, k); the line
// contractions run in registers and are exchanged through shared memory:
//  load: the column of u from HBM, split into pairs, into shared memory;
//  A: u_r on the r-line, u_s on the s-line, u_t on the column;
//  B: W = G (u_r, u_s, u_t) at the column's points, G streamed from HBM;
//  C: D^T W_r on the r-line and D^T W_s on the s-line (in place), D^T W_t
//     on the column;
//  sum: the three directions added at the column's points, w to HBM (and,
//     fused form, <u, w> accumulated).
// Four barriers per batch of elements.
template <int NP, bool FUSED>
__global__ void __launch_bounds__(PairShape<NP>::THREADS, PairShape<NP>::MIN_CTAS)
    ax_pair_kernel(int64_t E, Basis bs, const double *__restrict__ u, double *__restrict__ w,
                   const float2 *__restrict__ G2, PairFuse f) {
  using S = PairShape<NP>;
  constexpr int NP2 = S::NP2, NP3 = S::NP3, NE = S::NE, NEO = S::NEO;
  constexpr int H = NP / 2, HO = H + (NP & 1);
  extern __shared__ float2 smem_pair[];
  float2 *sEO = smem_pair;  // D odd, D even, D^T odd, D^T even
  float2(*sU)[NP3] = reinterpret_cast<float2(*)[NP3]>(sEO + 4 * NEO);
  float2(*sR)[NP3] = sU + NE;
  float2(*sS)[NP3] = sR + NE;

  const int le = threadIdx.x / NP2;
  const int ij = threadIdx.x - le * NP2;
  const int lo = ij % NP, hi = ij / NP;
  // column (i, j) = (lo, hi); r-line (j, k) = (hi, lo); s-line (i, k) = (lo, hi)
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
    const float h = (float)d;
    sEO[q] = make_float2(h, (float)(d - (double)h));
  }
  float ds = 0.f, dc = 0.f;  // <u, A_L u> of this thread's points (fused form)
  for (int64_t e0 = (int64_t)blockIdx.x * NE; e0 < E; e0 += (int64_t)gridDim.x * NE) {
    const int64_t e = e0 + le;
    const bool active = e < E;
    {
      // the next batch's u towards L2 while this one computes (G is read
      // one phase later, behind enough warps; prefetching it as well added
      // DRAM traffic and time)
      const int64_t n0 = e0 + (int64_t)gridDim.x * NE;
      if (threadIdx.x == 0 && n0 < E) {
        const int64_t nn = E - n0 < NE ? E - n0 : NE;
        prefetch_l2(u + n0 * NP3, nn * NP3 * (int64_t)sizeof(double));
      }
    }
    float2 rt[NP];
    if (active) {
      const double *ue = u + e * NP3;
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        rt[k] = split_f64(ue[ij + k * NP2]);
        sU[le][pair_slot<NP>(lo, hi, k)] = rt[k];
      }
    }
    __syncthreads();
    if (active) {
      float2 v[NP];
#pragma unroll
      for (int l = 0; l < NP; ++l) v[l] = sU[le][pair_slot<NP>(l, hi, lo)];
      pair_apply_eo<NP>(sEO, sEO + NEO, v);
#pragma unroll
      for (int l = 0; l < NP; ++l) sR[le][pair_slot<NP>(l, hi, lo)] = v[l];
#pragma unroll
      for (int l = 0; l < NP; ++l) v[l] = sU[le][pair_slot<NP>(lo, l, hi)];
      pair_apply_eo<NP>(sEO, sEO + NEO, v);
#pragma unroll
      for (int l = 0; l < NP; ++l) sS[le][pair_slot<NP>(lo, l, hi)] = v[l];
      pair_apply_eo<NP>(sEO, sEO + NEO, rt);
    }
    __syncthreads();
    if (active) {
      const float2 *Ge = G2 + e * 6 * NP3 + ij;
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        float2 g[6];
#pragma unroll
        for (int q = 0; q < 6; ++q) g[q] = __ldg(&Ge[q * NP3 + k * NP2]);
        const int sl = pair_slot<NP>(lo, hi, k);
        const float2 ur = sR[le][sl], us = sS[le][sl], ut = rt[k];
        float a, b;
        pair_mul_first(g[0], ur, a, b); pair_fma(g[1], us, a, b); pair_fma(g[2], ut, a, b);
        sR[le][sl] = make_float2(a, b);
        pair_mul_first(g[1], ur, a, b); pair_fma(g[3], us, a, b); pair_fma(g[4], ut, a, b);
        sS[le][sl] = make_float2(a, b);
        pair_mul_first(g[2], ur, a, b); pair_fma(g[4], us, a, b); pair_fma(g[5], ut, a, b);
        rt[k] = make_float2(a, b);
      }
    }
    __syncthreads();
    if (active) {
      float2 v[NP];
#pragma unroll
      for (int l = 0; l < NP; ++l) v[l] = sR[le][pair_slot<NP>(l, hi, lo)];
      pair_apply_eo<NP>(sEO + 2 * NEO, sEO + 3 * NEO, v);
#pragma unroll
      for (int l = 0; l < NP; ++l) sR[le][pair_slot<NP>(l, hi, lo)] = v[l];
#pragma unroll
      for (int l = 0; l < NP; ++l) v[l] = sS[le][pair_slot<NP>(lo, l, hi)];
      pair_apply_eo<NP>(sEO + 2 * NEO, sEO + 3 * NEO, v);
#pragma unroll
      for (int l = 0; l < NP; ++l) sS[le][pair_slot<NP>(lo, l, hi)] = v[l];
      pair_apply_eo<NP>(sEO + 2 * NEO, sEO + 3 * NEO, rt);
    }
    __syncthreads();
    if (active) {
      // no barrier after this phase: the next batch first writes this
      // thread's own sU slots, and its writes to sR and sS follow the
      // barrier after the load
      double *we = w + e * NP3;
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        const int sl = pair_slot<NP>(lo, hi, k);
        const float2 r = pair_add3(rt[k], sR[le][sl], sS[le][sl]);
        we[ij + k * NP2] = widen_f32(r.x) + widen_f32(r.y);
        if constexpr (FUSED) pair_fma(sU[le][sl], r, ds, dc);
      }
    }
  }
  if constexpr (FUSED) {
    __syncthreads();  // the reduction reuses the start of shared memory
    pair_fused_reduce<S::THREADS>(ds, dc, f, reinterpret_cast<double *>(smem_pair));
  }
}

}  // namespace sem
