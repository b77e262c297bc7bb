// ax_pair.cu -- FP64-accurate stiffness operator evaluated in FP32-pair
// ("double-float") arithmetic.
//
// Same operator as ax.cu (Sec. 2, footnote 1: w^e = sum_d D_d^T sum_f G_df D_f u^e),
// same thread layout, but every value is carried as an unevaluated sum of two
// floats (hi + lo, about 48 significant bits) and every multiply-add is
// error-free-transformed on the FP32 pipes:
//   product  p = fl(a_hi b_hi),  e = fma(a_hi, b_hi, -p)  (exact error, Ogita-Rump-Oishi)
//            e += a_hi b_lo + a_lo b_hi                     (cross terms)
//   sum      TwoSum(s, p) -> (s', err)  (Knuth), c += err + e.
// On GB300 the FP64 pipe issues about 2 FMA per clock per SM against 128 FP32
// FMA, so twelve FP32 instructions per multiply-add still run about 5x faster
// than one native FP64 FMA.  Relative error of one operator application stays
// near 2^-46 of the largest partial sums.
//
// FP64 inputs are split into (hi, lo) with integer instructions only (the
// FP64<->FP32 conversion instructions issue at the FP64 rate on this part):
// hi is the value truncated to 24 significant bits, lo the next 23 bits.
// The result is rebuilt from its float pair with integer instructions and one
// FP64 addition.  Geometric factors are stored pre-split (float2, 8 bytes).
#include <atomic>

#include "common.cuh"
#include "trace.cuh"

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
template <int NP>
__global__ void __launch_bounds__(PairShape<NP>::THREADS, PairShape<NP>::MIN_CTAS)
    ax_pair_kernel(int64_t E, Basis bs, const double *__restrict__ u, double *__restrict__ w,
                   const float2 *__restrict__ G2) {
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

  for (int64_t e0 = (int64_t)blockIdx.x * NE; e0 < E; e0 += (int64_t)gridDim.x * NE) {
    const int64_t e = e0 + le;
    const bool active = e < E;
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
      }
    }
    __syncthreads();
  }
}

template <int NP>
static void launch_pair_np(const Level &L, const double *u, double *w, cudaStream_t st) {
  using S = PairShape<NP>;
  int64_t blocks = (L.t.E + S::NE - 1) / S::NE;
  const int64_t cap = 152 * 16;
  int grid = (int)(blocks < 1 ? 1 : (blocks > cap ? cap : blocks));
  const size_t shm = sizeof(float2) * ((size_t)NP * (NP + 1) + 3 * (size_t)S::NE * S::NP3);
  static std::atomic<bool> attr_set[64] = {};  // per function and device (host threads may race)
  int dev = 0;
  SEM_CHECK_CUDA(cudaGetDevice(&dev));
  if (dev >= 64 || !attr_set[dev]) {
    SEM_CHECK_CUDA(cudaFuncSetAttribute(ax_pair_kernel<NP>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    if (dev < 64) attr_set[dev] = true;
  }
  TraceScope ts("ax_f64pair", L.t.N, st);
  ax_pair_kernel<NP><<<grid, S::THREADS, shm, st>>>(L.t.E, L.basis, u, w, L.G2.p);
  SEM_CHECK_CUDA(cudaGetLastError());
}

void launch_ax_pair(const Level &L, const double *u, double *w, cudaStream_t st) {
  SEM_REQUIRE(L.G2.p != nullptr, "pair-split geometric factors were not built");
  switch (L.t.Np) {
    case 2: launch_pair_np<2>(L, u, w, st); break;
    case 3: launch_pair_np<3>(L, u, w, st); break;
    case 4: launch_pair_np<4>(L, u, w, st); break;
    case 5: launch_pair_np<5>(L, u, w, st); break;
    case 6: launch_pair_np<6>(L, u, w, st); break;
    case 7: launch_pair_np<7>(L, u, w, st); break;
    case 8: launch_pair_np<8>(L, u, w, st); break;
    case 9: launch_pair_np<9>(L, u, w, st); break;
    case 10: launch_pair_np<10>(L, u, w, st); break;
    case 11: launch_pair_np<11>(L, u, w, st); break;
    case 12: launch_pair_np<12>(L, u, w, st); break;
    default: fail(SEM_EINVAL, "unsupported order N=%d", L.t.N);
  }
}

}  // namespace sem
