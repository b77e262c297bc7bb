// ax32.cu -- FP32 stiffness operator on stored geometric factors (FP32, FP16
// or BF16 storage), with the direct stiffness summation fused in.
//
// Sec. 2, footnote 1: w^e = sum_d D_d^T ( sum_e G_de D_e u^e ); Sec. 3: the
// assembled operator is gs(A_L u) followed by the Dirichlet mask.
//
// Shared-memory traffic, not HBM, limits a straightforward column kernel in
// FP32 (each FMA of the r and s contractions re-reads D and u from shared
// memory).  At N = 7, 4 and 2 (the levels of the smoother) each
// thread owns three lines of its element -- an (i, j) column, an r-line and
// an s-line -- and contracts each whole line in registers through the
// even/odd halves of D, so a line is read from shared memory once for its
// NP outputs (about
// half the shared-memory traffic of the column form; see line_slot for the
// conflict-free layout).  At the other orders each thread owns one (i, j)
// column of an element, loops over k, and
//   * keeps its rows D[i][.], D[j][.] and columns D[.][i], D[.][j] in registers;
//   * reads the contracted u values as float4 from two shared copies of the
//     element: natural (i fastest, for the r contraction) and transposed in
//     (i, j) (j fastest, for the s contraction); rows are padded to an odd
//     number of float4 so the eight rows a warp reads hit distinct banks;
//   * reads D[k][.] and D[.][k] of the t contraction as warp-uniform float4;
//   * keeps u and the t flux of its column in registers.
//
// Direct stiffness summation on the box is separable: summing the copies of
// every shared node across x-faces, then across y-faces, then across z-faces
// yields the full sum over all copies (a node shared by 2, 4 or 8 elements is
// summed as a + b, (a + b) + (c + d), ...; every copy receives the same bits).
// A CTA walks a segment of an x-line of elements in chunks of NE elements, so
// the x-face sums of neighbouring elements happen in shared memory; the right
// face of a chunk's last element waits in shared memory for the next chunk.
// Faces where segments meet (seams; only when the box has too few x-lines to
// fill the GPU) are summed by a small seam pass.  Two plane passes then sum
// across y-faces and z-faces; face planes normal to y and z are rows of NP
// contiguous values, so these passes move whole sectors.  Dirichlet masking is
// done by the pass of each boundary's direction: a masked node's copies all lie
// on that boundary plane, so later passes only add zeros.
#include <algorithm>
#include <cmath>
#include <atomic>
#include <cstring>
#include <type_traits>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"
#include "kernels.cuh"
#include "trace.cuh"

namespace sem {

// Shared-memory wavefronts per 8-lane phase of the float4 row reads of the
// unstaged kernel (rows of one plane: row j for the natural copy, row i for
// the transposed one), averaged over a CTA, for element stride es (floats).
constexpr double row_read_waves(int NP, int NE, int RS, int es) {
  const int T = NE * NP * NP;
  double tot = 0.0;
  int phases = 0;
  for (int pat = 0; pat < 2; ++pat)
    for (int c = 0; c < (NP + 3) / 4; ++c)
      for (int g0 = 0; g0 < T; g0 += 8) {
        int addr[8] = {}, n = 0;
        for (int t = g0; t < g0 + 8 && t < T; ++t) {
          const int le = t / (NP * NP), ij = t % (NP * NP), i = ij % NP, j = ij / NP;
          const int a = le * es + (pat == 0 ? j : i) * RS + 4 * c;
          bool seen = false;
          for (int q = 0; q < n; ++q) seen = seen || addr[q] == a;
          if (!seen) addr[n++] = a;
        }
        int worst = 0;
        for (int b = 0; b < 8; ++b) {  // 16-byte bank groups of a 128-byte row
          int m = 0;
          for (int q = 0; q < n; ++q) m += ((addr[q] / 4) % 8) == b;
          worst = m > worst ? m : worst;
        }
        tot += worst;
        ++phases;
      }
  return tot / phases;
}
// The element stride (floats, a whole number of float4, at least NP planes)
// with the fewest wavefronts; the first such stride above the minimum.
constexpr int best_element_stride(int NP, int NE, int RS) {
  const int base = NP * NP * RS;
  int best = base;
  double bw = row_read_waves(NP, NE, RS, base);
  for (int es = base + 4; es < base + 32; es += 4) {
    const double w = row_read_waves(NP, NE, RS, es);
    if (w < bw) {
      bw = w;
      best = es;
    }
  }
  return best;
}

// Element stride (floats) of the line form's shared copies (see line_slot).
constexpr int line_stride_of(int NP) { return NP == 8 ? 512 : NP == 5 ? 153 : NP == 3 ? 41 : 0; }

template <int NP>
struct A32 {
  static constexpr int NP2 = NP * NP;
  static constexpr int NP3 = NP2 * NP;
  // elements per CTA: two at N = 7 (128 threads, four CTAs per SM) and five
  // at N = 4 (125 threads, six per SM) measured faster than four and ten at
  // 48^3 (0.336 -> 0.322 and 0.107 -> 0.104 ms per launch); one at N = 7 was
  // slower (0.331)
#ifndef SEM_AX32_NE8
#define SEM_AX32_NE8 2
#endif
#ifndef SEM_AX32_NE5
#define SEM_AX32_NE5 5
#endif
  static constexpr int NE = NP == 8 ? SEM_AX32_NE8 : NP == 5 ? SEM_AX32_NE5
                          : (256 / NP2) < 1 ? 1 : (256 / NP2);
  static constexpr int THREADS = NE * NP2;
  static constexpr int C4 = (NP + 3) / 4;                            // float4 per row
  static constexpr int RS = (C4 % 2 == 0) ? 4 * C4 + 4 : 4 * C4;     // padded row stride
  static constexpr int PL = NP * RS;                                 // padded plane stride
#ifndef SEM_AX32_ES_SEARCH
#define SEM_AX32_ES_SEARCH 1
#endif
  // padded element: for the unstaged orders the stride whose rows a warp
  // reads across two neighbouring elements fall in distinct bank groups
  // (measured at 48^3: N = 4 0.144 -> 0.139 ms, N = 2 0.040 -> 0.036 ms)
  static constexpr int ES = (NP % 4 != 0 && SEM_AX32_ES_SEARCH)
                                ? best_element_stride(NP, NE, RS)
                                : (((NP * PL / 4) % 2 == 0) ? NP * PL + 4 : NP * PL);
  // element stride of the shared regions: the column form's, or the line
  // form's where that is larger
  static constexpr int ESB = ES < line_stride_of(NP) ? line_stride_of(NP) : ES;
  // Staged variant (NP a multiple of 4): natural-order arrays keep unpadded
  // rows (a warp reads at most four rows of one element, or of two elements
  // 16 banks apart); the element's u and factors arrive by bulk copy.
  static constexpr bool STAGED = NP % 4 == 0;
  static constexpr int ESN = NP3 + (NP2 < 32 ? 16 : 0);              // natural element stride
#ifndef SEM_AX32_MIN_CTAS
#define SEM_AX32_MIN_CTAS 2
#endif
#ifndef SEM_AX32_GPRE
#define SEM_AX32_GPRE 1
#endif
  // unstaged small orders: the element column's factors are loaded into
  // registers with u, before the barrier, so no load waits inside the k loop
  // (measured at 48^3: N = 4 0.139 -> 0.131 ms per launch; at N = 2 slower)
  static constexpr bool GPRE = !STAGED && NP == 5 && SEM_AX32_GPRE;
  // the unstaged small orders fit 64 registers (four CTAs, 32 warps per SM),
  // 80 with the factors in registers (three CTAs)
  static constexpr int MIN_CTAS =
      NP == 8 && NE <= 2 ? 8 / NE : NP == 5 && NE == 5 ? 6
      : !STAGED && NP <= 5 ? (GPRE ? 3 : 4) : (NP <= 8 ? SEM_AX32_MIN_CTAS : 1);
};

constexpr int round16(int b) { return (b + 15) & ~15; }

// Shared-memory layout (bytes) of one CTA.
template <int NP, int GK>
struct L32 {
  using S = A32<NP>;
  static constexpr int GB = GK == 0 ? 4 : 2;                          // bytes per factor
  static constexpr int U_BYTES = S::NE * S::NP3 * 4;                  // one stage of u
  static constexpr int G_BYTES = S::NE * 6 * S::NP3 * GB;             // one stage of factors
#ifndef SEM_AX32_STAGE_F32G
#define SEM_AX32_STAGE_F32G 0
#endif
  // factors staged in shared memory too (else read from global, L2-prefetched)
  static constexpr bool SG = S::STAGED && (GK != 0 || SEM_AX32_STAGE_F32G);
#ifndef SEM_AX32_F32G_SINGLE
#define SEM_AX32_F32G_SINGLE 1
#endif
  // FP32 factors in one stage of their own, refilled for the next chunk as
  // soon as the gradient phase has read them (two CTAs per SM still fit)
  static constexpr bool SGS = S::STAGED && !SG && GK == 0 && SEM_AX32_F32G_SINGLE;
  static constexpr int STAGE = round16(U_BYTES) + (SG ? round16(G_BYTES) : 0);
  static constexpr int MBAR = 0;                                      // 3 x 8 bytes
  static constexpr int STAGES = 32;
  static constexpr int STAGES_END = S::STAGED ? STAGES + 2 * STAGE : STAGES;
  static constexpr int GSTAGE = STAGES_END;                           // single factor stage
  static constexpr int GSTAGE_END = GSTAGE + (SGS ? round16(G_BYTES) : 0);
  static constexpr int DTAB = GSTAGE_END;                             // sD, sDT
  static constexpr int UN = DTAB + round16(2 * NP * S::RS * 4);       // direct: padded natural u
  static constexpr int UN_END = S::STAGED ? UN : UN + S::NE * S::ES * 4;
  static constexpr int UT = UN_END;                                   // transposed u
  static constexpr int WR = UT + S::NE * S::ESB * 4;                  // natural r flux
  static constexpr int WR_END = WR + S::NE * (S::STAGED ? S::ESN : S::ESB) * 4;
  static constexpr int WS = WR_END;                                   // transposed s flux
  static constexpr int FACES = WS + S::NE * S::ESB * 4;               // sFL, sFR, sCarry
  static constexpr int BYTES = FACES + (2 * S::NE + 2) * S::NP2 * 4;
};

// Factor value from its stored bits (GK: 0 FP32, 1 FP16, 2 BF16).
template <int GK>
__device__ __forceinline__ float factor_value(float v) { return v; }
template <int GK>
__device__ __forceinline__ float factor_value(unsigned short b) {
  if constexpr (GK == 1) return __half2float(__ushort_as_half(b));
  else return __bfloat162float(__ushort_as_bfloat16(b));
}
template <int GK>
using factor_t = typename std::conditional<GK == 0, float, unsigned short>::type;

__device__ __forceinline__ float f4get(const float4 &v, int q) {
  return q == 0 ? v.x : (q == 1 ? v.y : (q == 2 ? v.z : v.w));
}

// NP values of a 16-byte aligned shared row into registers.
template <int NP>
__device__ __forceinline__ void load_row(const float *row, float (&r)[NP]) {
#pragma unroll
  for (int c = 0; c < (NP + 3) / 4; ++c) {
    const float4 v = *reinterpret_cast<const float4 *>(row + 4 * c);
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (4 * c + q < NP) r[4 * c + q] = f4get(v, q);
  }
}

// ---- mbarrier and bulk-copy primitives (CTA scope)
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
// Bounded wait for the phase with the given parity; false if it never came.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int limit) {
  for (int it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
// Global -> shared bulk copy (16-byte aligned addresses, size a multiple of 16)
// that completes its bytes on the mbarrier.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes,
                                         uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

constexpr int kMbarWaitLimit = 1 << 22;  // try_wait polls before a wait is declared lost

struct Ax32Args {
  Topo t;
  const float *u;
  float *w;
  const void *G;       // [E][6][NP3] float or 16-bit
  const float *scale;  // [E] per-element scale of 16-bit factors, else null
  int32_t nseg;        // segments per x-line
  int32_t seg_len;     // elements per segment (the last may be shorter)
  int32_t dirichlet;
  int *err;            // set to 1 if a bulk copy never completed
};

// First element (x index) of work unit `unit`.
__device__ __forceinline__ int unit_ix0(const Ax32Args &a, int64_t unit) {
  return (int)(unit % a.nseg) * a.seg_len;
}

// Line form (N = 7 and N = 4): each of an element's NP^2 threads owns an
// (i,j) column (t-direction and the pointwise mix), an r-line (j,k) and an
// s-line (i,k), and applies each contraction to a whole line in registers
// through the even/odd halves of D.  A line is read from shared memory once
// for its NP outputs, where the column form re-reads a row for every output.
//
// Element-local slot of (i,j,k) and element stride of the line buffers.
// NP = 8: 64k + 32(j/4) + 8((j + k) mod 4) + (i ^ k); its bank,
// 8((j + k) mod 4) + (i ^ k), is distinct across a warp for column owners
// (i = 0..7, four j), r-line owners (k = 0..7, four j) and s-line owners
// (i = 0..7, four k).  NP = 5 (25 threads per element, warps straddle
// elements): i + 5j + 26k with elements 153 floats apart, the layout with
// the fewest wavefronts per warp access (1.6 on average, at most 2) found by
// enumerating row, plane and element strides.  NP = 3 likewise: i + 3j + 11k,
// elements 41 floats apart (1.7 wavefronts per access, at most 2).
template <int NP>
__device__ __forceinline__ int line_slot(int i, int j, int k) {
  if constexpr (NP == 8) return 64 * k + 32 * (j >> 2) + 8 * ((j + k) & 3) + (i ^ k);
  else if constexpr (NP == 5) return i + 5 * j + 26 * k;
  else return i + 3 * j + 11 * k;
}
template <int NP>
constexpr int line_stride() { return line_stride_of(NP); }

// v <- M v for a centro-antisymmetric NP x NP matrix M (the GLL D and D^T)
// from its halves in registers: with b' = NP-1-b and H = NP/2,
// od[a][b] = (M_ab - M_ab') / 2 ((H + NP%2) x H) and ev[a][b] =
// (M_ab + M_ab') / 2 (H x (H + NP%2), for odd NP the last column M_a,mid):
// (Mv)_a = P + Q, (Mv)_a' = P - Q with P = sum_b od[a][b] (v_b - v_b') and
// Q = sum_b ev[a][b] (v_b + v_b') (v_mid alone in the last column); for odd
// NP the middle row is sum_b od[H][b] (v_b - v_b').
template <int NP>
__device__ __forceinline__ void eo_apply(const float (&od)[(NP / 2) * (NP / 2 + (NP & 1))],
                                         const float (&ev)[(NP / 2) * (NP / 2 + (NP & 1))],
                                         float (&v)[NP]) {
  constexpr int H = NP / 2, HO = H + (NP & 1);
  float sv[HO], dv[H];
#pragma unroll
  for (int b = 0; b < H; ++b) {
    sv[b] = v[b] + v[NP - 1 - b];
    dv[b] = v[b] - v[NP - 1 - b];
  }
  if constexpr (HO > H) sv[H] = v[H];
#pragma unroll
  for (int a = 0; a < H; ++a) {
    float p = od[a * H] * dv[0], q = ev[a * HO] * sv[0];
#pragma unroll
    for (int b = 1; b < H; ++b) p = fmaf(od[a * H + b], dv[b], p);
#pragma unroll
    for (int b = 1; b < HO; ++b) q = fmaf(ev[a * HO + b], sv[b], q);
    v[a] = p + q;
    v[NP - 1 - a] = p - q;
  }
  if constexpr (HO > H) {
    float p = od[H * H] * dv[0];
#pragma unroll
    for (int b = 1; b < H; ++b) p = fmaf(od[H * H + b], dv[b], p);
    v[H] = p;
  }
}

// n floats of shared memory into registers (warp-uniform addresses).
template <int n>
__device__ __forceinline__ void load_coef(const float *p, float (&r)[n]) {
#pragma unroll
  for (int q = 0; q < n; ++q) r[q] = p[q];
}

template <int NP, int GK, bool ASSEMBLE>
__global__ void __launch_bounds__(A32<NP>::THREADS, A32<NP>::MIN_CTAS)
    ax32_kernel(Ax32Args a, Basis bs) {
  using S = A32<NP>;
  using Lay = L32<NP, GK>;
  using GT = factor_t<GK>;
  constexpr int NP2 = S::NP2, NP3 = S::NP3, NE = S::NE, RS = S::RS, PL = S::PL, ES = S::ES;
  constexpr int C4 = S::C4, N = NP - 1;
  constexpr bool STAGED = S::STAGED;
  extern __shared__ float4 smem4[];
  unsigned char *smem = reinterpret_cast<unsigned char *>(smem4);
  uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + Lay::MBAR);
  float *sD = reinterpret_cast<float *>(smem + Lay::DTAB);  // [NP][RS]  D[k][l]
  float *sDT = sD + NP * RS;                                // [NP][RS]  D[l][k]
  float *sU = reinterpret_cast<float *>(smem + Lay::UN);    // direct: padded natural u
  float *sUT = reinterpret_cast<float *>(smem + Lay::UT);
  float *sWR = reinterpret_cast<float *>(smem + Lay::WR);
  float *sWS = reinterpret_cast<float *>(smem + Lay::WS);
  float *sFL = reinterpret_cast<float *>(smem + Lay::FACES);  // [NE][NP2] left faces (i = 0)
  float *sFR = sFL + NE * NP2;                                // [NE][NP2] right faces (i = N)
  float *sCarry = sFR + NE * NP2;                             // [2][NP2]  deferred right face

  const int le = threadIdx.x / NP2;
  const int ij = threadIdx.x - le * NP2;
  const int i = ij % NP, j = ij / NP;
  constexpr bool LINES = (STAGED && NP == 8) || (!STAGED && (NP == 5 || NP == 3));
  constexpr int LH = NP / 2, LHO = LH + (NP & 1), NEO = LH * LHO;
  if constexpr (LINES) {
    // even/odd halves of D (od, ev) and of D^T (odT, evT), NEO floats each
    for (int q = threadIdx.x; q < 4 * NEO; q += blockDim.x) {
      const int m = q / NEO, r = q - m * NEO;
      const bool tr = m >= 2, ev = (m & 1) != 0;
      const int cols = ev ? LHO : LH;
      const int a = r / cols, b = r - a * cols;
      auto Dm = [&](int x, int y) { return tr ? bs.D[y * NP + x] : bs.D[x * NP + y]; };
      double v;
      if (!ev) v = 0.5 * (Dm(a, b) - Dm(a, NP - 1 - b));
      else v = b < LH ? 0.5 * (Dm(a, b) + Dm(a, NP - 1 - b)) : Dm(a, LH);
      sD[q] = (float)v;
    }
  } else {
    for (int q = threadIdx.x; q < NP * RS; q += blockDim.x) {
      const int r = q / RS, l = q % RS;
      sD[q] = l < NP ? bs.D32[r * NP + l] : 0.f;
      sDT[q] = l < NP ? bs.D32[l * NP + r] : 0.f;
    }
  }
  if (STAGED && threadIdx.x == 0) {
    mbar_init(smem_addr(&mbar[0]), 1);
    mbar_init(smem_addr(&mbar[1]), 1);
    mbar_init(smem_addr(&mbar[2]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();

  const Topo &t = a.t;
  const int64_t units = (int64_t)t.ey * t.ez * a.nseg;
  // natural-order views of this thread's element (rows along i)
  constexpr int NRS = STAGED ? NP : RS, NPL = STAGED ? NP2 : PL;
  float *uT = sUT + le * ES, *wS = sWS + le * ES;
  float *wR = sWR + le * (STAGED ? S::ESN : ES);

  // Bulk copies of a chunk's u and factors into stage `st`.
  auto issue = [&](int64_t unit, int cx, int st) {
    const int ix1 = min(t.ex, unit_ix0(a, unit) + a.seg_len);
    const int n = min(NE, ix1 - cx);
    const int64_t e0 = (unit / a.nseg) * t.ex + cx;
    const uint32_t ub = (uint32_t)(n * NP3 * 4), gb = (uint32_t)(n * 6 * NP3 * Lay::GB);
    unsigned char *dst = smem + Lay::STAGES + st * Lay::STAGE;
    const uint32_t bar = smem_addr(&mbar[st]);
    mbar_expect_tx(bar, ub + (Lay::SG ? gb : 0));
    bulk_g2s(smem_addr(dst), a.u + e0 * NP3, ub, bar);
    if (Lay::SG)
      bulk_g2s(smem_addr(dst + round16(Lay::U_BYTES)),
               static_cast<const unsigned char *>(a.G) + e0 * 6 * NP3 * Lay::GB, gb, bar);
    else if (!Lay::SGS)
      prefetch_l2(static_cast<const unsigned char *>(a.G) + e0 * 6 * NP3 * Lay::GB, gb);
  };
  // Bulk copy of a chunk's FP32 factors into the single factor stage.
  auto issue_g = [&](int64_t unit, int cx) {
    const int ix1 = min(t.ex, unit_ix0(a, unit) + a.seg_len);
    const int n = min(NE, ix1 - cx);
    const int64_t e0 = (unit / a.nseg) * t.ex + cx;
    const uint32_t gb = (uint32_t)(n * 6 * NP3 * Lay::GB);
    const uint32_t bar = smem_addr(&mbar[2]);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(bar, gb);
    bulk_g2s(smem_addr(smem + Lay::GSTAGE),
             static_cast<const unsigned char *>(a.G) + e0 * 6 * NP3 * Lay::GB, gb, bar);
  };

  int64_t unit = blockIdx.x;
  int cx = unit < units ? unit_ix0(a, unit) : 0;
  uint32_t g = 0;  // chunks done by this CTA (stage g & 1, phase parity (g >> 1) & 1)
  if (STAGED && threadIdx.x == 0 && unit < units) {
    issue(unit, cx, 0);
    if constexpr (Lay::SGS) issue_g(unit, cx);
  }

  while (unit < units) {
    const int64_t line = unit / a.nseg;
    const int ix0 = unit_ix0(a, unit);
    const int ix1 = min(t.ex, ix0 + a.seg_len);
    const int cc = (cx - ix0) / NE;
    const int nact = min(NE, ix1 - cx);
    const bool active = le < nact;
    const int ix = cx + le;
    const int64_t e = line * t.ex + ix;
    // the next chunk: in this segment, else the first of the next unit
    int64_t nunit = unit;
    int ncx = cx + NE;
    if (ncx >= ix1) {
      nunit = unit + gridDim.x;
      ncx = nunit < units ? unit_ix0(a, nunit) : 0;
    }
    const float *stU = nullptr;
    const GT *stG = nullptr;
    if constexpr (STAGED) {
      if (threadIdx.x == 0 && nunit < units) issue(nunit, ncx, (g + 1) & 1);
      bool ok = mbar_wait(smem_addr(&mbar[g & 1]), (g >> 1) & 1, kMbarWaitLimit);
      if constexpr (Lay::SGS) ok = mbar_wait(smem_addr(&mbar[2]), g & 1, kMbarWaitLimit) && ok;
      if (__syncthreads_or(!ok)) {
        // a copy never completed: record it, let copies in flight land, stop
        if (threadIdx.x == 0) {
          atomicExch(a.err, 1);
          mbar_wait(smem_addr(&mbar[g & 1]), (g >> 1) & 1, kMbarWaitLimit);
          if (nunit < units) mbar_wait(smem_addr(&mbar[(g + 1) & 1]), ((g + 1) >> 1) & 1,
                                       kMbarWaitLimit);
          if (Lay::SGS) mbar_wait(smem_addr(&mbar[2]), g & 1, kMbarWaitLimit);
        }
        __syncthreads();
        return;
      }
      const unsigned char *stage = smem + Lay::STAGES + (g & 1) * Lay::STAGE;
      stU = reinterpret_cast<const float *>(stage) + le * NP3;
      if constexpr (Lay::SGS) stG = reinterpret_cast<const GT *>(smem + Lay::GSTAGE) + le * 6 * NP3;
      else stG = reinterpret_cast<const GT *>(stage + round16(Lay::U_BYTES)) + le * 6 * NP3;
    } else if (threadIdx.x == 0 && nunit < units) {
      const int64_t ne0 = (nunit / a.nseg) * t.ex + ncx;
      const int nn = min(NE, min(t.ex, unit_ix0(a, nunit) + a.seg_len) - ncx);
      prefetch_l2(a.u + ne0 * NP3, (int64_t)nn * NP3 * 4);
      prefetch_l2(static_cast<const unsigned char *>(a.G) + ne0 * 6 * NP3 * Lay::GB,
                  (int64_t)nn * 6 * NP3 * Lay::GB);
    }
    const float *uN = STAGED ? stU : sU + le * ES;

    if constexpr (LINES) {
      constexpr int LS = line_stride<NP>();
      float *sUs = reinterpret_cast<float *>(smem + Lay::UT) + le * LS;
      float *sR = reinterpret_cast<float *>(smem + Lay::WR) + le * LS;
      float *sS = reinterpret_cast<float *>(smem + Lay::WS) + le * LS;
      // column (i, j); r-line (j, k) = (j, i); s-line (i, k) = (i, j)
      float ru[NP];
      float gpre[S::GPRE ? 6 : 1][S::GPRE ? NP : 1];
      if (active) {
        const float *ue = a.u + e * NP3 + ij;
#pragma unroll
        for (int k = 0; k < NP; ++k) {
          const float v = STAGED ? stU[k * NP2 + ij] : __ldg(ue + k * NP2);
          ru[k] = v;
          sUs[line_slot<NP>(i, j, k)] = v;
        }
        if constexpr (S::GPRE) {
          const GT *Gg = static_cast<const GT *>(a.G) + e * 6 * NP3 + ij;
#pragma unroll
          for (int f = 0; f < 6; ++f)
#pragma unroll
            for (int k = 0; k < NP; ++k) gpre[f][k] = factor_value<GK>(__ldg(Gg + f * NP3 + k * NP2));
        }
      }
      __syncthreads();
      // ---- gradients: u_r on the r-line, u_s on the s-line, u_t on the column
      if (active) {
        float od[NEO], ev[NEO], v[NP];
        load_coef(sD, od);
        load_coef(sD + NEO, ev);
#pragma unroll
        for (int l = 0; l < NP; ++l) v[l] = sUs[line_slot<NP>(l, j, i)];
        eo_apply<NP>(od, ev, v);
#pragma unroll
        for (int l = 0; l < NP; ++l) sR[line_slot<NP>(l, j, i)] = v[l];
#pragma unroll
        for (int l = 0; l < NP; ++l) v[l] = sUs[line_slot<NP>(i, l, j)];
        eo_apply<NP>(od, ev, v);
#pragma unroll
        for (int l = 0; l < NP; ++l) sS[line_slot<NP>(i, l, j)] = v[l];
        eo_apply<NP>(od, ev, ru);
      }
      __syncthreads();
      // ---- geometric factors at the column's points, in place
      if (active) {
#pragma unroll
        for (int k = 0; k < NP; ++k) {
          const int sl = line_slot<NP>(i, j, k);
          const float ur = sR[sl], us = sS[sl], ut = ru[k];
          float g6[6];
#pragma unroll
          for (int f = 0; f < 6; ++f) {
            if constexpr (Lay::SG || Lay::SGS) g6[f] = factor_value<GK>(stG[f * NP3 + k * NP2 + ij]);
            else if constexpr (S::GPRE) g6[f] = gpre[f][k];
            else g6[f] = factor_value<GK>(__ldg(static_cast<const GT *>(a.G) + e * 6 * NP3 +
                                                f * NP3 + k * NP2 + ij));
          }
          sR[sl] = g6[0] * ur + g6[1] * us + g6[2] * ut;
          sS[sl] = g6[1] * ur + g6[3] * us + g6[4] * ut;
          ru[k] = g6[2] * ur + g6[4] * us + g6[5] * ut;
        }
      }
      __syncthreads();
      // the factor stage is free: bring in the next chunk's factors
      if constexpr (Lay::SGS)
        if (threadIdx.x == 0 && nunit < units) issue_g(nunit, ncx);
      // ---- divergence: D^T on the r-line and the s-line (in place), on the column
      if (active) {
        float od[NEO], ev[NEO], v[NP];
        load_coef(sD + 2 * NEO, od);
        load_coef(sD + 3 * NEO, ev);
#pragma unroll
        for (int l = 0; l < NP; ++l) v[l] = sR[line_slot<NP>(l, j, i)];
        eo_apply<NP>(od, ev, v);
#pragma unroll
        for (int l = 0; l < NP; ++l) sR[line_slot<NP>(l, j, i)] = v[l];
#pragma unroll
        for (int l = 0; l < NP; ++l) v[l] = sS[line_slot<NP>(i, l, j)];
        eo_apply<NP>(od, ev, v);
#pragma unroll
        for (int l = 0; l < NP; ++l) sS[line_slot<NP>(i, l, j)] = v[l];
        eo_apply<NP>(od, ev, ru);
      }
      __syncthreads();
      if (active) {
        const float sc = GK == 0 ? 1.f : __ldg(a.scale + e);
        float *we = a.w + e * NP3 + ij;
#pragma unroll
        for (int k = 0; k < NP; ++k) {
          const int sl = line_slot<NP>(i, j, k);
          float acc = (sR[sl] + sS[sl]) + ru[k];
          if (GK != 0) acc *= sc;
          if (!ASSEMBLE || (i != 0 && i != N)) we[k * NP2] = acc;
          else if (i == 0) sFL[le * NP2 + k * NP + j] = acc;
          else sFR[le * NP2 + k * NP + j] = acc;
        }
      }
    } else {
      // ---- u: registers along k, transposed copy (and padded natural copy)
      float ru[NP];
      if (active) {
        if constexpr (STAGED) {
  #pragma unroll
          for (int k = 0; k < NP; ++k) {
            const float v = stU[k * NP2 + ij];
            ru[k] = v;
            uT[k * PL + i * RS + j] = v;
          }
        } else {
          const float *ue = a.u + e * NP3 + ij;
  #pragma unroll
          for (int k = 0; k < NP; ++k) {
            const float v = __ldg(ue + k * NP2);
            ru[k] = v;
            sU[le * ES + k * PL + j * RS + i] = v;
            uT[k * PL + i * RS + j] = v;
          }
        }
      }
      float gpre[S::GPRE ? 6 : 1][S::GPRE ? NP : 1];
      if constexpr (S::GPRE) {
        const GT *Gg = static_cast<const GT *>(a.G) + (active ? e : 0) * 6 * NP3 + ij;
  #pragma unroll
        for (int f = 0; f < 6; ++f)
  #pragma unroll
          for (int k = 0; k < NP; ++k)
            gpre[f][k] = active ? factor_value<GK>(__ldg(Gg + f * NP3 + k * NP2)) : 0.f;
      }
      __syncthreads();
      // ---- gradients, geometric factors, fluxes
      float wt[NP];
      if (active) {
        float Dr[NP], Ds[NP];
        load_row<NP>(sD + i * RS, Dr);
        load_row<NP>(sD + j * RS, Ds);
        const GT *Gg = static_cast<const GT *>(a.G) + e * 6 * NP3 + ij;
  #pragma unroll
        for (int k = 0; k < NP; ++k) {
          // two partial sums per contraction (even and odd l) halve the chains
          float ur2[2] = {0.f, 0.f}, us2[2] = {0.f, 0.f}, ut2[2] = {0.f, 0.f};
          const float *pa = uN + k * NPL + j * NRS, *pb = uT + k * PL + i * RS, *pd = sD + k * RS;
  #pragma unroll
          for (int c = 0; c < C4; ++c) {
            const float4 va = *reinterpret_cast<const float4 *>(pa + 4 * c);
            const float4 vb = *reinterpret_cast<const float4 *>(pb + 4 * c);
            const float4 vd = *reinterpret_cast<const float4 *>(pd + 4 * c);
  #pragma unroll
            for (int q = 0; q < 4; ++q) {
              const int l = 4 * c + q;
              if (l < NP) {
                ur2[q & 1] = fmaf(Dr[l], f4get(va, q), ur2[q & 1]);
                us2[q & 1] = fmaf(Ds[l], f4get(vb, q), us2[q & 1]);
                ut2[q & 1] = fmaf(f4get(vd, q), ru[l], ut2[q & 1]);
              }
            }
          }
          const float ur = ur2[0] + ur2[1], us = us2[0] + us2[1], ut = ut2[0] + ut2[1];
          float g6[6];
  #pragma unroll
          for (int f = 0; f < 6; ++f) {
            if constexpr (Lay::SG || Lay::SGS) g6[f] = factor_value<GK>(stG[f * NP3 + k * NP2 + ij]);
            else if constexpr (S::GPRE) g6[f] = gpre[f][k];
            else g6[f] = factor_value<GK>(__ldg(Gg + f * NP3 + k * NP2));
          }
          wR[k * NPL + j * NRS + i] = g6[0] * ur + g6[1] * us + g6[2] * ut;
          wS[k * PL + i * RS + j] = g6[1] * ur + g6[3] * us + g6[4] * ut;
          wt[k] = g6[2] * ur + g6[4] * us + g6[5] * ut;
        }
      }
      __syncthreads();
      // the factor stage is free: bring in the next chunk's factors
      if constexpr (Lay::SGS)
        if (threadIdx.x == 0 && nunit < units) issue_g(nunit, ncx);
      // ---- divergence: w = scale * (D_r^T wr + D_s^T ws + D_t^T wt)
      if (active) {
        float DTr[NP], DTs[NP];
        load_row<NP>(sDT + i * RS, DTr);
        load_row<NP>(sDT + j * RS, DTs);
        const float sc = GK == 0 ? 1.f : __ldg(a.scale + e);
        float *we = a.w + e * NP3 + ij;
  #pragma unroll
        for (int k = 0; k < NP; ++k) {
          // one partial sum per direction (three independent chains)
          float ar = 0.f, as = 0.f, at = 0.f;
          const float *pa = wR + k * NPL + j * NRS, *pb = wS + k * PL + i * RS, *pd = sDT + k * RS;
  #pragma unroll
          for (int c = 0; c < C4; ++c) {
            const float4 va = *reinterpret_cast<const float4 *>(pa + 4 * c);
            const float4 vb = *reinterpret_cast<const float4 *>(pb + 4 * c);
            const float4 vd = *reinterpret_cast<const float4 *>(pd + 4 * c);
  #pragma unroll
            for (int q = 0; q < 4; ++q) {
              const int l = 4 * c + q;
              if (l < NP) {
                ar = fmaf(DTr[l], f4get(va, q), ar);
                as = fmaf(DTs[l], f4get(vb, q), as);
                at = fmaf(f4get(vd, q), wt[l], at);
              }
            }
          }
          float acc = (ar + as) + at;
          if (GK != 0) acc *= sc;
          if (!ASSEMBLE || (i != 0 && i != N)) we[k * NP2] = acc;
          else if (i == 0) sFL[le * NP2 + k * NP + j] = acc;
          else sFR[le * NP2 + k * NP + j] = acc;
        }
      }
    }
    if constexpr (ASSEMBLE) {
      __syncthreads();
      // ---- x-face sums (lower-x copy + upper-x copy), masks, carries: one
      // thread per node of the chunk's left faces, then of its last right face
      for (int q = threadIdx.x; q < NE * NP2; q += blockDim.x) {
        const int l2 = q / NP2, jk = q - l2 * NP2;  // jk = k * NP + j
        if (l2 >= nact) continue;
        const int ix2 = cx + l2;
        const int jj = jk % NP, kk = jk / NP;
        float *wl = a.w + (line * t.ex + ix2) * NP3 + kk * NP2 + jj * NP;  // i = 0
        const float own = sFL[q];
        if (l2 > 0 || cx > ix0) {
          const float left = l2 > 0 ? sFR[q - NP2] : sCarry[((cc - 1) & 1) * NP2 + jk];
          const float v = left + own;
          wl[0] = v;
          wl[N - NP3] = v;  // element e - 1, i = N
        } else {
          wl[0] = (ix2 == 0 && a.dirichlet) ? 0.f : own;  // box boundary or seam
        }
      }
      for (int q = threadIdx.x; q < NP2; q += blockDim.x) {
        const int ix2 = cx + nact - 1;
        const float own = sFR[(nact - 1) * NP2 + q];
        if (ix2 == ix1 - 1) {  // box boundary or seam
          const int jj = q % NP, kk = q / NP;
          a.w[(line * t.ex + ix2) * NP3 + kk * NP2 + jj * NP + N] =
              (ix2 == t.ex - 1 && a.dirichlet) ? 0.f : own;
        } else {
          sCarry[(cc & 1) * NP2 + q] = own;  // summed by the next chunk
        }
      }
    }
    unit = nunit;
    cx = ncx;
    ++g;
  }
}

// Seams: x-faces where two segments of a line meet (lower + upper copy).
__global__ void ax32_seam_kernel(Topo t, int nseg, int seg_len, float *__restrict__ w) {
  const int Np = t.Np, Np2 = Np * Np;
  const int64_t seams = (int64_t)t.ey * t.ez * (nseg - 1);
  const int64_t total = seams * Np2;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = q / Np2;
    const int jk = (int)(q - s * Np2);
    const int64_t line = s / (nseg - 1);
    const int part = (int)(s - line * (nseg - 1)) + 1;
    const int64_t e = line * t.ex + (int64_t)part * seg_len;
    float *hi = w + e * t.Np3 + (int64_t)jk * Np;  // i = 0 of the upper element
    float *lo = hi - t.Np3 + (Np - 1);             // i = N of the lower element
    const float v = *lo + *hi;
    *lo = v;
    *hi = v;
  }
}

static int sm_count() {
  static std::atomic<int> n[64] = {};  // per device; host threads may race to fill it
  int dev = 0;
  SEM_CHECK_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return 152;
  if (!n[dev]) {
    int v = 0;
    SEM_CHECK_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev));
    n[dev] = v;
  }
  return n[dev];
}

// Resident CTAs per SM of one kernel instantiation (queried once per device;
// sets the dynamic shared-memory limit on the way).
template <int NP, int GK, bool ASSEMBLE>
static int ax32_resident() {
  static std::atomic<int> res[64] = {};  // per device; filling it twice is harmless
  int dev = 0;
  SEM_CHECK_CUDA(cudaGetDevice(&dev));
  SEM_REQUIRE(dev >= 0 && dev < 64, "device index %d out of range", dev);
  if (!res[dev]) {
    auto kern = ax32_kernel<NP, GK, ASSEMBLE>;
    constexpr int bytes = L32<NP, GK>::BYTES;
    SEM_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    int r = 0;
    SEM_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, kern, A32<NP>::THREADS, bytes));
    SEM_REQUIRE(r >= 1, "operator kernel does not fit on an SM");
    res[dev] = r;
  }
  return res[dev];
}

template <int NP, int GK>
static void ax32_np(const Level &L, const float *u, float *w, bool assemble, cudaStream_t st) {
  using S = A32<NP>;
  const Topo &t = L.t;
  Ax32Args a;
  a.t = t;
  a.u = u;
  a.w = w;
  const int s = GK == 2 ? 1 : 0;
  a.G = GK == 0 ? (const void *)L.G32.p : (const void *)L.G16[s].p;
  a.scale = GK == 0 ? nullptr : L.G16scale[s].p;
  a.err = L.err.p;
  SEM_REQUIRE(a.G != nullptr, "stored factors of this precision were not built");
  SEM_REQUIRE(a.err != nullptr, "level has no error flag");
  if (S::STAGED)
    SEM_REQUIRE(reinterpret_cast<uintptr_t>(u) % 16 == 0 && reinterpret_cast<uintptr_t>(a.G) % 16 == 0,
                "u must be 16-byte aligned");
  a.dirichlet = t.bc == SEM_DIRICHLET;
  const int resident = assemble ? ax32_resident<NP, GK, true>() : ax32_resident<NP, GK, false>();
  const int64_t slots = (int64_t)sm_count() * resident;
  // Work units are x-line segments: whole lines when there are at least two
  // per resident CTA (no seams), otherwise lines are split.
  const int64_t lines = (int64_t)t.ey * t.ez;
  const double fill = L.ax32_fill > 0.f ? (double)L.ax32_fill : 2.0;
  const int64_t target = std::max<int64_t>(1, (int64_t)std::ceil(fill * (double)slots));
  const int64_t cap = std::min<int64_t>(slots, target);
  int nseg = 1;
  if (lines < target) {
    const int64_t want = (target + lines - 1) / lines;
    const int64_t most = (t.ex + S::NE - 1) / S::NE;  // at least one chunk per segment
    nseg = (int)(want < most ? want : most);
    if (nseg < 1) nseg = 1;
  }
  a.seg_len = (t.ex + nseg - 1) / nseg;
  a.nseg = (t.ex + a.seg_len - 1) / a.seg_len;
  const int64_t units = lines * a.nseg;
  const int grid = (int)(units < cap ? units : cap);  // persistent: every CTA resident
  constexpr int bytes = L32<NP, GK>::BYTES;
  static const char *names[3][2] = {{"ax32_f32", "ax32_f32_local"},
                                    {"ax32_f16g", "ax32_f16g_local"},
                                    {"ax32_bf16g", "ax32_bf16g_local"}};
  {
    TraceScope ts(names[GK][assemble ? 0 : 1], t.N, st);
    if (assemble) ax32_kernel<NP, GK, true><<<grid, S::THREADS, bytes, st>>>(a, L.basis);
    else ax32_kernel<NP, GK, false><<<grid, S::THREADS, bytes, st>>>(a, L.basis);
    SEM_CHECK_CUDA(cudaGetLastError());
  }
  if (!assemble) return;
  SEM_REQUIRE((uint64_t)t.E * t.Np * t.Np < (1ull << 32), "mesh too large for the plane passes");
  TraceScope ts("plane_sum", t.N, st, a.nseg > 1 ? 3 : 2);
  if (a.nseg > 1) {
    const int64_t n = lines * (a.nseg - 1) * t.Np * t.Np;
    const int64_t b = (n + 255) / 256;
    ax32_seam_kernel<<<(int)(b < 152 * 8 ? b : 152 * 8), 256, 0, st>>>(t, a.nseg, a.seg_len, w);
    SEM_CHECK_CUDA(cudaGetLastError());
  }
  launch_plane_pass(t, 1, w, a.dirichlet, st);
  launch_plane_pass(t, 2, w, a.dirichlet, st);
}


template <int GK>
static void ax32_dispatch(const Level &L, const float *u, float *w, bool assemble,
                          cudaStream_t st) {
  switch (L.t.Np) {
    case 2: ax32_np<2, GK>(L, u, w, assemble, st); break;
    case 3: ax32_np<3, GK>(L, u, w, assemble, st); break;
    case 4: ax32_np<4, GK>(L, u, w, assemble, st); break;
    case 5: ax32_np<5, GK>(L, u, w, assemble, st); break;
    case 6: ax32_np<6, GK>(L, u, w, assemble, st); break;
    case 7: ax32_np<7, GK>(L, u, w, assemble, st); break;
    case 8: ax32_np<8, GK>(L, u, w, assemble, st); break;
    case 9: ax32_np<9, GK>(L, u, w, assemble, st); break;
    case 10: ax32_np<10, GK>(L, u, w, assemble, st); break;
    case 11: ax32_np<11, GK>(L, u, w, assemble, st); break;
    case 12: ax32_np<12, GK>(L, u, w, assemble, st); break;
    default: fail(SEM_EINVAL, "unsupported order N=%d", L.t.N);
  }
}

// FP32 operator on stored factors: kind SEM_F32 (float factors), SEM_F16 or
// SEM_BF16 (16-bit factors); assemble: w = mask * gs(A_L u), else w = A_L u.
void launch_ax32(const Level &L, int kind, const float *u, float *w, bool assemble,
                 cudaStream_t st) {
  SEM_REQUIRE(L.geom == SEM_GEOM_STORED, "launch_ax32 needs stored geometry");
  if (kind == SEM_F32) ax32_dispatch<0>(L, u, w, assemble, st);
  else if (kind == SEM_F16) ax32_dispatch<1>(L, u, w, assemble, st);
  else if (kind == SEM_BF16) ax32_dispatch<2>(L, u, w, assemble, st);
  else fail(SEM_EINVAL, "launch_ax32: unknown kind %d", kind);
}

}  // namespace sem
