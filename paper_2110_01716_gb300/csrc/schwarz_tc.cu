// schwarz_tc.cu -- the Schwarz local solves (Sec. 3, Eq. 3: fast
// diagonalisation of each extended element's separable operator) on the
// fifth-generation tensor cores.
//
// An extended element holds n^3 points (n = N + 3 <= 11).  Each of its six
// directional transforms (S^T along x, y, z, then S along z, y, x, with the
// eigenvalue division in the middle) is one product of the n^2 pencils of the
// current direction (the rows, M = 128 with zero rows beyond n^2) by an n x n
// matrix (K = N = 16 with zero padding): a 128 x 16 x 16 tcgen05.mma of kind
// tf32 with FP32 accumulation in tensor memory.  FP32 accuracy comes from the
// split of both operands into a TF32 head and a TF32 remainder
// (a b ~= a_h b_h + a_h b_r + a_r b_h, three products into one accumulator);
// without the split (SPLIT = false) the operands are rounded to TF32 once,
// an element needs half the shared memory and twice as many fit an SM.
// One CTA of 128 threads owns one element at a time: thread p is row p of
// the accumulator; it reads its row back from tensor memory (tcgen05.ld) and
// writes it into shared memory in the layout of the next direction (the
// contracted index becomes K), so the data of an element stays on chip from
// the gather to the final store.  Several CTAs per SM overlap their products.
//
// Shared-memory operands are K-major without swizzle: 8-row core matrices of
// 16 bytes (4 TF32 values) along K, 128 B apart along K and 512 B apart along
// the rows (a 16-wide K slab per 8 rows).
#include <atomic>
#include <cstdint>

#include "common.cuh"
#include "kernels.cuh"
#include "schwarz.cuh"
#include "trace.cuh"

namespace sem {

namespace {

constexpr int kTcThreads = 128;
constexpr int kTile = 8192;                       // one 128 x 16 FP32 operand
constexpr int kMat = 1024;                        // one 16 x 16 FP32 operand
constexpr int kTcWaitLimit = 1 << 22;             // polls of a commit barrier
// Dynamic shared memory: operand A (head, and the remainder with SPLIT), the
// six matrices (heads, and remainders with SPLIT), the eigenvalues, the
// commit barrier and the tensor-memory slot.
template <bool SPLIT>
struct TcLay {
  static constexpr int NA = SPLIT ? 2 : 1, NB = SPLIT ? 12 : 6;
  static constexpr int OFF_A = 0;
  static constexpr int OFF_B = NA * kTile;
  static constexpr int OFF_L = OFF_B + NB * kMat;
  static constexpr int OFF_BAR = OFF_L + 3 * 16 * 4;
  static constexpr int BYTES = OFF_BAR + 16;
};

__device__ __forceinline__ uint32_t su32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// (row, k) -> byte offset in a K-major, no-swizzle, K = 16 operand
__device__ __forceinline__ int toff(int row, int k) {
  return (row >> 3) * 512 + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4;
}

// TF32 rounding (to nearest, ties away) of an FP32 value, as the tensor core
// reads it.
__device__ __forceinline__ float tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// v at (row, k): its TF32 head, and with SPLIT the TF32 remainder
template <bool SPLIT>
__device__ __forceinline__ void put_split(unsigned char *head, unsigned char *rem, int off,
                                          float v) {
  const float h = tf32(v);
  *reinterpret_cast<float *>(head + off) = h;
  if constexpr (SPLIT) *reinterpret_cast<float *>(rem + off) = tf32(v - h);
}

// Shared-memory matrix descriptor: start, leading (K) and stride (rows) byte
// offsets, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16) |
         ((uint64_t)(512u >> 4) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B, both
// K-major, N = 16, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((16u >> 3) << 17) |
                            ((128u >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(kIdesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity) {
  for (int it = 0; it < kTcWaitLimit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int c = 0; c < 16; ++c) v[c] = __uint_as_float(r[c]);
}

}  // namespace

template <int NP, bool SPLIT>
__global__ void __launch_bounds__(kTcThreads)
    asm_solve_tc_kernel(Topo t, const float *__restrict__ S, const float *__restrict__ lam,
                        const float *__restrict__ r, float *__restrict__ z,
                        float *__restrict__ ext, int *err) {
  constexpr int n = NP + 2, n2 = n * n, N = NP - 1, NP2 = NP * NP;
  static_assert(n2 <= 128 && n <= 16, "extended element too large for one 128 x 16 product");
  extern __shared__ __align__(1024) unsigned char smt[];
  using Lay = TcLay<SPLIT>;
  unsigned char *Ah = smt + Lay::OFF_A, *Ar = SPLIT ? Ah + kTile : nullptr;  // A: head, rem.
  unsigned char *Bh = smt + Lay::OFF_B, *Br = SPLIT ? Bh + 6 * kMat : nullptr;  // 6 matrices
  float *sL = reinterpret_cast<float *>(smt + Lay::OFF_L);  // [3][16] eigenvalues
  uint64_t *bar = reinterpret_cast<uint64_t *>(smt + Lay::OFF_BAR);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(smt + Lay::OFF_BAR + 8);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int p = tid;  // accumulator row of this thread

  // zero the operands once: rows >= n^2 and K, N >= n are never written again
  for (int q = tid; q < (Lay::NA * kTile + Lay::NB * kMat) / 4; q += kTcThreads)
    reinterpret_cast<float *>(smt)[q] = 0.f;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(
                     su32(tslot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);  // this warp's 32 lanes
  uint32_t commits = 0;
  bool failed = false;

  for (int64_t e = blockIdx.x; e < t.E && !failed; e += gridDim.x) {
    // S of the three directions: forward matrices (K = point, N = mode) and
    // backward ones (K = mode, N = point); the eigenvalues
    for (int q = tid; q < 3 * n * n; q += kTcThreads) {
      const int d = q / (n * n), a = (q / n) % n, m = q % n;
      const float v = S[e * 3 * n * n + q];
      put_split<SPLIT>(Bh + d * kMat, Br + d * kMat, toff(m, a), v);
      put_split<SPLIT>(Bh + (3 + d) * kMat, Br + (3 + d) * kMat, toff(a, m), v);
    }
    for (int q = tid; q < 3 * n; q += kTcThreads) sL[(q / n) * 16 + q % n] = lam[e * 3 * n + q];
    // gather: row p = (c, b) is the pencil along a (x); extended points
    // outside the element in two directions carry no data
    if (p < n2) {
      const int c = p / n, b = p % n;
      const int ix = (int)(e % t.ex), iy = (int)((e / t.ex) % t.ey),
                iz = (int)(e / ((int64_t)t.ex * t.ey));
      const int64_t exy = (int64_t)t.ex * t.ey;
      const int64_t nxm = ix > 0 ? e - 1 : -1, nxp = ix < t.ex - 1 ? e + 1 : -1;
      const int64_t nym = iy > 0 ? e - t.ex : -1, nyp = iy < t.ey - 1 ? e + t.ex : -1;
      const int64_t nzm = iz > 0 ? e - exy : -1, nzp = iz < t.ez - 1 ? e + exy : -1;
      const int bi = b - 1, ci = c - 1;
      const bool bown = bi >= 0 && bi <= N, cown = ci >= 0 && ci <= N;
#pragma unroll
      for (int a = 0; a < n; ++a) {
        const int ai = a - 1;
        const bool aown = ai >= 0 && ai <= N;
        int64_t src = -1;
        if (aown && bown && cown) {
          src = e * t.Np3 + ai + NP * (bi + NP * ci);
        } else if (!aown && bown && cown) {
          const int64_t f = ai < 0 ? nxm : nxp;
          if (f >= 0) src = f * t.Np3 + (ai < 0 ? N - 1 : 1) + NP * (bi + NP * ci);
        } else if (aown && !bown && cown) {
          const int64_t f = bi < 0 ? nym : nyp;
          if (f >= 0) src = f * t.Np3 + ai + NP * ((bi < 0 ? N - 1 : 1) + NP * ci);
        } else if (aown && bown && !cown) {
          const int64_t f = ci < 0 ? nzm : nzp;
          if (f >= 0) src = f * t.Np3 + ai + NP * (bi + NP * (ci < 0 ? N - 1 : 1));
        }
        put_split<SPLIT>(Ah, Ar, toff(p, a), src >= 0 ? r[src] : 0.f);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();

    // six transforms: x, y, z forward (matrices 0, 1, 2), z, y, x backward (5, 4, 3)
    for (int step = 0; step < 6; ++step) {
      const int mi = step < 3 ? step : 8 - step;
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t ah = su32(Ah), bh = su32(Bh + mi * kMat);
        if constexpr (SPLIT) {
          // remainder products first, the head product last (two K steps each)
          const uint32_t ar = su32(Ar), br = su32(Br + mi * kMat);
          mma_tf32(tmem, sdesc(ah), sdesc(br), 0u);
          mma_tf32(tmem, sdesc(ah + 256), sdesc(br + 256), 1u);
          mma_tf32(tmem, sdesc(ar), sdesc(bh), 1u);
          mma_tf32(tmem, sdesc(ar + 256), sdesc(bh + 256), 1u);
          mma_tf32(tmem, sdesc(ah), sdesc(bh), 1u);
        } else {
          mma_tf32(tmem, sdesc(ah), sdesc(bh), 0u);
        }
        mma_tf32(tmem, sdesc(ah + 256), sdesc(bh + 256), 1u);
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                su32(bar))
            : "memory");
      }
      const bool ok = bar_wait(su32(bar), commits & 1u);
      ++commits;
      if (__syncthreads_or(!ok)) {
        // the product never completed: record it, give it one more bounded
        // wait, and leave (tensor memory is released below)
        if (tid == 0) atomicExch(err, 1);
        bar_wait(su32(bar), (commits - 1) & 1u);
        failed = true;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      float v[16];
      tmem_ld16(trow, v);
      if (p < n2) {
        const int hi = p / n, lo = p % n;
        if (step == 0) {  // row (c, b), columns ma -> rows (c, ma), K = b
#pragma unroll
          for (int m = 0; m < n; ++m) put_split<SPLIT>(Ah, Ar, toff(hi * n + m, lo), v[m]);
        } else if (step == 1) {  // row (c, ma), columns mb -> rows (mb, ma), K = c
#pragma unroll
          for (int m = 0; m < n; ++m) put_split<SPLIT>(Ah, Ar, toff(m * n + lo, hi), v[m]);
        } else if (step == 2) {  // row (mb, ma), columns mc: divide, same rows, K = mc
          const float lxy = sL[lo] + sL[16 + hi];
#pragma unroll
          for (int m = 0; m < n; ++m) put_split<SPLIT>(Ah, Ar, toff(p, m), v[m] / (sL[32 + m] + lxy));
        } else if (step == 3) {  // row (mb, ma), columns c -> rows (c, ma), K = mb
#pragma unroll
          for (int m = 0; m < n; ++m) put_split<SPLIT>(Ah, Ar, toff(m * n + lo, hi), v[m]);
        } else if (step == 4) {  // row (c, ma), columns b -> rows (c, b), K = ma
#pragma unroll
          for (int m = 0; m < n; ++m) put_split<SPLIT>(Ah, Ar, toff(hi * n + m, lo), v[m]);
        } else {  // row (c, b), columns a: own points to z, face layers to ext
          const int c = hi, b = lo;
          const bool bown = b >= 1 && b <= N + 1, cown = c >= 1 && c <= N + 1;
#pragma unroll
          for (int a = 0; a < n; ++a) {
            const bool aown = a >= 1 && a <= N + 1;
            if (aown && bown && cown) {
              z[e * t.Np3 + (a - 1) + NP * ((b - 1) + NP * (c - 1))] = v[a];
            } else if (!aown && bown && cown) {
              ext[(e * 6 + (a == 0 ? 0 : 1)) * NP2 + (b - 1) + NP * (c - 1)] = v[a];
            } else if (aown && !bown && cown) {
              ext[(e * 6 + (b == 0 ? 2 : 3)) * NP2 + (a - 1) + NP * (c - 1)] = v[a];
            } else if (aown && bown && !cown) {
              ext[(e * 6 + (c == 0 ? 4 : 5)) * NP2 + (a - 1) + NP * (b - 1)] = v[a];
            }
          }
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tmem) : "memory");
}

template <int NP, bool SPLIT>
static void asm_tc_np(const AsmData &A, const Level &L, const float *r, float *z, float *ext,
                      cudaStream_t st) {
  auto kern = asm_solve_tc_kernel<NP, SPLIT>;
  constexpr int kSmemTc = TcLay<SPLIT>::BYTES;
  static std::atomic<int> occ[64] = {};
  int dev = 0;
  SEM_CHECK_CUDA(cudaGetDevice(&dev));
  SEM_REQUIRE(dev >= 0 && dev < 64, "device index %d out of range", dev);
  if (!occ[dev]) {
    SEM_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemTc));
    // resident CTAs per SM from the shared-memory and register limits (the
    // occupancy query answers one CTA for this kernel, while the profiler's
    // limits allow seven); 32 tensor-memory columns per CTA allow 16
    int smem_sm = 0, regs_sm = 0;
    SEM_CHECK_CUDA(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    SEM_CHECK_CUDA(cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev));
    cudaFuncAttributes fa{};
    SEM_CHECK_CUDA(cudaFuncGetAttributes(&fa, kern));
    const int by_smem = smem_sm / (kSmemTc + 1024);
    const int by_regs = regs_sm / (fa.numRegs * kTcThreads);
    int o = by_smem < by_regs ? by_smem : by_regs;
    o = o < 16 ? o : 16;
    SEM_REQUIRE(o >= 1, "tensor-core Schwarz kernel does not fit on an SM");
    occ[dev] = o;
  }
  int sms = 0;
  SEM_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int64_t slots = (int64_t)sms * occ[dev];
  const int grid = (int)(L.t.E < slots ? L.t.E : slots);
  kern<<<grid, kTcThreads, kSmemTc, st>>>(L.t, A.S32.p, A.lam32.p, r, z, ext, L.err.p);
  SEM_CHECK_CUDA(cudaGetLastError());
}

template <bool SPLIT>
static void asm_tc_any(const AsmData &A, const Level &L, const float *r, float *z, float *ext,
                       cudaStream_t st) {
  switch (L.t.Np) {
    case 2: asm_tc_np<2, SPLIT>(A, L, r, z, ext, st); break;
    case 3: asm_tc_np<3, SPLIT>(A, L, r, z, ext, st); break;
    case 4: asm_tc_np<4, SPLIT>(A, L, r, z, ext, st); break;
    case 5: asm_tc_np<5, SPLIT>(A, L, r, z, ext, st); break;
    case 6: asm_tc_np<6, SPLIT>(A, L, r, z, ext, st); break;
    case 7: asm_tc_np<7, SPLIT>(A, L, r, z, ext, st); break;
    case 8: asm_tc_np<8, SPLIT>(A, L, r, z, ext, st); break;
    case 9: asm_tc_np<9, SPLIT>(A, L, r, z, ext, st); break;
    default: fail(SEM_EINVAL, "tensor-core Schwarz smoother: order %d unsupported", L.t.N);
  }
}

void launch_asm_solve_tc(const AsmData &A, const Level &L, const float *r, float *z, float *ext,
                         bool split, cudaStream_t st) {
  SEM_REQUIRE(A.S32.p && A.lam32.p && ext && L.err.p, "Schwarz FP32 data were not built");
  if (split) asm_tc_any<true>(A, L, r, z, ext, st);
  else asm_tc_any<false>(A, L, r, z, ext, st);
}

}  // namespace sem
