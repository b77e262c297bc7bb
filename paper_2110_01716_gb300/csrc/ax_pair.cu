// ax_pair.cu -- FP64-accurate stiffness operator evaluated in FP32-pair
// ("double-float") arithmetic.
//
// Same operator as ax.cu (Sec. 2, footnote 1: w^e = sum_d D_d^T sum_f G_df D_f u^e),
// but every value is carried as an unevaluated sum of two
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

#include "pair.cuh"
#include "trace.cuh"

namespace sem {

template <int NP>
static void launch_pair_np(const Level &L, const double *u, double *w, cudaStream_t st) {
  using S = PairShape<NP>;
  int64_t blocks = (L.t.E + S::NE - 1) / S::NE;
  const int64_t cap = 152 * 16;
  int grid = (int)(blocks < 1 ? 1 : (blocks > cap ? cap : blocks));
  auto kern = ax_pair_kernel<NP, false>;
  const size_t shm = sizeof(float2) * (size_t)S::SMEM_PAIRS;
  static std::atomic<bool> attr_set[64] = {};  // per function and device (host threads may race)
  int dev = 0;
  SEM_CHECK_CUDA(cudaGetDevice(&dev));
  if (dev >= 64 || !attr_set[dev]) {
    SEM_CHECK_CUDA(cudaFuncSetAttribute(kern,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    if (dev < 64) attr_set[dev] = true;
  }
  TraceScope ts("ax_f64pair", L.t.N, st);
  kern<<<grid, S::THREADS, shm, st>>>(L.t.E, L.basis, u, w, L.G2.p,
                                                                   PairFuse{});
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
