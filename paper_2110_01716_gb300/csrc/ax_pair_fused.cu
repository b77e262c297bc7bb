// ax_pair_fused.cu -- the FP64-accurate (FP32-pair) operator with the inner
// product of the CG iteration (Sec. 3) folded in: w = A_L p and <p, A_L p>
// in one pass.  For a continuous p (masked under Dirichlet) the local sum
// equals <p, mask gs(A_L p)> over unique points, so the separate pass over
// p and w that the inner product would take is saved.  (Forming the
// direction p = z + beta p in the same pass was measured slower: this
// kernel's time grows with the bytes it moves, at well under the HBM rate.)
#include <atomic>

#include "pair.cuh"
#include "trace.cuh"

namespace sem {

template <int NP>
static void launch_fused_np(const Level &L, const double *u, double *w, const PairFuse &f,
                            cudaStream_t st) {
  using S = PairShape<NP>;
  int64_t blocks = (L.t.E + S::NE - 1) / S::NE;
  const int64_t cap = 152 * 16;
  int grid = (int)(blocks < 1 ? 1 : (blocks > cap ? cap : blocks));
  auto kern = ax_pair_kernel<NP, true>;
  const size_t shm = sizeof(float2) * (size_t)S::SMEM_PAIRS;
  static std::atomic<bool> attr_set[64] = {};
  int dev = 0;
  SEM_CHECK_CUDA(cudaGetDevice(&dev));
  if (dev >= 64 || !attr_set[dev]) {
    SEM_CHECK_CUDA(cudaFuncSetAttribute(kern,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    if (dev < 64) attr_set[dev] = true;
  }
  TraceScope ts("ax_f64pair", L.t.N, st);
  kern<<<grid, S::THREADS, shm, st>>>(L.t.E, L.basis, u, w, L.G2.p, f);
  SEM_CHECK_CUDA(cudaGetLastError());
}

int pair_fused_grid(const Level &L) {
  int64_t ne = 1;
  switch (L.t.Np) {
    case 2: ne = PairShape<2>::NE; break;
    case 3: ne = PairShape<3>::NE; break;
    case 4: ne = PairShape<4>::NE; break;
    case 5: ne = PairShape<5>::NE; break;
    case 6: ne = PairShape<6>::NE; break;
    case 7: ne = PairShape<7>::NE; break;
    case 8: ne = PairShape<8>::NE; break;
    case 9: ne = PairShape<9>::NE; break;
    case 10: ne = PairShape<10>::NE; break;
    case 11: ne = PairShape<11>::NE; break;
    case 12: ne = PairShape<12>::NE; break;
    default: fail(SEM_EINVAL, "unsupported order N=%d", L.t.N);
  }
  const int64_t blocks = (L.t.E + ne - 1) / ne;
  return (int)(blocks < 1 ? 1 : (blocks > 152 * 16 ? 152 * 16 : blocks));
}

void launch_ax_pair_dot(const Level &L, const double *u, double *w, double *pw, Reducer &R,
                        cudaStream_t st) {
  SEM_REQUIRE(L.G2.p != nullptr, "pair-split geometric factors were not built");
  SEM_REQUIRE(pw != nullptr, "null inner-product target");
  SEM_REQUIRE((size_t)pair_fused_grid(L) <= R.capacity,
              "fused operator: reduction buffer too small");
  PairFuse g;
  g.partials = R.partials.p;
  g.counter = R.counter.p;
  g.pw = pw;
  switch (L.t.Np) {
    case 2: launch_fused_np<2>(L, u, w, g, st); break;
    case 3: launch_fused_np<3>(L, u, w, g, st); break;
    case 4: launch_fused_np<4>(L, u, w, g, st); break;
    case 5: launch_fused_np<5>(L, u, w, g, st); break;
    case 6: launch_fused_np<6>(L, u, w, g, st); break;
    case 7: launch_fused_np<7>(L, u, w, g, st); break;
    case 8: launch_fused_np<8>(L, u, w, g, st); break;
    case 9: launch_fused_np<9>(L, u, w, g, st); break;
    case 10: launch_fused_np<10>(L, u, w, g, st); break;
    case 11: launch_fused_np<11>(L, u, w, g, st); break;
    case 12: launch_fused_np<12>(L, u, w, g, st); break;
    default: fail(SEM_EINVAL, "unsupported order N=%d", L.t.N);
  }
}

}  // namespace sem
