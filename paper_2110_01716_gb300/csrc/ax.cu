// ax.cu -- matrix-free stiffness operator w = A_L u on deformed hexahedra.
//
// Sec. 2, footnote 1: derivatives are tensor contractions u_r = Dhat u along
// each reference direction; the operator is
//   w^e = sum_d D_d^T ( sum_e G_de D_e u^e ),
// with the six symmetric geometric factors G (rr, rs, rt, ss, st, tt) either
// read from HBM (stored) or recomputed from the element's 8 vertices
// (trilinear).
//
// Thread layout: one thread per (i, j) column of an element, looping over k;
// NE elements per CTA.  The element's u is staged in shared memory (the r and s
// contractions read across the column) and kept in registers along k (the t
// contraction is thread-local).  The second half reuses the same buffers for
// the r and s fluxes.
#include "common.cuh"
#include "device_basis.cuh"
#include "trace.cuh"

namespace sem {

template <int NP>
struct AxShape {
  static constexpr int NP2 = NP * NP;
  static constexpr int NP3 = NP2 * NP;
  static constexpr int NE = (256 / NP2) < 1 ? 1 : (256 / NP2);
  static constexpr int THREADS = NE * NP2;
};

template <typename T>
__device__ __forceinline__ const T *basis_D(const Basis &b);
template <>
__device__ __forceinline__ const double *basis_D<double>(const Basis &b) {
  return b.D;
}
template <>
__device__ __forceinline__ const float *basis_D<float>(const Basis &b) {
  return b.D32;
}

template <typename T, int NP, bool TRILINEAR>
__global__ void __launch_bounds__(AxShape<NP>::THREADS)
    ax_kernel(int64_t E, Basis bs, const T *__restrict__ u, T *__restrict__ w,
              const T *__restrict__ G, const double *__restrict__ verts) {
  using S = AxShape<NP>;
  constexpr int NP2 = S::NP2, NP3 = S::NP3, NE = S::NE;
  __shared__ T sD[NP][NP + 1];
  __shared__ T sA[NE][NP3];
  __shared__ T sB[NE][NP3];
  __shared__ T sV[NE][24];

  const int le = threadIdx.x / NP2;
  const int ij = threadIdx.x - le * NP2;
  const int i = ij % NP, j = ij / NP;
  const T *Dg = basis_D<T>(bs);
  for (int q = threadIdx.x; q < NP * NP; q += blockDim.x) sD[q / NP][q % NP] = Dg[q];

  for (int64_t e0 = (int64_t)blockIdx.x * NE; e0 < E; e0 += (int64_t)gridDim.x * NE) {
    const int64_t e = e0 + le;
    const bool active = (threadIdx.x < NE * NP2) && e < E;
    T ru[NP];
    if (active) {
      const T *ue = u + e * NP3;
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        ru[k] = ue[ij + k * NP2];
        sA[le][ij + k * NP2] = ru[k];
      }
      if (TRILINEAR)
        for (int q = ij; q < 24; q += NP2) sV[le][q] = (T)verts[e * 24 + q];
    }
    __syncthreads();
    T wr[NP], ws[NP], wt[NP];
    if (active) {
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        T ur = 0, us = 0, ut = 0;
#pragma unroll
        for (int l = 0; l < NP; ++l) {
          ur += sD[i][l] * sA[le][l + j * NP + k * NP2];
          us += sD[j][l] * sA[le][i + l * NP + k * NP2];
          ut += sD[k][l] * ru[l];
        }
        T g[6];
        if (TRILINEAR) {
          T B, X[3];
          trilinear_metric<T>(sV[le], (T)bs.xi[i], (T)bs.xi[j], (T)bs.xi[k],
                              (T)(bs.w[i] * bs.w[j] * bs.w[k]), g, &B, X);
        } else {
          const T *Ge = G + e * 6 * NP3 + ij + k * NP2;
#pragma unroll
          for (int f = 0; f < 6; ++f) g[f] = Ge[f * NP3];
        }
        wr[k] = g[0] * ur + g[1] * us + g[2] * ut;
        ws[k] = g[1] * ur + g[3] * us + g[4] * ut;
        wt[k] = g[2] * ur + g[4] * us + g[5] * ut;
      }
    }
    __syncthreads();
    if (active) {
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        sA[le][ij + k * NP2] = wr[k];
        sB[le][ij + k * NP2] = ws[k];
      }
    }
    __syncthreads();
    if (active) {
      T *we = w + e * NP3;
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        T acc = 0;
#pragma unroll
        for (int l = 0; l < NP; ++l) {
          acc += sD[l][i] * sA[le][l + j * NP + k * NP2];
          acc += sD[l][j] * sB[le][i + l * NP + k * NP2];
          acc += sD[l][k] * wt[l];
        }
        we[ij + k * NP2] = acc;
      }
    }
    __syncthreads();
  }
}

static int ax_grid(int64_t E, int ne) {
  int64_t b = (E + ne - 1) / ne;
  const int64_t cap = 152 * 16;
  return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

template <typename T, int NP>
static void ax_dispatch_geom(const Level &L, const T *u, T *w, cudaStream_t st) {
  using S = AxShape<NP>;
  const T *G = nullptr;
  const bool f64 = sizeof(T) == 8;
  const bool tri = L.geom != SEM_GEOM_STORED;
  TraceScope ts(tri ? (f64 ? "ax_f64_tri" : "ax_f32_tri") : (f64 ? "ax_f64" : "ax_f32"), L.t.N, st);
  if (L.geom == SEM_GEOM_STORED) {
    if constexpr (sizeof(T) == 8) G = (const T *)L.G64.p;
    else G = (const T *)L.G32.p;
    SEM_REQUIRE(G != nullptr, "geometric factors of this precision were not built");
    ax_kernel<T, NP, false><<<ax_grid(L.t.E, S::NE), S::THREADS, 0, st>>>(L.t.E, L.basis, u, w, G,
                                                                           L.verts.p);
  } else {
    ax_kernel<T, NP, true><<<ax_grid(L.t.E, S::NE), S::THREADS, 0, st>>>(L.t.E, L.basis, u, w,
                                                                          nullptr, L.verts.p);
  }
  SEM_CHECK_CUDA(cudaGetLastError());
}

template <typename T>
void launch_ax(const Level &L, const T *u, T *w, cudaStream_t st) {
  if constexpr (sizeof(T) == 8) {
    if (L.geom == SEM_GEOM_STORED && L.arith == SEM_ARITH_PAIR) {
      launch_ax_pair(L, u, w, st);
      return;
    }
  }
  switch (L.t.Np) {
    case 2: ax_dispatch_geom<T, 2>(L, u, w, st); break;
    case 3: ax_dispatch_geom<T, 3>(L, u, w, st); break;
    case 4: ax_dispatch_geom<T, 4>(L, u, w, st); break;
    case 5: ax_dispatch_geom<T, 5>(L, u, w, st); break;
    case 6: ax_dispatch_geom<T, 6>(L, u, w, st); break;
    case 7: ax_dispatch_geom<T, 7>(L, u, w, st); break;
    case 8: ax_dispatch_geom<T, 8>(L, u, w, st); break;
    case 9: ax_dispatch_geom<T, 9>(L, u, w, st); break;
    case 10: ax_dispatch_geom<T, 10>(L, u, w, st); break;
    case 11: ax_dispatch_geom<T, 11>(L, u, w, st); break;
    case 12: ax_dispatch_geom<T, 12>(L, u, w, st); break;
    default: fail(SEM_EINVAL, "unsupported order N=%d", L.t.N);
  }
}

template void launch_ax<double>(const Level &, const double *, double *, cudaStream_t);
template void launch_ax<float>(const Level &, const float *, float *, cudaStream_t);

}  // namespace sem
