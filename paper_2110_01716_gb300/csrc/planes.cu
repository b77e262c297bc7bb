// planes.cu -- direct stiffness summation on the structured box by face-plane
// passes (Sec. 2: the C0 sum of the copies of each shared node).  On a box
// the copies of a node form a tensor product of at most two copies per
// direction, so summing across x-faces, then y-faces, then z-faces gives the
// full sum, and every copy receives the same bits.  Each pass also applies
// the Dirichlet mask of its direction's boundary planes.
#include <cstdint>

#include "common.cuh"
#include "kernels.cuh"
#include "trace.cuh"

namespace sem {

// V consecutive values as one vector access (16-byte aligned for V > 1).
template <typename T, int V>
struct VecOf {
  using type = T;
};
template <>
struct VecOf<float, 4> {
  using type = float4;
};
template <>
struct VecOf<double, 2> {
  using type = double2;
};
template <typename T, int V>
__device__ __forceinline__ void vload(const T *p, T (&o)[V]) {
  using VT = typename VecOf<T, V>::type;
  const VT v = *reinterpret_cast<const VT *>(p);
  const T *pv = reinterpret_cast<const T *>(&v);
#pragma unroll
  for (int c = 0; c < V; ++c) o[c] = pv[c];
}
template <typename T, int V>
__device__ __forceinline__ void vstore(T *p, const T (&o)[V]) {
  using VT = typename VecOf<T, V>::type;
  VT v;
  T *pv = reinterpret_cast<T *>(&v);
#pragma unroll
  for (int c = 0; c < V; ++c) pv[c] = o[c];
  *reinterpret_cast<VT *>(p) = v;
}

// Face planes normal to x (DIR 0), y (DIR 1) or z (DIR 2): lower copy + upper copy, and
// the Dirichlet mask of the box boundary planes of that direction.  One thread
// per V consecutive nodes of each element's lower plane (plus the upper plane
// of the last layer under Dirichlet); V > 1 only for y and z planes, whose rows
// run along i, and then every access is one aligned vector.
template <int DIR, typename T = float, int V = 1>
__global__ void plane_sum_kernel(Topo t, T *__restrict__ w, int dirichlet) {
  const int Np = t.Np, N = t.N;
  const uint32_t Np2 = (uint32_t)Np * Np;
  const uint64_t total = (uint64_t)t.E * Np2 / V;
  for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
       q += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t q32 = (uint32_t)(q * V);  // E * Np2 < 2^32 (checked by the launcher)
    const uint32_t r = t.div_np.div(q32);
    const uint32_t a = q32 - r * Np;   // fastest in-plane index: i
    const uint32_t e = t.div_np.div(r);
    const uint32_t b = r - e * Np;     // second in-plane index: k (y planes) or j (z planes)
    int64_t lo_off, hi_off, stride_e;
    int layer, layers;
    if (DIR == 0) {  // in-plane (a, b) = (j, k); rows of the plane are Np apart
      layer = (int)(e - t.div_ex.div(e) * t.ex);
      layers = t.ex;
      lo_off = (int64_t)b * Np2 + (int64_t)a * Np;
      hi_off = lo_off + N;
      stride_e = 1;
    } else if (DIR == 1) {
      const uint32_t ex_e = t.div_ex.div(e);
      layer = (int)(ex_e - t.div_ey.div(ex_e) * t.ey);
      layers = t.ey;
      lo_off = (int64_t)b * Np2 + a;
      hi_off = lo_off + (int64_t)N * Np;
      stride_e = t.ex;
    } else {
      layer = (int)t.div_ey.div(t.div_ex.div(e));
      layers = t.ez;
      lo_off = (int64_t)b * Np + a;
      hi_off = lo_off + (int64_t)N * Np2;
      stride_e = (int64_t)t.ex * t.ey;
    }
    T *we = w + (int64_t)e * t.Np3;
    T zero[V];
#pragma unroll
    for (int c = 0; c < V; ++c) zero[c] = T(0);
    if (layer > 0) {
      T *below = we - stride_e * t.Np3 + hi_off;
      T lo[V], hi[V];
      vload<T, V>(below, hi);
      vload<T, V>(we + lo_off, lo);
#pragma unroll
      for (int c = 0; c < V; ++c) lo[c] = hi[c] + lo[c];
      vstore<T, V>(below, lo);
      vstore<T, V>(we + lo_off, lo);
    } else if (dirichlet) {
      vstore<T, V>(we + lo_off, zero);
    }
    if (dirichlet && layer == layers - 1) vstore<T, V>(we + hi_off, zero);
  }
}

// One plane pass with the widest vector the order and alignment allow.
template <int DIR, typename T>
static void launch_plane(const Topo &t, T *w, int dirichlet, cudaStream_t st) {
  constexpr int VW = sizeof(T) == 4 ? 4 : 2;  // 16 bytes
  const bool vec = DIR != 0 && t.Np % VW == 0 && (reinterpret_cast<uintptr_t>(w) & 15u) == 0 &&
                   ((int64_t)t.Np3 * (int64_t)sizeof(T)) % 16 == 0;
  const int v = vec ? VW : 1;
  const int64_t n = t.E * t.Np * t.Np / v;
  const int64_t b = (n + 255) / 256;
  const int pg = (int)(b < 152 * 16 ? b : 152 * 16);
  if (vec) plane_sum_kernel<DIR, T, VW><<<pg, 256, 0, st>>>(t, w, dirichlet);
  else plane_sum_kernel<DIR, T, 1><<<pg, 256, 0, st>>>(t, w, dirichlet);
  SEM_CHECK_CUDA(cudaGetLastError());
}

void launch_plane_pass(const Topo &t, int dir, float *w, int dirichlet, cudaStream_t st) {
  SEM_REQUIRE((uint64_t)t.E * t.Np * t.Np < (1ull << 32), "mesh too large for the plane passes");
  if (dir == 0) launch_plane<0, float>(t, w, dirichlet, st);
  else if (dir == 1) launch_plane<1, float>(t, w, dirichlet, st);
  else launch_plane<2, float>(t, w, dirichlet, st);
}

// Direct stiffness summation of an FP32 E-layout vector by three plane
// passes (x, then y, then z faces; every copy receives the same bits) and the
// Dirichlet mask.
template <typename T>
void launch_planes_assemble(const Level &L, T *w, cudaStream_t st, bool mask) {
  const Topo &t = L.t;
  SEM_REQUIRE((uint64_t)t.E * t.Np * t.Np < (1ull << 32), "mesh too large for the plane passes");
  TraceScope ts(mask ? (sizeof(T) == 8 ? "plane_sum3_f64" : "plane_sum3")
                     : (sizeof(T) == 8 ? "gs_planes_f64" : "gs_planes_f32"),
                t.N, st, 3);
  const int dir = mask && t.bc == SEM_DIRICHLET;
  launch_plane<0, T>(t, w, dir, st);
  launch_plane<1, T>(t, w, dir, st);
  launch_plane<2, T>(t, w, dir, st);
}
template void launch_planes_assemble<float>(const Level &, float *, cudaStream_t, bool);
template void launch_planes_assemble<double>(const Level &, double *, cudaStream_t, bool);

}  // namespace sem
