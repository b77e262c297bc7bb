// gs.cu -- direct stiffness summation and Dirichlet masking on the box.
//
// Sec. 2: C0 continuity makes the SEM exchange a unit-depth stencil: a node
// on an element face, edge or vertex has 2, 4 or 8 local copies, and the
// gather-scatter (gs) replaces every copy by the sum of all copies.  Sec. 3
// builds that exchange from global vertex ids; on the box the ids are the
// lattice coordinates, so each thread takes one shared node from a table of
// unique ids and finds its copies arithmetically (no CSR index arrays).
// Copies are summed in a fixed order (x fastest, lower element first), so all
// copies end bit-identical and the result does not depend on scheduling.
#include "common.cuh"
#include "trace.cuh"

namespace sem {

struct GsGeom {
  Topo t;
  FastDiv div_nx, div_nxy, div_N;
  uint32_t nx, nxy;
};

static GsGeom gs_geom(const Topo &t) {
  GsGeom g;
  g.t = t;
  g.nx = (uint32_t)(t.ex * t.N + 1);
  g.nxy = g.nx * (uint32_t)(t.ey * t.N + 1);
  g.div_nx = FastDiv(g.nx);
  g.div_nxy = FastDiv(g.nxy);
  g.div_N = FastDiv((uint32_t)t.N);
  return g;
}

// Copies of lattice coordinate c along one direction with ne elements:
// (element index, local index) pairs, lower element first.
__device__ __forceinline__ int copies_1d(uint32_t c, int ne, int N, const FastDiv &dN, int *el,
                                         int *lo) {
  int q = (int)dN.div(c);
  int r = (int)c - q * N;
  if (r == 0 && q > 0 && q < ne) {
    el[0] = q - 1; lo[0] = N;
    el[1] = q;     lo[1] = 0;
    return 2;
  }
  if (q == ne) { el[0] = ne - 1; lo[0] = N; return 1; }
  el[0] = q; lo[0] = r;
  return 1;
}

template <typename T>
__global__ void gs_kernel(GsGeom g, const int32_t *__restrict__ nodes, int64_t nsh,
                          T *__restrict__ u) {
  const Topo &t = g.t;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < nsh;
       s += (int64_t)gridDim.x * blockDim.x) {
    uint32_t id = (uint32_t)nodes[s];
    uint32_t gz = g.div_nxy.div(id);
    uint32_t rem = id - gz * g.nxy;
    uint32_t gy = g.div_nx.div(rem);
    uint32_t gx = rem - gy * g.nx;
    int ex_[2], ix_[2], ey_[2], iy_[2], ez_[2], iz_[2];
    int cx = copies_1d(gx, t.ex, t.N, g.div_N, ex_, ix_);
    int cy = copies_1d(gy, t.ey, t.N, g.div_N, ey_, iy_);
    int cz = copies_1d(gz, t.ez, t.N, g.div_N, ez_, iz_);
    size_t idx[8];
    int n = 0;
    for (int c = 0; c < cz; ++c)
      for (int b = 0; b < cy; ++b)
        for (int a = 0; a < cx; ++a) {
          size_t e = (size_t)ex_[a] + (size_t)t.ex * ((size_t)ey_[b] + (size_t)t.ey * ez_[c]);
          idx[n++] = e * t.Np3 + ix_[a] + t.Np * (iy_[b] + t.Np * iz_[c]);
        }
    T sum = u[idx[0]];
    for (int q = 1; q < n; ++q) sum += u[idx[q]];
    for (int q = 0; q < n; ++q) u[idx[q]] = sum;
  }
}

// Zero the Dirichlet boundary: the points of element faces lying on the box
// boundary.  One thread per (boundary face, face point).
// 32-bit index arithmetic with multiplicative division throughout (64-bit
// integer division is emulated and competes for the FP64 pipe).
template <typename T>
__global__ void mask_faces_kernel(Topo t, uint32_t nfaces, FastDiv div_np2, T *__restrict__ u) {
  const uint32_t Np = (uint32_t)t.Np, Np2 = Np * Np;
  const uint32_t fx = (uint32_t)(t.ey * t.ez), fy = (uint32_t)(t.ex * t.ez);
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < nfaces * Np2;
       s += gridDim.x * blockDim.x) {
    const uint32_t f = div_np2.div(s);
    const uint32_t q = s - f * Np2;
    const uint32_t b = t.div_np.div(q), a = q - b * Np;
    int ix, iy, iz, i, j, k;
    const int side = (int)(f & 1);
    uint32_t h = f >> 1;
    if (h < fx) {  // x = 0 or x = 1 faces
      const uint32_t zz = t.div_ey.div(h);
      iy = (int)(h - zz * (uint32_t)t.ey); iz = (int)zz;
      ix = side ? t.ex - 1 : 0; i = side ? t.N : 0; j = (int)a; k = (int)b;
    } else if (h < fx + fy) {
      h -= fx;
      const uint32_t zz = t.div_ex.div(h);
      ix = (int)(h - zz * (uint32_t)t.ex); iz = (int)zz;
      iy = side ? t.ey - 1 : 0; j = side ? t.N : 0; i = (int)a; k = (int)b;
    } else {
      h -= fx + fy;
      const uint32_t yy = t.div_ex.div(h);
      ix = (int)(h - yy * (uint32_t)t.ex); iy = (int)yy;
      iz = side ? t.ez - 1 : 0; k = side ? t.N : 0; i = (int)a; j = (int)b;
    }
    size_t e = (size_t)ix + (size_t)t.ex * ((size_t)iy + (size_t)t.ey * iz);
    u[e * t.Np3 + i + Np * (j + Np * k)] = T(0);
  }
}

static int grid_1d(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  const int64_t cap = 152 * 8;
  return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

template <typename T>
void launch_gs(const Level &L, T *u, cudaStream_t st) {
  if (L.n_shared == 0) return;
  TraceScope ts(sizeof(T) == 8 ? "gs_f64" : "gs_f32", L.t.N, st);
  gs_kernel<T><<<grid_1d(L.n_shared, 256), 256, 0, st>>>(gs_geom(L.t), L.shared_nodes.p,
                                                          L.n_shared, u);
  SEM_CHECK_CUDA(cudaGetLastError());
}

template <typename T>
void launch_mask(const Level &L, T *u, cudaStream_t st) {
  if (L.t.bc != SEM_DIRICHLET) return;
  const Topo &t = L.t;
  int64_t nfaces = 2 * ((int64_t)t.ey * t.ez + (int64_t)t.ex * t.ez + (int64_t)t.ex * t.ey);
  TraceScope ts(sizeof(T) == 8 ? "mask_f64" : "mask_f32", t.N, st);
  mask_faces_kernel<T><<<grid_1d(nfaces * t.Np * t.Np, 256), 256, 0, st>>>(
      t, (uint32_t)nfaces, FastDiv((uint32_t)(t.Np * t.Np)), u);
  SEM_CHECK_CUDA(cudaGetLastError());
}

template void launch_gs<double>(const Level &, double *, cudaStream_t);
template void launch_gs<float>(const Level &, float *, cudaStream_t);
template void launch_mask<double>(const Level &, double *, cudaStream_t);
template void launch_mask<float>(const Level &, float *, cudaStream_t);

}  // namespace sem
