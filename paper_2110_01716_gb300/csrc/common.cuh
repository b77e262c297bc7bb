// common.cuh -- internal declarations shared by the library's translation units.
//
// Nothing here is part of the C ABI (include/sem.h).  Errors inside the library
// are raised as sem::Failure and turned into a sem_status at the ABI boundary.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <cstdarg>
#include <map>
#include <string>
#include <vector>

#include "sem.h"

namespace sem {

// ------------------------------------------------------------------ errors
struct Failure {
  sem_status status;
};
[[noreturn]] void fail(sem_status st, const char *fmt, ...);
void set_error_message(const char *msg);

#define SEM_CHECK_CUDA(call)                                                              \
  do {                                                                                    \
    cudaError_t err_ = (call);                                                            \
    if (err_ != cudaSuccess)                                                              \
      ::sem::fail(err_ == cudaErrorMemoryAllocation ? SEM_ENOMEM : SEM_ECUDA, "%s:%d: %s: %s", \
                  __FILE__, __LINE__, #call, cudaGetErrorString(err_));                   \
  } while (0)

#define SEM_REQUIRE(cond, ...)                       \
  do {                                               \
    if (!(cond)) ::sem::fail(SEM_EINVAL, __VA_ARGS__); \
  } while (0)

// Host-side fault injection (sem_inject_alloc_failure): armed with k > 0,
// the k-th device allocation through DevBuf from then on fails with
// SEM_ENOMEM before cudaMalloc is called; 0 disarms.
inline std::atomic<int> g_alloc_fail_countdown{0};

// Device memory arena.  While a thread has one installed (ArenaScope), every
// DevBuf allocation made on that thread is carved from it: 256-byte aligned
// bump allocation from chunks of at least `chunk` bytes, so that building many
// small problems costs a few cudaMalloc calls instead of hundreds (each of
// which synchronises the device).  Buffers carved from an arena release
// nothing; the arena frees its chunks when it is destroyed, after every
// object built in it.
struct DevArena {
  size_t chunk = (size_t)1 << 30;
  std::vector<void *> chunks;
  char *cur = nullptr;
  size_t cap = 0, used = 0;
  size_t carved = 0;    // bytes handed out (alignment included)
  size_t reserved = 0;  // bytes of all chunks
  DevArena() = default;
  DevArena(const DevArena &) = delete;
  DevArena &operator=(const DevArena &) = delete;
  ~DevArena() {
    for (void *c : chunks) cudaFree(c);
  }
  void *take(size_t bytes) {
    const size_t a = (used + 255) & ~(size_t)255;
    if (!cur || a + bytes > cap) {
      const size_t sz = bytes > chunk ? bytes : chunk;
      if (g_alloc_fail_countdown.load(std::memory_order_relaxed) > 0 &&
          g_alloc_fail_countdown.fetch_sub(1) == 1)
        ::sem::fail(SEM_ENOMEM, "injected device allocation failure");
      void *c = nullptr;
      SEM_CHECK_CUDA(cudaMalloc(&c, sz));
      chunks.push_back(c);
      cur = static_cast<char *>(c);
      cap = sz;
      reserved += sz;
      carved += bytes;
      used = bytes;
      return cur;
    }
    carved += (a - used) + bytes;
    used = a + bytes;
    return cur + a;
  }
};
inline thread_local DevArena *t_arena = nullptr;
struct ArenaScope {
  DevArena *prev;
  explicit ArenaScope(DevArena *a) : prev(t_arena) { t_arena = a; }
  ~ArenaScope() { t_arena = prev; }
  ArenaScope(const ArenaScope &) = delete;
  ArenaScope &operator=(const ArenaScope &) = delete;
};

// Device allocation owned by a library object; freed in the destructor
// (unless it was carved from an arena, which frees it).
template <typename T>
struct DevBuf {
  T *p = nullptr;
  size_t n = 0;
  bool pooled = false;
  DevBuf() = default;
  DevBuf(const DevBuf &) = delete;
  DevBuf &operator=(const DevBuf &) = delete;
  ~DevBuf() { release(); }
  void alloc(size_t count) {
    release();
    if (count == 0) return;
    if (t_arena) {
      p = static_cast<T *>(t_arena->take(count * sizeof(T)));
      pooled = true;
      n = count;
      return;
    }
    if (g_alloc_fail_countdown.load(std::memory_order_relaxed) > 0 &&
        g_alloc_fail_countdown.fetch_sub(1) == 1)
      ::sem::fail(SEM_ENOMEM, "injected device allocation failure");
    SEM_CHECK_CUDA(cudaMalloc(&p, count * sizeof(T)));
    n = count;
  }
  void release() {
    if (p && !pooled) cudaFree(p);
    p = nullptr;
    n = 0;
    pooled = false;
  }
  size_t bytes() const { return n * sizeof(T); }
};

// ------------------------------------------------------------------ fast division
// Division of non-negative 32-bit integers below 2^31 by a runtime constant d
// with one high multiply (Granlund and Montgomery, PLDI 1994):
//   s = ceil(log2 d),  m = floor(2^32 (2^s - d) / d) + 1,
//   n / d = (umulhi(n, m) + n) >> s.
struct FastDiv {
  uint32_t d = 1, m = 0, s = 0;
  FastDiv() = default;
  explicit FastDiv(uint32_t div) : d(div) {
    s = 0;
    while ((1ull << s) < div) ++s;
    m = (uint32_t)((((1ull << s) - div) << 32) / div + 1);
  }
  __host__ __device__ __forceinline__ uint32_t div(uint32_t n) const {
#ifdef __CUDA_ARCH__
    return (__umulhi(n, m) + n) >> s;
#else
    return (uint32_t)((((uint64_t)n * m >> 32) + n) >> s);
#endif
  }
};

// ------------------------------------------------------------------ topology
// Structural description of a box mesh of order N.  Every quantity that
// depends only on where a local point sits (multiplicity, Dirichlet mask,
// copies of a shared node) is computed from indices on the fly, so no
// per-point integer arrays live in HBM.
struct Topo {
  int32_t ex, ey, ez, N, Np, Np3;
  int32_t bc;        // SEM_DIRICHLET / SEM_NEUMANN
  int64_t E, nl, ng; // elements, local points, unique nodes
  FastDiv div_np3, div_np, div_ex, div_ey;
};

// Six face bits of a point inside its element and of an element inside the box:
// bit 0: -r face (i = 0 / ix = 0), 1: +r, 2: -s, 3: +s, 4: -t, 5: +t.
__device__ __forceinline__ uint32_t point_face_bits(int i, int j, int k, int N) {
  return (i == 0) | ((i == N) << 1) | ((j == 0) << 2) | ((j == N) << 3) | ((k == 0) << 4) |
         ((k == N) << 5);
}
__device__ __forceinline__ uint32_t elem_face_bits(int ix, int iy, int iz, const Topo &t) {
  return (ix == 0) | ((ix == t.ex - 1) << 1) | ((iy == 0) << 2) | ((iy == t.ey - 1) << 3) |
         ((iz == 0) << 4) | ((iz == t.ez - 1) << 5);
}

struct PointInfo {
  uint32_t e, p;         // element, point in element
  int i, j, k;           // point indices
  int ix, iy, iz;        // element indices
  int log2_mult;         // number of copies = 2^log2_mult (0..3)
  float inv_mult;        // 1 / number of copies (exact: 1, 1/2, 1/4, 1/8)
  float mask;            // 0 on the Dirichlet boundary, else 1
};

// v / 2^k for k in 0..3 through the exponent field (integer instructions only,
// which keeps the scarce FP64 pipe free); values too small to scale become 0.
__device__ __forceinline__ double scale_pow2_down(double v, int k) {
  long long b = __double_as_longlong(v);
  long long ex = (b >> 52) & 0x7FF;
  return ex > k ? __longlong_as_double(b - ((long long)k << 52)) : 0.0;
}

__device__ __forceinline__ PointInfo point_info(uint32_t l, const Topo &t) {
  PointInfo q;
  q.e = t.div_np3.div(l);
  q.p = l - q.e * (uint32_t)t.Np3;
  uint32_t jk = t.div_np.div(q.p);
  q.i = (int)(q.p - jk * (uint32_t)t.Np);
  q.k = (int)t.div_np.div(jk);
  q.j = (int)(jk - (uint32_t)q.k * t.Np);
  uint32_t yz = t.div_ex.div(q.e);
  q.ix = (int)(q.e - yz * (uint32_t)t.ex);
  q.iz = (int)t.div_ey.div(yz);
  q.iy = (int)(yz - (uint32_t)q.iz * t.ey);
  uint32_t pf = point_face_bits(q.i, q.j, q.k, t.N);
  uint32_t ef = elem_face_bits(q.ix, q.iy, q.iz, t);
  q.log2_mult = __popc(pf & ~ef);
  q.inv_mult = 1.0f / (float)(1u << q.log2_mult);
  q.mask = (t.bc == SEM_DIRICHLET && (pf & ef)) ? 0.0f : 1.0f;
  return q;
}

// ------------------------------------------------------------------ basis tables
constexpr int kMaxNp = SEM_MAX_ORDER + 1;

// GLL nodes, weights and derivative matrix of one order (Sec. 2, footnote 1),
// small enough to travel to kernels as a parameter.
struct Basis {
  int N;
  double xi[kMaxNp];
  double w[kMaxNp];
  double D[kMaxNp * kMaxNp];  // D[i*Np + l] = h_l'(xi_i)
  float D32[kMaxNp * kMaxNp];
};
Basis make_basis(int N);

// ------------------------------------------------------------------ levels
// One discretisation of the box at order N: geometry, numbering and the
// Jacobi diagonal, in the precisions its users need.
struct Level {
  Topo t{};
  Basis basis{};
  int32_t geom = SEM_GEOM_STORED;
  int32_t arith = SEM_ARITH_PAIR;  // FP64 operator arithmetic (stored geometry)
  std::vector<double> verts_host;  // lattice [(ex+1)(ey+1)(ez+1)][3]
  DevBuf<double> verts;            // per element [E][8][3], corner (a,b,c) at a+2b+4c
  DevBuf<double> G64;              // [E][6][Np3]  (rr, rs, rt, ss, st, tt)
  DevBuf<float> G32;               // [E][6][Np3]
  DevBuf<float2> G2;               // [E][6][Np3] FP64 factors split into float pairs
  DevBuf<uint16_t> G16[2];         // [E][6][Np3] G / scale as FP16 [0] or BF16 [1] bits
  DevBuf<float> G16scale[2];       // [E] per element: max |G| over its six factors
  DevBuf<int> err;                 // set by kernels whose bounded waits ran out
  // Work units (x-line segments) the FP32 operator aims for per resident CTA
  // slot of the GPU; below 1 the operator also uses only that share of the
  // slots (batched solves share the GPU).  The x-face sums are the same bits
  // for any value: this only moves work between CTAs.
  float ax32_fill = 2.0f;
  DevBuf<int32_t> shared_nodes;    // unique ids of nodes with more than one copy
  int64_t n_shared = 0;
  DevBuf<double> dinv64;           // mask / assembled diagonal
  DevBuf<float> dinv32;
  size_t device_bytes() const {
    return verts.bytes() + G64.bytes() + G32.bytes() + G2.bytes() + G16[0].bytes() +
           G16[1].bytes() + G16scale[0].bytes() + G16scale[1].bytes() + err.bytes() + shared_nodes.bytes() + dinv64.bytes() + dinv32.bytes();
  }
};

// ------------------------------------------------------------------ basis (host)
void gll_points(int N, double *xi, double *w);
void derivative_matrix(int N, const double *xi, double *D);
void interpolation_matrix(int Nf, int Nc, double *J);

// ------------------------------------------------------------------ launches
void build_level(Level &L, int ex, int ey, int ez, int N, int bc, int geom, int arith,
                 const double *verts_host, bool want_g32, cudaStream_t st);
void launch_ax_pair(const Level &L, const double *u, double *w, cudaStream_t st);
void level_ensure_f32(Level &L, cudaStream_t st);
// 16-bit geometric factors (kind SEM_F16 or SEM_BF16) with per-element,
// per-factor scales, plus the FP32 Jacobi inverse.
void level_ensure_g16(Level &L, int kind, cudaStream_t st);
void level_ensure_dinv32(Level &L, cudaStream_t st);
// FP32 operator on stored factors, kind SEM_F32 / SEM_F16 / SEM_BF16 (the
// factor storage); assemble: w = mask * gs(A_L u), else w = A_L u.
void launch_ax32(const Level &L, int kind, const float *u, float *w, bool assemble,
                 cudaStream_t st);
// Sum the copies of every node of an E-layout vector (x, y, z face passes)
// and, with `mask`, apply the Dirichlet mask.
template <typename T>
void launch_planes_assemble(const Level &L, T *w, cudaStream_t st, bool mask = true);
// One FP32 face-plane pass (dir 0, 1, 2: x, y, z) with that direction's
// Dirichlet mask (planes.cu).
void launch_plane_pass(const Topo &t, int dir, float *w, int dirichlet, cudaStream_t st);
// FP64 geometric factors of a level into `out` (computed again; for setup).
void level_fp64_factors(const Level &L, DevBuf<double> &out, cudaStream_t st);

template <typename T>
void launch_ax(const Level &L, const T *u, T *w, cudaStream_t st);
template <typename T>
void launch_gs(const Level &L, T *u, cudaStream_t st);
template <typename T>
void launch_mask(const Level &L, T *u, cudaStream_t st);
void launch_field(const Level &L, int which, double *out, cudaStream_t st);

// Deterministic reductions into device scalars (see vec.cu).
struct Reducer {
  DevBuf<double> partials;  // [nblocks][nsums]
  DevBuf<unsigned int> counter;
  int nblocks = 0;
  size_t capacity = 0;      // partials held (nblocks x nsums)
  void init(int blocks, int max_sums);
};

}  // namespace sem

// Opaque handles of the ABI.
struct sem_proj {
  sem_mesh *mesh = nullptr;
  int Lmax = 0, nvec = 0;
  sem::DevBuf<double> P, AP;  // [Lmax][stride], [Lmax + 1][stride] (last: scratch)
  sem::DevBuf<double> bp, dx; // projected right-hand side, correction
  sem::DevBuf<double> coef;   // device coefficients of one multi-dot
};
struct sem_mesh {
  sem::Level fine;
  cudaStream_t stream = nullptr;
  sem::Reducer red;
  sem::DevBuf<double> scal;   // device scalars of the solvers
  sem::DevBuf<double> work;   // solver work vectors
  sem::DevBuf<double> host_b, host_x;  // device copies for sem_solve_host
  double *pinned = nullptr;   // host-pinned scalars
  sem::DevBuf<double> krylov; // FGMRES: V (restart + 1) and Z (restart) vectors
  int krylov_m = 0;
  sem::Reducer kred;          // reductions of up to restart + 1 sums
  sem::DevBuf<double> kscal;  // FGMRES device scalars
  double *kpinned = nullptr;  // host-pinned copy of one Hessenberg column
  // FlexCG loop captured into a CUDA graph (sem_solve_desc.use_graph)
  cudaGraphExec_t graph = nullptr;
  cudaStream_t cstream = nullptr;  // capture stream
  uint64_t graph_pmg = 0;          // serial of the pMG captured
  const double *graph_x = nullptr; // solution vector captured
  int graph_kernels = 0;           // kernels per loop pass
  std::map<std::string, int64_t> graph_tally;  // of them, per trace class
};
