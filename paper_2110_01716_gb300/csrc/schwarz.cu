// schwarz.cu -- overlapping Schwarz preconditioner with fast-diagonalisable
// local problems (Sec. 3, Eq. 3), the second smoother family of the pMG.
//
// Each element is extended by one point into each face neighbour (n = N + 3
// points per direction) and carries a separable local operator
//   K_e = Bz x By x Ax + Bz x Ay x Bx + Az x By x Bx,
// whose 1D factors are the 1D SEM stiffness and mass assembled over the
// neighbour, the element and the other neighbour (each at its mean length
// along that direction: the mean of its four edges there), restricted to the
// extended points; without a neighbour the extension point is decoupled, and
// a Dirichlet boundary face is decoupled too.  With the generalised
// eigenpairs A S = B S L, S^T B S = I of each direction,
//   K_e^{-1} = (Sz x Sy x Sx) (I x I x Lx + I x Ly x I + Lz x I x I)^{-1} (Sz x Sy x Sx)^T.
// The preconditioner is z = mask sum_e R_e^T K_e^{-1} R_e r with face data
// only (extended points outside the element in two directions carry none).
//
// Setup: one thread per (element, direction) builds the 1D pencil and
// diagonalises B^{-1/2} A B^{-1/2} with the cyclic Jacobi method (Golub and
// Van Loan, Matrix Computations, Alg. 8.5.3), in FP64.
// Apply: one CTA holds several extended elements in shared memory; one
// thread per pencil applies the six 1D contractions (and the diagonal solve)
// along the pencil's direction.  Own points go to z, the six face layers to a
// side buffer; a second kernel adds each element's neighbours' layers to its
// own points, and the copies of shared nodes are then summed.
#include <cmath>

#include "common.cuh"
#include "kernels.cuh"
#include "schwarz.cuh"
#include "trace.cuh"

namespace sem {

constexpr int kMaxExt = kMaxNp + 2;  // points per direction of an extended element

// mean length of element e along d from its 8 vertices ([24] per element,
// vertex a + 2 b + 4 c)
__device__ double mean_length(const double *__restrict__ V, int d) {
  double s = 0.0;
  for (int q = 0; q < 4; ++q) {
    int c0[3] = {0, 0, 0};
    const int o1 = (d + 1) % 3, o2 = (d + 2) % 3;
    c0[o1] = q & 1;
    c0[o2] = (q >> 1) & 1;
    int c1[3] = {c0[0], c0[1], c0[2]};
    c1[d] = 1;
    const int v0 = c0[0] + 2 * c0[1] + 4 * c0[2], v1 = c1[0] + 2 * c1[1] + 4 * c1[2];
    double l2 = 0.0;
    for (int m = 0; m < 3; ++m) {
      const double dx = V[3 * v1 + m] - V[3 * v0 + m];
      l2 += dx * dx;
    }
    s += sqrt(l2);
  }
  return 0.25 * s;
}

__global__ void asm_setup_kernel(Topo t, Basis bs, const double *__restrict__ verts,
                                 double *__restrict__ S, double *__restrict__ lam) {
  const int N = t.N, Np = t.Np, n = N + 3;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < t.E * 3;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = q / 3;
    const int d = (int)(q - e * 3);
    const int ix = (int)(e % t.ex), iy = (int)((e / t.ex) % t.ey), iz = (int)(e / ((int64_t)t.ex * t.ey));
    const int pos = d == 0 ? ix : (d == 1 ? iy : iz);
    const int cnt = d == 0 ? t.ex : (d == 1 ? t.ey : t.ez);
    const int64_t stride = d == 0 ? 1 : (d == 1 ? t.ex : (int64_t)t.ex * t.ey);
    double A[kMaxExt * kMaxExt], Bd[kMaxExt], V[kMaxExt * kMaxExt];
    for (int k = 0; k < n * n; ++k) A[k] = 0.0;
    for (int k = 0; k < n; ++k) Bd[k] = 0.0;
    // 1D reference stiffness sum_q w_q D_qi D_qj, scaled by 2/h; mass (h/2) w_i
    auto add_elem = [&](double h, int i0, int i1, int a0) {
      for (int i = i0; i <= i1; ++i) {
        for (int j = i0; j <= i1; ++j) {
          double s = 0.0;
          for (int k = 0; k < Np; ++k) s += bs.w[k] * bs.D[k * Np + i] * bs.D[k * Np + j];
          A[(a0 + i - i0) * n + (a0 + j - i0)] += (2.0 / h) * s;
        }
        Bd[a0 + i - i0] += 0.5 * h * bs.w[i];
      }
    };
    add_elem(mean_length(verts + e * 24, d), 0, N, 1);
    if (pos > 0) add_elem(mean_length(verts + (e - stride) * 24, d), N - 1, N, 0);
    if (pos < cnt - 1) add_elem(mean_length(verts + (e + stride) * 24, d), 0, 1, N + 1);
    int dec[4], nd = 0;
    if (pos == 0) {
      dec[nd++] = 0;
      if (t.bc == SEM_DIRICHLET) dec[nd++] = 1;
    }
    if (pos == cnt - 1) {
      dec[nd++] = N + 2;
      if (t.bc == SEM_DIRICHLET) dec[nd++] = N + 1;
    }
    for (int k = 0; k < nd; ++k) {
      const int a = dec[k];
      for (int m = 0; m < n; ++m) A[a * n + m] = A[m * n + a] = 0.0;
      A[a * n + a] = 1.0;
      Bd[a] = 1.0;
    }
    // C = B^-1/2 A B^-1/2, then cyclic Jacobi: C = V diag V^T
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) A[i * n + j] /= sqrt(Bd[i] * Bd[j]);
    for (int i = 0; i < n * n; ++i) V[i] = 0.0;
    for (int i = 0; i < n; ++i) V[i * n + i] = 1.0;
    for (int sweep = 0; sweep < 40; ++sweep) {
      double off = 0.0, tot = 0.0;
      for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
          tot += A[i * n + j] * A[i * n + j];
          if (i != j) off += A[i * n + j] * A[i * n + j];
        }
      if (off <= 1e-30 * tot) break;
      for (int p = 0; p < n - 1; ++p)
        for (int r = p + 1; r < n; ++r) {
          const double apq = A[p * n + r];
          if (fabs(apq) < 1e-300) continue;
          const double theta = (A[r * n + r] - A[p * n + p]) / (2.0 * apq);
          const double tt = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(1.0 + theta * theta));
          const double c = 1.0 / sqrt(1.0 + tt * tt), s = tt * c;
          for (int k = 0; k < n; ++k) {  // A <- A J (columns p, r)
            const double akp = A[k * n + p], akr = A[k * n + r];
            A[k * n + p] = c * akp - s * akr;
            A[k * n + r] = s * akp + c * akr;
          }
          for (int k = 0; k < n; ++k) {  // A <- J^T A (rows p, r)
            const double apk = A[p * n + k], ark = A[r * n + k];
            A[p * n + k] = c * apk - s * ark;
            A[r * n + k] = s * apk + c * ark;
          }
          for (int k = 0; k < n; ++k) {  // V <- V J
            const double vkp = V[k * n + p], vkr = V[k * n + r];
            V[k * n + p] = c * vkp - s * vkr;
            V[k * n + r] = s * vkp + c * vkr;
          }
        }
    }
    // S = B^-1/2 V; store S[point][mode] and the eigenvalues
    double *So = S + (e * 3 + d) * (int64_t)n * n;
    double *lo = lam + (e * 3 + d) * (int64_t)n;
    for (int i = 0; i < n; ++i) {
      lo[i] = A[i * n + i];
      for (int m = 0; m < n; ++m) So[i * n + m] = V[i * n + m] / sqrt(Bd[i]);
    }
  }
}

template <typename A, typename B>
__global__ void asm_convert_kernel(int64_t n, const A *__restrict__ a, B *__restrict__ b) {
  for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < n;
       l += (int64_t)gridDim.x * blockDim.x)
    b[l] = (B)a[l];
}

template <int NP>
struct AsmShape {
  static constexpr int n = NP + 2;
  static constexpr int n2 = n * n;
  static constexpr int NEL = (256 / n2) < 1 ? 1 : (256 / n2);  // elements per CTA
  static constexpr int THREADS = NEL * n2;
  static constexpr int RS = n + 1;                                // padded row stride
  static constexpr int PS = n * RS;                               // plane stride
  static constexpr int ES = n * PS;                               // element stride
  static constexpr int SR = (n + 3) / 4 * 4;                      // S row stride (16-byte rows)
  // resident CTAs asked of the register allocator (about 20 warps per SM)
  static constexpr int MIN_CTAS = (20 * 32 + THREADS - 1) / THREADS;
};

// n values of a padded shared row (16-byte aligned) into registers
template <typename T, int n>
__device__ __forceinline__ void load_srow(const T *row, T (&o)[n]) {
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int c = 0; c < (n + 3) / 4; ++c) {
      const float4 v = *reinterpret_cast<const float4 *>(row + 4 * c);
      if (4 * c + 0 < n) o[4 * c + 0] = v.x;
      if (4 * c + 1 < n) o[4 * c + 1] = v.y;
      if (4 * c + 2 < n) o[4 * c + 2] = v.z;
      if (4 * c + 3 < n) o[4 * c + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int c = 0; c < (n + 1) / 2; ++c) {
      const double2 v = *reinterpret_cast<const double2 *>(row + 2 * c);
      if (2 * c + 0 < n) o[2 * c + 0] = v.x;
      if (2 * c + 1 < n) o[2 * c + 1] = v.y;
    }
  }
}

// out[m] = sum_a M[m][a] in[a], rows of M padded to SR in shared memory
template <typename T, int n, int SR>
__device__ __forceinline__ void pencil_mv(const T *M, const T (&in)[n], T (&out)[n]) {
#pragma unroll
  for (int m = 0; m < n; ++m) {
    T row[n];
    load_srow<T, n>(M + m * SR, row);
    T s = 0;
#pragma unroll
    for (int a = 0; a < n; ++a) s += row[a] * in[a];
    out[m] = s;
  }
}

// Local solves of every element: own points of K_e^{-1} R_e r into z, face
// layers into ext[E][6][Np^2] (0: x-, 1: x+, 2: y-, 3: y+, 4: z-, 5: z+).
// The separable inverse S (Lambda)^{-1} S^T is applied direction by
// direction, z first and last: thread (a, b) gathers its pencil along c
// straight from HBM into registers (consecutive threads read consecutive
// points of a row, and a thread's loads are independent), transforms it and
// leaves it in shared memory; y and x run on shared memory (with the
// diagonal between the forward and backward x transforms); the backward z
// transform returns each pencil to registers and stores it straight to z and
// ext.  Shared memory per element: the extended data (rows padded against
// bank conflicts) and S and S^T of the three directions with rows padded to
// whole 16-byte vectors, so that a pencil thread reads a matrix row per
// vector load.
template <typename T, int NP>
__global__ void __launch_bounds__(AsmShape<NP>::THREADS, AsmShape<NP>::MIN_CTAS)
    asm_solve_kernel(Topo t, const T *__restrict__ S, const T *__restrict__ lam,
                     const T *__restrict__ r, T *__restrict__ z, T *__restrict__ ext) {
  using Sh = AsmShape<NP>;
  constexpr int n = Sh::n, n2 = Sh::n2, NEL = Sh::NEL, RS = Sh::RS, PS = Sh::PS, ES = Sh::ES;
  constexpr int SR = Sh::SR, N = NP - 1, NP2 = NP * NP;
  __shared__ T sU[NEL * ES];
  __shared__ __align__(16) T sS[NEL][3][n * SR];   // S[d]: row a (point), by mode
  __shared__ __align__(16) T sST[NEL][3][n * SR];  // S[d]^T: row m (mode), by point
  __shared__ T sL[NEL][3][n];
  const int le = threadIdx.x / n2, pq = threadIdx.x - le * n2;
  const int p = pq % n, q = pq / n;
  T *U = sU + le * ES;
  for (int64_t e0 = (int64_t)blockIdx.x * NEL; e0 < t.E; e0 += (int64_t)gridDim.x * NEL) {
    const int64_t e = e0 + le;
    const bool active = e < t.E;
    T v[n], o[n];
    if (active) {
      for (int k = pq; k < 3 * n * n; k += n2) {
        const int d = k / (n * n), a = (k / n) % n, m = k % n;
        const T sv = S[e * 3 * n * n + k];
        sS[le][d][a * SR + m] = sv;
        sST[le][d][m * SR + a] = sv;
      }
      for (int k = pq; k < 3 * n; k += n2) sL[le][k / n][k % n] = lam[e * 3 * n + k];
      const int ix = (int)(e % t.ex), iy = (int)((e / t.ex) % t.ey),
                iz = (int)(e / ((int64_t)t.ex * t.ey));
      const int64_t exy = (int64_t)t.ex * t.ey;
      // face neighbours (or -1), scalars so that no local array is indexed
      const int64_t nxm = ix > 0 ? e - 1 : -1, nxp = ix < t.ex - 1 ? e + 1 : -1;
      const int64_t nym = iy > 0 ? e - t.ex : -1, nyp = iy < t.ey - 1 ? e + t.ex : -1;
      const int64_t nzm = iz > 0 ? e - exy : -1, nzp = iz < t.ez - 1 ? e + exy : -1;
      // gather the pencil (a = p, b = q) along c; extended points outside
      // the element in two directions carry no data
      const int ai = p - 1, bi = q - 1;
      const bool aown = ai >= 0 && ai <= N, bown = bi >= 0 && bi <= N;
#pragma unroll
      for (int c = 0; c < n; ++c) {
        const int ci = c - 1;
        const bool cown = ci >= 0 && ci <= N;
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
        v[c] = src >= 0 ? r[src] : (T)0;
      }
    }
    __syncthreads();
    // z: (Sz^T u) along c, thread (a = p, b = q)
    if (active) {
      pencil_mv<T, n, SR>(sST[le][2], v, o);
#pragma unroll
      for (int m = 0; m < n; ++m) U[m * PS + q * RS + p] = o[m];
    }
    __syncthreads();
    // y: thread (a = p, c = q)
    if (active) {
#pragma unroll
      for (int b = 0; b < n; ++b) v[b] = U[q * PS + b * RS + p];
      pencil_mv<T, n, SR>(sST[le][1], v, o);
#pragma unroll
      for (int m = 0; m < n; ++m) U[q * PS + m * RS + p] = o[m];
    }
    __syncthreads();
    // x, diagonal solve, x back: thread (b = p, c = q)
    if (active) {
#pragma unroll
      for (int a = 0; a < n; ++a) v[a] = U[q * PS + p * RS + a];
      pencil_mv<T, n, SR>(sST[le][0], v, o);
      const T lyz = sL[le][1][p] + sL[le][2][q];
#pragma unroll
      for (int m = 0; m < n; ++m) o[m] = o[m] / (sL[le][0][m] + lyz);
      pencil_mv<T, n, SR>(sS[le][0], o, v);
#pragma unroll
      for (int a = 0; a < n; ++a) U[q * PS + p * RS + a] = v[a];
    }
    __syncthreads();
    // y back: thread (a = p, c = q)
    if (active) {
#pragma unroll
      for (int m = 0; m < n; ++m) v[m] = U[q * PS + m * RS + p];
      pencil_mv<T, n, SR>(sS[le][1], v, o);
#pragma unroll
      for (int b = 0; b < n; ++b) U[q * PS + b * RS + p] = o[b];
    }
    __syncthreads();
    // z back and output: thread (a = p, b = q); own points to z, the face
    // layers to ext (rows of consecutive threads are consecutive points)
    if (active) {
#pragma unroll
      for (int m = 0; m < n; ++m) v[m] = U[m * PS + q * RS + p];
      pencil_mv<T, n, SR>(sS[le][2], v, o);
      const bool aown = p >= 1 && p <= N + 1, bown = q >= 1 && q <= N + 1;
#pragma unroll
      for (int c = 0; c < n; ++c) {
        const bool cown = c >= 1 && c <= N + 1;
        if (aown && bown && cown) {
          z[e * t.Np3 + (p - 1) + NP * ((q - 1) + NP * (c - 1))] = o[c];
        } else if (!aown && bown && cown) {
          ext[(e * 6 + (p == 0 ? 0 : 1)) * NP2 + (q - 1) + NP * (c - 1)] = o[c];
        } else if (aown && !bown && cown) {
          ext[(e * 6 + (q == 0 ? 2 : 3)) * NP2 + (p - 1) + NP * (c - 1)] = o[c];
        } else if (aown && bown && !cown) {
          ext[(e * 6 + (c == 0 ? 4 : 5)) * NP2 + (p - 1) + NP * (q - 1)] = o[c];
        }
      }
    }
    __syncthreads();
  }
}

// z_e(p) += the face layers of e's neighbours that cover p: a neighbour's x+
// layer covers e's i = 1 plane, its x- layer e's i = N - 1 plane (and the
// same in y and z).  Layers of missing neighbours are not read.
template <typename T>
__global__ void asm_pull_kernel(Topo t, const T *__restrict__ ext, T *__restrict__ z) {
  const int N = t.N, Np = t.Np, Np2 = Np * Np;
  for (uint32_t l = blockIdx.x * blockDim.x + threadIdx.x; l < (uint32_t)t.nl;
       l += gridDim.x * blockDim.x) {
    const PointInfo pi = point_info(l, t);
    const int64_t e = pi.e;
    T s = z[l];
    if (pi.i == 1 && pi.ix > 0) s += ext[((e - 1) * 6 + 1) * Np2 + pi.j + Np * pi.k];
    if (pi.i == N - 1 && pi.ix < t.ex - 1) s += ext[((e + 1) * 6 + 0) * Np2 + pi.j + Np * pi.k];
    if (pi.j == 1 && pi.iy > 0) s += ext[((e - t.ex) * 6 + 3) * Np2 + pi.i + Np * pi.k];
    if (pi.j == N - 1 && pi.iy < t.ey - 1) s += ext[((e + t.ex) * 6 + 2) * Np2 + pi.i + Np * pi.k];
    const int64_t exy = (int64_t)t.ex * t.ey;
    if (pi.k == 1 && pi.iz > 0) s += ext[((e - exy) * 6 + 5) * Np2 + pi.i + Np * pi.j];
    if (pi.k == N - 1 && pi.iz < t.ez - 1) s += ext[((e + exy) * 6 + 4) * Np2 + pi.i + Np * pi.j];
    z[l] = s;
  }
}

void asm_setup(AsmData &A, const Level &L, bool want_f32, cudaStream_t st) {
  const Topo &t = L.t;
  SEM_REQUIRE(t.N >= 1 && t.Np + 2 <= kMaxExt, "Schwarz smoother: order %d unsupported", t.N);
  A.n = t.N + 3;
  const int64_t ns = t.E * 3 * (int64_t)A.n * A.n, nl = t.E * 3 * (int64_t)A.n;
  A.S64.alloc(ns);
  A.lam64.alloc(nl);
  {
    TraceScope ts("asm_setup", t.N, st);
    const int64_t g = (t.E * 3 + 127) / 128;
    asm_setup_kernel<<<(int)(g < 152 * 16 ? g : 152 * 16), 128, 0, st>>>(t, L.basis, L.verts.p,
                                                                        A.S64.p, A.lam64.p);
    SEM_CHECK_CUDA(cudaGetLastError());
  }
  const int64_t next = t.E * 6 * (int64_t)t.Np * t.Np;
  if (want_f32) {
    A.S32.alloc(ns);
    A.lam32.alloc(nl);
    asm_convert_kernel<double, float><<<vec_grid(ns), kVecThreads, 0, st>>>(ns, A.S64.p, A.S32.p);
    asm_convert_kernel<double, float><<<vec_grid(nl), kVecThreads, 0, st>>>(nl, A.lam64.p, A.lam32.p);
    SEM_CHECK_CUDA(cudaGetLastError());
    A.ext32.alloc(next);
  }
  A.ext64.alloc(next);
  SEM_CHECK_CUDA(cudaStreamSynchronize(st));
}

template <typename T, int NP>
static void asm_solve_np(const AsmData &A, const Level &L, const T *r, T *z, T *ext,
                         cudaStream_t st) {
  using Sh = AsmShape<NP>;
  const int64_t g = (L.t.E + Sh::NEL - 1) / Sh::NEL;
  const T *S, *lam;
  if constexpr (sizeof(T) == 8) {
    S = A.S64.p;
    lam = A.lam64.p;
  } else {
    S = A.S32.p;
    lam = A.lam32.p;
  }
  asm_solve_kernel<T, NP><<<(int)(g < 152 * 16 ? g : 152 * 16), Sh::THREADS, 0, st>>>(L.t, S, lam,
                                                                                       r, z, ext);
  SEM_CHECK_CUDA(cudaGetLastError());
}

template <typename T>
void launch_asm(const AsmData &A, const Level &L, const T *r, T *z, cudaStream_t st) {
  T *ext;
  if constexpr (sizeof(T) == 8) ext = A.ext64.p;
  else ext = A.ext32.p;
  SEM_REQUIRE(ext != nullptr, "Schwarz data of this precision were not built");
  {
    // on the tensor cores while the extended element's n^2 pencils fit the 128
    // accumulator rows (N <= 8), else on the CUDA cores
    const bool tc = sizeof(T) == 4 && A.tc != 0 && L.t.Np <= 9;
    TraceScope ts(sizeof(T) == 8 ? "asm_f64"
                  : tc           ? (A.tc == 1 ? "asm_tc" : "asm_tf32")
                                 : "asm_f32",
                  L.t.N, st, 2);
    if constexpr (sizeof(T) == 4)
      if (tc) launch_asm_solve_tc(A, L, r, z, ext, A.tc == 1, st);
    if (!tc) switch (L.t.Np) {
      case 2: asm_solve_np<T, 2>(A, L, r, z, ext, st); break;
      case 3: asm_solve_np<T, 3>(A, L, r, z, ext, st); break;
      case 4: asm_solve_np<T, 4>(A, L, r, z, ext, st); break;
      case 5: asm_solve_np<T, 5>(A, L, r, z, ext, st); break;
      case 6: asm_solve_np<T, 6>(A, L, r, z, ext, st); break;
      case 7: asm_solve_np<T, 7>(A, L, r, z, ext, st); break;
      case 8: asm_solve_np<T, 8>(A, L, r, z, ext, st); break;
      case 9: asm_solve_np<T, 9>(A, L, r, z, ext, st); break;
      case 10: asm_solve_np<T, 10>(A, L, r, z, ext, st); break;
      default: fail(SEM_EINVAL, "Schwarz smoother: order %d unsupported", L.t.N);
    }
    asm_pull_kernel<T><<<vec_grid(L.t.nl), kVecThreads, 0, st>>>(L.t, ext, z);
    SEM_CHECK_CUDA(cudaGetLastError());
  }
  if constexpr (sizeof(T) == 4) {
    launch_planes_assemble(L, z, st);
  } else {
    launch_gs<double>(L, z, st);
    launch_mask<double>(L, z, st);
  }
}

template void launch_asm<double>(const AsmData &, const Level &, const double *, double *,
                                 cudaStream_t);
template void launch_asm<float>(const AsmData &, const Level &, const float *, float *,
                                cudaStream_t);

}  // namespace sem
