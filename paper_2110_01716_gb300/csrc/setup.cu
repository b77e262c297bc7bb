// setup.cu -- 1D basis, mesh construction, geometric factors, shared-node
// numbering and the Jacobi diagonal.
//
// Sec. 2, Eq. (2): nodal tensor-product basis on Gauss-Lobatto-Legendre (GLL)
// points with an isoparametric map; footnote 1: Dhat_il = h_l'(xi_i).
// Sec. 3 (pMG): J_il = coarse basis h_l evaluated at fine node xi_i.
#include <cmath>
#include <cstring>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"
#include "device_basis.cuh"

namespace sem {

// ------------------------------------------------------------------ basis (host)
// Legendre P_n at x by the Bonnet recurrence.
static double legendre(int n, double x) {
  double pm = 1.0, p = x;
  if (n == 0) return 1.0;
  for (int k = 2; k <= n; ++k) {
    double pn = ((2 * k - 1) * x * p - (k - 1) * pm) / k;
    pm = p;
    p = pn;
  }
  return p;
}

// GLL nodes are the zeros of q(x) = P_{N+1}(x) - P_{N-1}(x) = c (1 - x^2) P'_N(x),
// whose derivative is q'(x) = (2N+1) P_N(x).  Newton from the Chebyshev-Lobatto
// points converges to every zero including +-1.  Weights 2 / (N(N+1) P_N^2).
void gll_points(int N, double *xi, double *w) {
  for (int i = 0; i <= N; ++i) {
    double x = -std::cos(M_PI * i / N);
    if (i > 0 && i < N) {
      for (int it = 0; it < 200; ++it) {
        double q = legendre(N + 1, x) - legendre(N - 1, x);
        double dq = (2 * N + 1) * legendre(N, x);
        double dx = q / dq;
        x -= dx;
        if (std::fabs(dx) <= 2e-16) break;
      }
    }
    xi[i] = x;
  }
  for (int i = 0; i <= N; ++i) {
    double p = legendre(N, xi[i]);
    w[i] = 2.0 / (N * (N + 1.0) * p * p);
  }
}

// Closed form of the GLL derivative matrix (Deville, Fischer and Mund 2002).
void derivative_matrix(int N, const double *xi, double *D) {
  int Np = N + 1;
  for (int i = 0; i < Np; ++i)
    for (int l = 0; l < Np; ++l) {
      double v;
      if (i != l)
        v = legendre(N, xi[i]) / (legendre(N, xi[l]) * (xi[i] - xi[l]));
      else if (i == 0)
        v = -0.25 * N * (N + 1);
      else if (i == N)
        v = 0.25 * N * (N + 1);
      else
        v = 0.0;
      D[i * Np + l] = v;
    }
}

// Barycentric form of Lagrange interpolation (Berrut and Trefethen 2004):
// h_l(x) = (b_l / (x - z_l)) / sum_m b_m / (x - z_m), b_l = 1 / prod_{m != l}(z_l - z_m).
void interpolation_matrix(int Nf, int Nc, double *J) {
  double xf[SEM_MAX_ORDER + 1], xc[SEM_MAX_ORDER + 1], w[SEM_MAX_ORDER + 1],
      bw[SEM_MAX_ORDER + 1];
  gll_points(Nf, xf, w);
  gll_points(Nc, xc, w);
  for (int l = 0; l <= Nc; ++l) {
    double b = 1.0;
    for (int m = 0; m <= Nc; ++m)
      if (m != l) b *= xc[l] - xc[m];
    bw[l] = 1.0 / b;
  }
  for (int i = 0; i <= Nf; ++i) {
    int hit = -1;
    for (int l = 0; l <= Nc; ++l)
      if (xf[i] == xc[l]) hit = l;
    if (hit >= 0) {
      for (int l = 0; l <= Nc; ++l) J[i * (Nc + 1) + l] = (l == hit) ? 1.0 : 0.0;
      continue;
    }
    double den = 0.0;
    for (int l = 0; l <= Nc; ++l) den += bw[l] / (xf[i] - xc[l]);
    for (int l = 0; l <= Nc; ++l) J[i * (Nc + 1) + l] = bw[l] / (xf[i] - xc[l]) / den;
  }
}

Basis make_basis(int N) {
  Basis b;
  std::memset(&b, 0, sizeof(b));
  b.N = N;
  gll_points(N, b.xi, b.w);
  derivative_matrix(N, b.xi, b.D);
  for (int q = 0; q < (N + 1) * (N + 1); ++q) b.D32[q] = (float)b.D[q];
  return b;
}

// ------------------------------------------------------------------ kernels
// Geometric factors of every point from the element's 8 vertices (setup).
__global__ void geometry_kernel(Topo t, Basis bs, const double *__restrict__ verts,
                                double *__restrict__ G64, float *__restrict__ G32,
                                float2 *__restrict__ G2, int *__restrict__ bad) {
  for (uint32_t l = blockIdx.x * blockDim.x + threadIdx.x; l < (uint32_t)t.nl;
       l += gridDim.x * blockDim.x) {
    uint32_t e = t.div_np3.div(l);
    uint32_t p = l - e * (uint32_t)t.Np3;
    uint32_t jk = t.div_np.div(p);
    int i = (int)(p - jk * (uint32_t)t.Np);
    int k = (int)t.div_np.div(jk);
    int j = (int)(jk - (uint32_t)k * t.Np);
    double V[24];
#pragma unroll
    for (int q = 0; q < 24; ++q) V[q] = verts[(size_t)e * 24 + q];
    double g[6], B, X[3];
    double wgt = bs.w[i] * bs.w[j] * bs.w[k];
    trilinear_metric<double>(V, bs.xi[i], bs.xi[j], bs.xi[k], wgt, g, &B, X);
    if (!(B > 0.0)) atomicExch(bad, 1);
    size_t base = (size_t)e * 6 * t.Np3 + p;
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      if (G64) G64[base + (size_t)f * t.Np3] = g[f];
      if (G32) G32[base + (size_t)f * t.Np3] = (float)g[f];
      if (G2) {
        const float hi = (float)g[f];
        G2[base + (size_t)f * t.Np3] = make_float2(hi, (float)(g[f] - (double)hi));
      }
    }
  }
}

// Local diagonal of A_L in closed form from the stored or recomputed factors:
//   sum_a D_ai^2 Grr(a,j,k) + sum_b D_bj^2 Gss(i,b,k) + sum_c D_ck^2 Gtt(i,j,c)
//   + 2 (D_ii D_jj Grs + D_ii D_kk Grt + D_jj D_kk Gst)(i,j,k).
__global__ void local_diag_kernel(Topo t, Basis bs, const double *__restrict__ G,
                                  const double *__restrict__ verts, double *__restrict__ d) {
  const int Np = t.Np;
  const double *D = bs.D;
  for (uint32_t l = blockIdx.x * blockDim.x + threadIdx.x; l < (uint32_t)t.nl;
       l += gridDim.x * blockDim.x) {
    uint32_t e = t.div_np3.div(l);
    uint32_t p = l - e * (uint32_t)t.Np3;
    uint32_t jk = t.div_np.div(p);
    int i = (int)(p - jk * (uint32_t)Np);
    int k = (int)t.div_np.div(jk);
    int j = (int)(jk - (uint32_t)k * Np);
    auto factor = [&](int f, int a, int b, int c) -> double {
      int q = a + Np * (b + Np * c);
      if (G) return G[((size_t)e * 6 + f) * t.Np3 + q];
      double V[24], g[6], B, X[3];
      for (int s = 0; s < 24; ++s) V[s] = verts[(size_t)e * 24 + s];
      trilinear_metric<double>(V, bs.xi[a], bs.xi[b], bs.xi[c], bs.w[a] * bs.w[b] * bs.w[c], g,
                               &B, X);
      return g[f];
    };
    double s = 0.0;
    for (int a = 0; a < Np; ++a) {
      s += D[a * Np + i] * D[a * Np + i] * factor(0, a, j, k);
      s += D[a * Np + j] * D[a * Np + j] * factor(3, i, a, k);
      s += D[a * Np + k] * D[a * Np + k] * factor(5, i, j, a);
    }
    double Di = D[i * Np + i], Dj = D[j * Np + j], Dk = D[k * Np + k];
    if (Di != 0.0 && Dj != 0.0) s += 2.0 * Di * Dj * factor(1, i, j, k);
    if (Di != 0.0 && Dk != 0.0) s += 2.0 * Di * Dk * factor(2, i, j, k);
    if (Dj != 0.0 && Dk != 0.0) s += 2.0 * Dj * Dk * factor(4, i, j, k);
    d[l] = s;
  }
}

__global__ void invert_diag_kernel(Topo t, const double *__restrict__ d, double *__restrict__ d64,
                                   float *__restrict__ d32) {
  for (uint32_t l = blockIdx.x * blockDim.x + threadIdx.x; l < (uint32_t)t.nl;
       l += gridDim.x * blockDim.x) {
    PointInfo q = point_info(l, t);
    double v = q.mask != 0.0f ? 1.0 / d[l] : 0.0;
    if (d64) d64[l] = v;
    if (d32) d32[l] = (float)v;
  }
}

// Per-point fields of the mesh (coordinates, mass, multiplicity, mask).
__global__ void field_kernel(Topo t, Basis bs, int which, const double *__restrict__ verts,
                             double *__restrict__ out) {
  for (uint32_t l = blockIdx.x * blockDim.x + threadIdx.x; l < (uint32_t)t.nl;
       l += gridDim.x * blockDim.x) {
    PointInfo q = point_info(l, t);
    double v;
    if (which == SEM_FIELD_MULT) {
      v = 1.0 / (double)q.inv_mult;
    } else if (which == SEM_FIELD_MASK) {
      v = q.mask;
    } else {
      double V[24], g[6], B, X[3];
      for (int s = 0; s < 24; ++s) V[s] = verts[(size_t)q.e * 24 + s];
      trilinear_metric<double>(V, bs.xi[q.i], bs.xi[q.j], bs.xi[q.k],
                               bs.w[q.i] * bs.w[q.j] * bs.w[q.k], g, &B, X);
      v = which == SEM_FIELD_MASS ? B : X[which];
    }
    out[l] = v;
  }
}

static int grid_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  const int64_t cap = 152 * 32;
  return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

void launch_field(const Level &L, int which, double *out, cudaStream_t st) {
  if (which == SEM_FIELD_DINV) {
    SEM_CHECK_CUDA(cudaMemcpyAsync(out, L.dinv64.p, L.t.nl * sizeof(double),
                                   cudaMemcpyDeviceToDevice, st));
    return;
  }
  field_kernel<<<grid_for(L.t.nl, 256), 256, 0, st>>>(L.t, L.basis, which, L.verts.p, out);
  SEM_CHECK_CUDA(cudaGetLastError());
}

// ------------------------------------------------------------------ level build
static Topo make_topo(int ex, int ey, int ez, int N, int bc) {
  Topo t;
  t.ex = ex; t.ey = ey; t.ez = ez; t.N = N; t.Np = N + 1;
  t.Np3 = t.Np * t.Np * t.Np;
  t.bc = bc;
  t.E = (int64_t)ex * ey * ez;
  t.nl = t.E * t.Np3;
  t.ng = ((int64_t)ex * N + 1) * ((int64_t)ey * N + 1) * ((int64_t)ez * N + 1);
  t.div_np3 = FastDiv((uint32_t)t.Np3);
  t.div_np = FastDiv((uint32_t)t.Np);
  t.div_ex = FastDiv((uint32_t)ex);
  t.div_ey = FastDiv((uint32_t)ey);
  return t;
}

// Unique ids of the nodes shared by more than one element, ascending.  A node
// of lattice coordinate g along a direction is shared there when g is a
// multiple of N strictly inside the box.
static std::vector<int32_t> shared_node_table(const Topo &t) {
  std::vector<int32_t> out;
  int64_t nx = (int64_t)t.ex * t.N + 1, ny = (int64_t)t.ey * t.N + 1, nz = (int64_t)t.ez * t.N + 1;
  auto on_iface = [&](int64_t g, int64_t n) { return g % t.N == 0 && g > 0 && g < n - 1; };
  for (int64_t gz = 0; gz < nz; ++gz) {
    bool sz = on_iface(gz, nz);
    for (int64_t gy = 0; gy < ny; ++gy) {
      bool sy = on_iface(gy, ny);
      if (sz || sy) {
        for (int64_t gx = 0; gx < nx; ++gx) out.push_back((int32_t)(gx + nx * (gy + ny * gz)));
      } else {
        for (int64_t gx = t.N; gx < nx - 1; gx += t.N) out.push_back((int32_t)(gx + nx * (gy + ny * gz)));
      }
    }
  }
  return out;
}

void build_level(Level &L, int ex, int ey, int ez, int N, int bc, int geom, int arith,
                 const double *verts_host, bool want_g32, cudaStream_t st) {
  SEM_REQUIRE(ex >= 1 && ey >= 1 && ez >= 1, "element counts must be >= 1 (got %d %d %d)", ex,
              ey, ez);
  SEM_REQUIRE(N >= 1 && N <= SEM_MAX_ORDER, "order N=%d outside [1, %d]", N, SEM_MAX_ORDER);
  SEM_REQUIRE(bc == SEM_DIRICHLET || bc == SEM_NEUMANN, "unknown boundary condition %d", bc);
  SEM_REQUIRE(geom == SEM_GEOM_STORED || geom == SEM_GEOM_TRILINEAR, "unknown geometry mode %d",
              geom);
  SEM_REQUIRE(arith == SEM_ARITH_PAIR || arith == SEM_ARITH_NATIVE, "unknown FP64 arithmetic %d",
              arith);
  Topo t = make_topo(ex, ey, ez, N, bc);
  SEM_REQUIRE(t.nl <= 0x7fffffffLL && t.ng <= 0x7fffffffLL,
              "mesh too large: %lld local points (limit 2^31-1)", (long long)t.nl);
  L.t = t;
  L.basis = make_basis(N);
  L.geom = geom;
  L.arith = arith;
  size_t nv = (size_t)(ex + 1) * (ey + 1) * (ez + 1);
  L.verts_host.assign(verts_host, verts_host + 3 * nv);
  // per-element corners
  std::vector<double> ev((size_t)t.E * 24);
  for (int iz = 0; iz < ez; ++iz)
    for (int iy = 0; iy < ey; ++iy)
      for (int ix = 0; ix < ex; ++ix) {
        size_t e = ix + (size_t)ex * (iy + (size_t)ey * iz);
        for (int c = 0; c < 2; ++c)
          for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a) {
              size_t v = (ix + a) + (size_t)(ex + 1) * ((iy + b) + (size_t)(ey + 1) * (iz + c));
              for (int m = 0; m < 3; ++m) ev[e * 24 + 3 * (a + 2 * b + 4 * c) + m] = verts_host[3 * v + m];
            }
      }
  L.verts.alloc(ev.size());
  SEM_CHECK_CUDA(cudaMemcpyAsync(L.verts.p, ev.data(), ev.size() * sizeof(double),
                                 cudaMemcpyHostToDevice, st));
  L.err.alloc(1);
  SEM_CHECK_CUDA(cudaMemsetAsync(L.err.p, 0, sizeof(int), st));
  DevBuf<int> bad;
  bad.alloc(1);
  SEM_CHECK_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), st));
  // geometric factors: always computed once (they also give the diagonal)
  DevBuf<double> Gtmp;
  double *G = nullptr;
  if (geom == SEM_GEOM_STORED && arith == SEM_ARITH_NATIVE) {
    L.G64.alloc((size_t)t.E * 6 * t.Np3);
    G = L.G64.p;
  } else {
    Gtmp.alloc((size_t)t.E * 6 * t.Np3);
    G = Gtmp.p;
  }
  if (geom == SEM_GEOM_STORED && arith == SEM_ARITH_PAIR) L.G2.alloc((size_t)t.E * 6 * t.Np3);
  if (want_g32) L.G32.alloc((size_t)t.E * 6 * t.Np3);
  geometry_kernel<<<grid_for(t.nl, 256), 256, 0, st>>>(t, L.basis, L.verts.p, G, L.G32.p, L.G2.p,
                                                       bad.p);
  SEM_CHECK_CUDA(cudaGetLastError());
  int hbad = 0;
  SEM_CHECK_CUDA(cudaMemcpyAsync(&hbad, bad.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  SEM_CHECK_CUDA(cudaStreamSynchronize(st));
  SEM_REQUIRE(hbad == 0, "an element has a non-positive Jacobian determinant (folded mesh)");
  // gather-scatter numbering
  std::vector<int32_t> sh = shared_node_table(t);
  L.n_shared = (int64_t)sh.size();
  L.shared_nodes.alloc(sh.size());
  if (!sh.empty())
    SEM_CHECK_CUDA(cudaMemcpyAsync(L.shared_nodes.p, sh.data(), sh.size() * sizeof(int32_t),
                                   cudaMemcpyHostToDevice, st));
  // Jacobi diagonal: local closed form, assembled, inverted and masked
  DevBuf<double> d;
  d.alloc(t.nl);
  local_diag_kernel<<<grid_for(t.nl, 256), 256, 0, st>>>(t, L.basis, G, L.verts.p, d.p);
  SEM_CHECK_CUDA(cudaGetLastError());
  launch_gs<double>(L, d.p, st);
  L.dinv64.alloc(t.nl);
  if (want_g32) L.dinv32.alloc(t.nl);
  invert_diag_kernel<<<grid_for(t.nl, 256), 256, 0, st>>>(t, d.p, L.dinv64.p, L.dinv32.p);
  SEM_CHECK_CUDA(cudaGetLastError());
  SEM_CHECK_CUDA(cudaStreamSynchronize(st));
}

void level_fp64_factors(const Level &L, DevBuf<double> &out, cudaStream_t st) {
  const Topo &t = L.t;
  DevBuf<int> bad;
  bad.alloc(1);
  SEM_CHECK_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), st));
  out.alloc((size_t)t.E * 6 * t.Np3);
  geometry_kernel<<<grid_for(t.nl, 256), 256, 0, st>>>(t, L.basis, L.verts.p, out.p, nullptr,
                                                       nullptr, bad.p);
  SEM_CHECK_CUDA(cudaGetLastError());
  SEM_CHECK_CUDA(cudaStreamSynchronize(st));
}

// One thread per element: scale = max |G| over the element's six factors and
// points, in FP32 (1 if all are zero); stored value = G / scale rounded once
// from FP64 to FP16 or BF16 (nearest, ties to even).
__global__ void g16_kernel(int64_t E, int Np3, int kind, const double *__restrict__ G,
                           uint16_t *__restrict__ G16, float *__restrict__ scale) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double *g = G + e * 6 * Np3;
    double m = 0.0;
    for (int p = 0; p < 6 * Np3; ++p) m = fmax(m, fabs(g[p]));
    const float sc = m > 0.0 ? (float)m : 1.0f;
    scale[e] = sc;
    uint16_t *o = G16 + e * 6 * Np3;
    for (int p = 0; p < 6 * Np3; ++p) {
      const double v = g[p] / (double)sc;
      o[p] = kind == SEM_F16 ? __half_as_ushort(__double2half(v))
                             : __bfloat16_as_ushort(__double2bfloat16(v));
    }
  }
}

void level_ensure_dinv32(Level &L, cudaStream_t st) {
  if (L.dinv32.p) return;
  const Topo &t = L.t;
  DevBuf<double> g;
  level_fp64_factors(L, g, st);
  L.dinv32.alloc(t.nl);
  DevBuf<double> d;
  d.alloc(t.nl);
  local_diag_kernel<<<grid_for(t.nl, 256), 256, 0, st>>>(t, L.basis, g.p, L.verts.p, d.p);
  SEM_CHECK_CUDA(cudaGetLastError());
  launch_gs<double>(L, d.p, st);
  invert_diag_kernel<<<grid_for(t.nl, 256), 256, 0, st>>>(t, d.p, nullptr, L.dinv32.p);
  SEM_CHECK_CUDA(cudaGetLastError());
  SEM_CHECK_CUDA(cudaStreamSynchronize(st));
}

void level_ensure_g16(Level &L, int kind, cudaStream_t st) {
  SEM_REQUIRE(kind == SEM_F16 || kind == SEM_BF16, "16-bit kind must be SEM_F16 or SEM_BF16");
  SEM_REQUIRE(L.geom == SEM_GEOM_STORED, "16-bit factors need stored geometry");
  level_ensure_dinv32(L, st);
  const int s = kind == SEM_F16 ? 0 : 1;
  if (L.G16[s].p) return;
  const Topo &t = L.t;
  DevBuf<double> g;
  level_fp64_factors(L, g, st);
  L.G16[s].alloc((size_t)t.E * 6 * t.Np3);
  L.G16scale[s].alloc((size_t)t.E);
  g16_kernel<<<grid_for(t.E, 128), 128, 0, st>>>(t.E, t.Np3, kind, g.p, L.G16[s].p,
                                                 L.G16scale[s].p);
  SEM_CHECK_CUDA(cudaGetLastError());
  SEM_CHECK_CUDA(cudaStreamSynchronize(st));
}

void level_ensure_f32(Level &L, cudaStream_t st) {
  const Topo &t = L.t;
  const bool need_g32 = L.geom == SEM_GEOM_STORED && !L.G32.p;
  if (L.dinv32.p && !need_g32) return;
  // FP64 factors again (temporarily): they give the FP32 copies and the diagonal
  DevBuf<int> bad;
  bad.alloc(1);
  SEM_CHECK_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), st));
  DevBuf<double> g;
  g.alloc((size_t)t.E * 6 * t.Np3);
  if (need_g32) L.G32.alloc((size_t)t.E * 6 * t.Np3);
  geometry_kernel<<<grid_for(t.nl, 256), 256, 0, st>>>(t, L.basis, L.verts.p, g.p,
                                                       need_g32 ? L.G32.p : nullptr, nullptr, bad.p);
  SEM_CHECK_CUDA(cudaGetLastError());
  if (!L.dinv32.p) {
    L.dinv32.alloc(t.nl);
    DevBuf<double> d;
    d.alloc(t.nl);
    local_diag_kernel<<<grid_for(t.nl, 256), 256, 0, st>>>(t, L.basis, g.p, L.verts.p, d.p);
    SEM_CHECK_CUDA(cudaGetLastError());
    launch_gs<double>(L, d.p, st);
    invert_diag_kernel<<<grid_for(t.nl, 256), 256, 0, st>>>(t, d.p, nullptr, L.dinv32.p);
    SEM_CHECK_CUDA(cudaGetLastError());
  }
  SEM_CHECK_CUDA(cudaStreamSynchronize(st));
}

}  // namespace sem
