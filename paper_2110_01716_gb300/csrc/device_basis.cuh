// device_basis.cuh -- the trilinear metric shared by the setup kernels and
// the operator kernels that recompute geometric factors.
#pragma once

#include "common.cuh"

namespace sem {

// Metric of the trilinear map at reference point (r,s,t).
// V holds the 8 corners, corner (a,b,c) at V[3*(a+2b+4c) + m].
// With x_r, x_s, x_t the columns of the Jacobian, the rows of its inverse are
// (x_s x x_t, x_t x x_r, x_r x x_s) / det, det = x_r . (x_s x x_t), so
//   G_de = wgt * (c_d . c_e) / det,  c_0 = x_s x x_t, c_1 = x_t x x_r, c_2 = x_r x x_s,
//   B = wgt * det,  X = x(r,s,t).
// Output order of g: rr, rs, rt, ss, st, tt.
template <typename T>
__host__ __device__ __forceinline__ void trilinear_metric(const T *V, T r, T s, T t, T wgt,
                                                          T g[6], T *B, T X[3]) {
  const T lr0 = (T(1) - r) * T(0.5), lr1 = (T(1) + r) * T(0.5);
  const T ls0 = (T(1) - s) * T(0.5), ls1 = (T(1) + s) * T(0.5);
  const T lt0 = (T(1) - t) * T(0.5), lt1 = (T(1) + t) * T(0.5);
  T xr[3], xs[3], xt[3];
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    const T v000 = V[0 + m], v100 = V[3 + m], v010 = V[6 + m], v110 = V[9 + m];
    const T v001 = V[12 + m], v101 = V[15 + m], v011 = V[18 + m], v111 = V[21 + m];
    // edge differences along r, s, t, bilinearly weighted by the other two
    xr[m] = T(0.5) * (ls0 * lt0 * (v100 - v000) + ls1 * lt0 * (v110 - v010) +
                      ls0 * lt1 * (v101 - v001) + ls1 * lt1 * (v111 - v011));
    xs[m] = T(0.5) * (lr0 * lt0 * (v010 - v000) + lr1 * lt0 * (v110 - v100) +
                      lr0 * lt1 * (v011 - v001) + lr1 * lt1 * (v111 - v101));
    xt[m] = T(0.5) * (lr0 * ls0 * (v001 - v000) + lr1 * ls0 * (v101 - v100) +
                      lr0 * ls1 * (v011 - v010) + lr1 * ls1 * (v111 - v110));
    X[m] = lt0 * (ls0 * (lr0 * v000 + lr1 * v100) + ls1 * (lr0 * v010 + lr1 * v110)) +
           lt1 * (ls0 * (lr0 * v001 + lr1 * v101) + ls1 * (lr0 * v011 + lr1 * v111));
  }
  T c0[3], c1[3], c2[3];
  c0[0] = xs[1] * xt[2] - xs[2] * xt[1];
  c0[1] = xs[2] * xt[0] - xs[0] * xt[2];
  c0[2] = xs[0] * xt[1] - xs[1] * xt[0];
  c1[0] = xt[1] * xr[2] - xt[2] * xr[1];
  c1[1] = xt[2] * xr[0] - xt[0] * xr[2];
  c1[2] = xt[0] * xr[1] - xt[1] * xr[0];
  c2[0] = xr[1] * xs[2] - xr[2] * xs[1];
  c2[1] = xr[2] * xs[0] - xr[0] * xs[2];
  c2[2] = xr[0] * xs[1] - xr[1] * xs[0];
  const T det = xr[0] * c0[0] + xr[1] * c0[1] + xr[2] * c0[2];
  const T q = wgt / det;
  g[0] = q * (c0[0] * c0[0] + c0[1] * c0[1] + c0[2] * c0[2]);
  g[1] = q * (c0[0] * c1[0] + c0[1] * c1[1] + c0[2] * c1[2]);
  g[2] = q * (c0[0] * c2[0] + c0[1] * c2[1] + c0[2] * c2[2]);
  g[3] = q * (c1[0] * c1[0] + c1[1] * c1[1] + c1[2] * c1[2]);
  g[4] = q * (c1[0] * c2[0] + c1[1] * c2[1] + c1[2] * c2[2]);
  g[5] = q * (c2[0] * c2[0] + c2[1] * c2[1] + c2[2] * c2[2]);
  *B = wgt * det;
}

}  // namespace sem
