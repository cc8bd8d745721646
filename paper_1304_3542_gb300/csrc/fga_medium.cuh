// Velocity medium on the device: the tensor-product cubic B-spline whose
// coefficients are the velocity samples, c(x) = sum_i c_i prod_k beta3(u_k - i_k),
// u_k = (x_k - o_k)/h_k, with coefficient indices clamped on open axes and
// wrapped on periodic ones. The ray equations (Eqs. characline, dzQ, dzP) need
// c, grad c and the Hessian of c at the ray centre Q; they are evaluated in FP64
// from the 4^d coefficients around Q (read through the read-only path; the whole
// coefficient array is small enough to stay resident in L2).
#pragma once

#include "fga_internal.cuh"

namespace fga {

// Weights of the four taps i0-1 .. i0+2 for the fractional position t in [0,1),
// and their first and second derivatives in t (polynomial pieces of beta3).
__device__ __forceinline__ void spline_taps(double t, double w[4], double dw[4], double ddw[4]) {
  double t2 = t * t, t3 = t2 * t, s = 1.0 - t;
  const double sixth = 1.0 / 6.0;
  w[0] = s * s * s * sixth;
  w[1] = (3.0 * t3 - 6.0 * t2 + 4.0) * sixth;
  w[2] = (-3.0 * t3 + 3.0 * t2 + 3.0 * t + 1.0) * sixth;
  w[3] = t3 * sixth;
  dw[0] = -0.5 * s * s;
  dw[1] = 0.5 * (3.0 * t2 - 4.0 * t);
  dw[2] = 0.5 * (-3.0 * t2 + 2.0 * t + 1.0);
  dw[3] = 0.5 * t2;
  ddw[0] = s;
  ddw[1] = 3.0 * t - 2.0;
  ddw[2] = 1.0 - 3.0 * t;
  ddw[3] = t;
}

__device__ __forceinline__ void spline_taps_value(double t, double w[4]) {
  double t2 = t * t, t3 = t2 * t, s = 1.0 - t;
  const double sixth = 1.0 / 6.0;
  w[0] = s * s * s * sixth;
  w[1] = (3.0 * t3 - 6.0 * t2 + 4.0) * sixth;
  w[2] = (-3.0 * t3 + 3.0 * t2 + 3.0 * t + 1.0) * sixth;
  w[3] = t3 * sixth;
}

__device__ __forceinline__ int64_t tap_index(int64_t i, int64_t n, int periodic) {
  if (periodic) {
    int64_t r = i % n;
    return r < 0 ? r + n : r;
  }
  return i < 0 ? 0 : (i > n - 1 ? n - 1 : i);
}

struct Med {
  double c;
  double g[kMaxDim];
  double K[kMaxDim][kMaxDim];
};

// c, grad c, Hessian of c at x (dimension D = 1 or 2).
template <int D>
__device__ __forceinline__ void medium_eval(const GridDev& gd, const double* __restrict__ C,
                                            const double* x, Med& m) {
  double w[D][4], dw[D][4], ddw[D][4];
  int64_t idx[D][4];
#pragma unroll
  for (int k = 0; k < D; ++k) {
    double u = (x[k] - gd.o[k]) * gd.inv_h[k];
    double fl = floor(u);
    spline_taps(u - fl, w[k], dw[k], ddw[k]);
    int64_t i0 = (int64_t)fl - 1;
#pragma unroll
    for (int a = 0; a < 4; ++a) idx[k][a] = tap_index(i0 + a, gd.n[k], gd.periodic[k]);
  }
  if constexpr (D == 1) {
    double c = 0, c1 = 0, c2 = 0;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      double v = __ldg(C + idx[0][a]);
      c += w[0][a] * v;
      c1 += dw[0][a] * v;
      c2 += ddw[0][a] * v;
    }
    m.c = c;
    m.g[0] = c1 * gd.inv_h[0];
    m.K[0][0] = c2 * gd.inv_h[0] * gd.inv_h[0];
  } else {
    double r[4], rz[4], rzz[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const double* row = C + idx[0][a] * gd.n[1];
      double s0 = 0, s1 = 0, s2 = 0;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        double v = __ldg(row + idx[D - 1][b]);
        s0 += w[D - 1][b] * v;
        s1 += dw[D - 1][b] * v;
        s2 += ddw[D - 1][b] * v;
      }
      r[a] = s0;
      rz[a] = s1;
      rzz[a] = s2;
    }
    double c = 0, cx = 0, cz = 0, cxx = 0, cxz = 0, czz = 0;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      c += w[0][a] * r[a];
      cx += dw[0][a] * r[a];
      cz += w[0][a] * rz[a];
      cxx += ddw[0][a] * r[a];
      cxz += dw[0][a] * rz[a];
      czz += w[0][a] * rzz[a];
    }
    double ix = gd.inv_h[0], iz = gd.inv_h[D - 1];
    m.c = c;
    m.g[0] = cx * ix;
    m.g[D - 1] = cz * iz;
    m.K[0][0] = cxx * ix * ix;
    m.K[0][D - 1] = cxz * ix * iz;
    m.K[D - 1][0] = m.K[0][D - 1];
    m.K[D - 1][D - 1] = czz * iz * iz;
  }
}

// c(x) only.
template <int D>
__device__ __forceinline__ double medium_value(const GridDev& gd, const double* __restrict__ C,
                                               const double* x) {
  double w[D][4];
  int64_t idx[D][4];
#pragma unroll
  for (int k = 0; k < D; ++k) {
    double u = (x[k] - gd.o[k]) * gd.inv_h[k];
    double fl = floor(u);
    spline_taps_value(u - fl, w[k]);
    int64_t i0 = (int64_t)fl - 1;
#pragma unroll
    for (int a = 0; a < 4; ++a) idx[k][a] = tap_index(i0 + a, gd.n[k], gd.periodic[k]);
  }
  double c = 0;
  if constexpr (D == 1) {
#pragma unroll
    for (int a = 0; a < 4; ++a) c += w[0][a] * __ldg(C + idx[0][a]);
  } else {
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const double* row = C + idx[0][a] * gd.n[1];
      double s0 = 0;
#pragma unroll
      for (int b = 0; b < 4; ++b) s0 += w[D - 1][b] * __ldg(row + idx[D - 1][b]);
      c += w[0][a] * s0;
    }
  }
  return c;
}

}  // namespace fga
