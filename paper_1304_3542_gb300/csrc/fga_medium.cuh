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
  } else if constexpr (D == 3) {
    // contract z, then y, then x; s[ordz][ordy] after the first two, ord = derivative order
    double c = 0, cg[3] = {0, 0, 0}, ck[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      double y0 = 0, yz = 0, yzz = 0, yy = 0, yyz = 0, yyy = 0;  // sums over (b, c)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const double* row = C + (idx[0][a] * gd.n[1] + idx[1][b]) * gd.n[2];
        double s0 = 0, s1 = 0, s2 = 0;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          double v = __ldg(row + idx[2][e]);
          s0 += w[2][e] * v;
          s1 += dw[2][e] * v;
          s2 += ddw[2][e] * v;
        }
        y0 += w[1][b] * s0;
        yz += w[1][b] * s1;
        yzz += w[1][b] * s2;
        yy += dw[1][b] * s0;
        yyz += dw[1][b] * s1;
        yyy += ddw[1][b] * s0;
      }
      c += w[0][a] * y0;
      cg[0] += dw[0][a] * y0;
      cg[1] += w[0][a] * yy;
      cg[2] += w[0][a] * yz;
      ck[0][0] += ddw[0][a] * y0;
      ck[0][1] += dw[0][a] * yy;
      ck[0][2] += dw[0][a] * yz;
      ck[1][1] += w[0][a] * yyy;
      ck[1][2] += w[0][a] * yyz;
      ck[2][2] += w[0][a] * yzz;
    }
    m.c = c;
#pragma unroll
    for (int k = 0; k < 3; ++k) m.g[k] = cg[k] * gd.inv_h[k];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int l = k; l < 3; ++l) {
        m.K[k][l] = ck[k][l] * gd.inv_h[k] * gd.inv_h[l];
        m.K[l][k] = m.K[k][l];
      }
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

// ---------------------------------------------------------------------------
// The same spline as a table of polynomials, for the ray kernels. On the cell
// [i, i+1) x [j, j+1) (index units) c is a bicubic polynomial; the table holds its
// power-basis coefficients in the physical offsets tx = x - x_i, tz = z - z_j:
// c = sum_{k,l} a[k][l] tx^k tz^l, a = diag(h^-k) M^T Cij M diag(h^-l), where Cij are the
// 4 x 4 clamped/wrapped coefficients around the cell and M[a][k] is the power-basis
// matrix of beta3's four pieces (applied in the difference form of spline_power4). Cells run from -1 to n on each axis: below -1 (and
// from n up) all four taps of an open axis are clamped to the same sample, so c is
// constant along that axis there; such positions use cell -1 (or n) at offset 0, where
// the derivative coefficients along the axis vanish exactly (they are differences of
// equal samples). Evaluating value, gradient and Hessian takes about 90 FP64 flops
// instead of about 230 for the tap form. In 3D the cell is [i, i+1) x [j, j+1) x [k, k+1)
// and the tricubic's 64 coefficients a[kx][ky][l] multiply tx^kx ty^ky tz^l: about 360
// flops for value, gradient and Hessian instead of about 800 for the 64-tap form.

// Power-basis coefficients of sum_t C_t beta3-piece_t(t) on one cell from its four
// taps, written with differences so that a constant (or clamped) run of taps gives
// exactly zero derivative coefficients:
//   a0 = (C0 + 4 C1 + C2)/6, a1 = (C2 - C0)/2, a2 = (C0 - 2 C1 + C2)/2,
//   a3 = ((C3 - C0) + 3 (C1 - C2))/6.
__device__ __forceinline__ void spline_power4(double c0, double c1, double c2, double c3, double* a) {
  const double sixth = 1.0 / 6.0;
  a[0] = (c0 + 4.0 * c1 + c2) * sixth;
  a[1] = 0.5 * (c2 - c0);
  a[2] = 0.5 * ((c0 - c1) + (c2 - c1));
  a[3] = ((c3 - c0) + 3.0 * (c1 - c2)) * sixth;
}

// Coefficients of table cell ci (cell index + 1 on each axis) into a[4^D], scaled to
// physical offsets (2D: a[k][l] multiplies tx^k tz^l; 3D: see above).
template <int D>
__device__ __forceinline__ void medium_cell(const GridDev& gd, const double* __restrict__ C,
                                            const int64_t* ci, double* a) {
  int64_t idx[D][4];
#pragma unroll
  for (int k = 0; k < D; ++k)
#pragma unroll
    for (int t = 0; t < 4; ++t) idx[k][t] = tap_index(ci[k] - 2 + t, gd.n[k], gd.periodic[k]);
  if constexpr (D == 1) {
    spline_power4(C[idx[0][0]], C[idx[0][1]], C[idx[0][2]], C[idx[0][3]], a);
    double sc = 1.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      a[k] *= sc;
      sc *= gd.inv_h[0];
    }
  } else if constexpr (D == 3) {
    // the tap rows' polynomials in z, then in y, then in x: a[(kx * 4 + ky) * 4 + l]
    // multiplies tx^kx ty^ky tz^l
    double s[4][4][4], u[4][4][4];
#pragma unroll
    for (int rx = 0; rx < 4; ++rx)
#pragma unroll
      for (int ry = 0; ry < 4; ++ry) {
        const double* row = C + (idx[0][rx] * gd.n[1] + idx[1][ry]) * gd.n[2];
        spline_power4(row[idx[2][0]], row[idx[2][1]], row[idx[2][2]], row[idx[2][3]], s[rx][ry]);
      }
    double col[4];
#pragma unroll
    for (int rx = 0; rx < 4; ++rx)
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        spline_power4(s[rx][0][l], s[rx][1][l], s[rx][2][l], s[rx][3][l], col);
#pragma unroll
        for (int ky = 0; ky < 4; ++ky) u[rx][ky][l] = col[ky];
      }
    double sx = 1.0;
#pragma unroll
    for (int ky = 0; ky < 4; ++ky)
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        spline_power4(u[0][ky][l], u[1][ky][l], u[2][ky][l], u[3][ky][l], col);
#pragma unroll
        for (int kx = 0; kx < 4; ++kx) a[(kx * 4 + ky) * 4 + l] = col[kx];
      }
#pragma unroll
    for (int kx = 0; kx < 4; ++kx) {
      double sy = 1.0;
#pragma unroll
      for (int ky = 0; ky < 4; ++ky) {
        double sz = 1.0;
#pragma unroll
        for (int l = 0; l < 4; ++l) {
          a[(kx * 4 + ky) * 4 + l] *= sx * sy * sz;
          sz *= gd.inv_h[2];
        }
        sy *= gd.inv_h[1];
      }
      sx *= gd.inv_h[0];
    }
  } else {
    double s[4][4];  // s[tap row][l]: the row's polynomial in z
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const double* row = C + idx[0][r] * gd.n[1];
      spline_power4(row[idx[1][0]], row[idx[1][1]], row[idx[1][2]], row[idx[1][3]], s[r]);
    }
    double sx = 1.0;
    double col[4];
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      spline_power4(s[0][l], s[1][l], s[2][l], s[3][l], col);
#pragma unroll
      for (int k = 0; k < 4; ++k) a[k * 4 + l] = col[k];
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      double sz = 1.0;
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        a[k * 4 + l] *= sx * sz;
        sz *= gd.inv_h[1];
      }
      sx *= gd.inv_h[0];
    }
  }
}

// Table cell (index + 1) and physical offset of x along axis k. On an open axis the
// cell index is one rounding-down conversion of u = (x - o)/h, clamped to the table's
// cells -1 .. n in integer arithmetic; where it was clamped the offset is 0 (below cell
// -1 the spline is constant along the axis and cell -1 is evaluated at its left edge;
// cell n is constant, all its derivative coefficients being exact zeros). A position a
// rounding error below a cell boundary evaluates the neighbouring cell's polynomial at
// offset h: the spline is C2 there, so the two agree to within rounding.
// clamped is set where the position lies beyond cell -1 or n (the spline is constant
// along the axis there; the cell's cubic coefficient along the axis need not vanish, so
// a third derivative along the axis must be taken as 0 there, not from the cell).
__device__ __forceinline__ int64_t medium_cell_of(const GridDev& gd, int k, double x, double& off,
                                                  bool& clamped) {
  if (gd.periodic[k]) {
    const double u = (x - gd.o[k]) * gd.inv_h[k];
    double fl = floor(u);
    off = (u - fl) * gd.h[k];
    int64_t i = (int64_t)fl % gd.n[k];
    clamped = false;
    return (i < 0 ? i + gd.n[k] : i) + 1;
  }
  const double u = fma(x, gd.inv_h[k], gd.mo[k]);
  const int i = __double2int_rd(u);
  const int ic = min(max(i, -1), (int)gd.n[k]);
  off = (u - (double)ic) * gd.h[k];
  clamped = i != ic;
  if (clamped) off = 0.0;
  return (int64_t)ic + 1;
}
__device__ __forceinline__ int64_t medium_cell_of(const GridDev& gd, int k, double x, double& off) {
  bool clamped;
  return medium_cell_of(gd, k, x, off, clamped);
}

// Value, first derivative and half the second derivative of the cubic
// a0 + a1 t + a2 t^2 + a3 t^3 at t by Horner's scheme with derivatives (six fused
// multiply-adds).
__device__ __forceinline__ void horner3(double a0, double a1, double a2, double a3, double t,
                                        double& v, double& d1, double& d2h) {
  double w = fma(a3, t, a2);
  double d = fma(a3, t, w);
  w = fma(w, t, a1);
  d2h = fma(a3, t, d);
  d = fma(d, t, w);
  v = fma(w, t, a0);
  d1 = d;
}

// Value and first derivative of the cubic a0 + a1 t + a2 t^2 + a3 t^3 at t (five fused
// multiply-adds).
__device__ __forceinline__ void horner2d(double a0, double a1, double a2, double a3, double t,
                                         double& v, double& d1) {
  double w = fma(a3, t, a2);
  double d = fma(a3, t, w);
  w = fma(w, t, a1);
  d = fma(d, t, w);
  v = fma(w, t, a0);
  d1 = d;
}

// c, grad c, Hessian of c at x from the table gd.tab.
template <int D>
__device__ __forceinline__ void medium_eval_tab(const GridDev& gd, const double* x, Med& m) {
  if constexpr (D == 3) {
    double tx, ty, tz;
    const int64_t cx = medium_cell_of(gd, 0, x[0], tx);
    const int64_t cy = medium_cell_of(gd, 1, x[1], ty);
    const int64_t cz = medium_cell_of(gd, 2, x[2], tz);
    const double2* cell =
        reinterpret_cast<const double2*>(gd.tab) + ((cx * (gd.n[1] + 2) + cy) * (gd.n[2] + 2) + cz) * 32;
    // per power kx of tx: the (ky, l) square in tz, then in ty, with the derivatives
    // the Hessian needs (v: value, vy/vz: d/dy, d/dz, vyz: d2/dydz, hyy/hzz: half of
    // d2/dy2, d2/dz2)
    double v[4], vy[4], vz[4], vyz[4], hyy[4], hzz[4];
#pragma unroll
    for (int kx = 0; kx < 4; ++kx) {
      double r[4], rz[4], hz[4];
#pragma unroll
      for (int ky = 0; ky < 4; ++ky) {
        const double2 a01 = __ldg(cell + kx * 8 + ky * 2), a23 = __ldg(cell + kx * 8 + ky * 2 + 1);
        horner3(a01.x, a01.y, a23.x, a23.y, tz, r[ky], rz[ky], hz[ky]);
      }
      horner3(r[0], r[1], r[2], r[3], ty, v[kx], vy[kx], hyy[kx]);
      horner2d(rz[0], rz[1], rz[2], rz[3], ty, vz[kx], vyz[kx]);
      hzz[kx] = fma(fma(fma(hz[3], ty, hz[2]), ty, hz[1]), ty, hz[0]);
    }
    double hxx;
    horner3(v[0], v[1], v[2], v[3], tx, m.c, m.g[0], hxx);
    horner2d(vy[0], vy[1], vy[2], vy[3], tx, m.g[1], m.K[0][1]);
    horner2d(vz[0], vz[1], vz[2], vz[3], tx, m.g[2], m.K[0][2]);
    m.K[1][2] = fma(fma(fma(vyz[3], tx, vyz[2]), tx, vyz[1]), tx, vyz[0]);
    const double hy = fma(fma(fma(hyy[3], tx, hyy[2]), tx, hyy[1]), tx, hyy[0]);
    const double hz = fma(fma(fma(hzz[3], tx, hzz[2]), tx, hzz[1]), tx, hzz[0]);
    m.K[0][0] = 2.0 * hxx;
    m.K[1][1] = 2.0 * hy;
    m.K[2][2] = 2.0 * hz;
    m.K[1][0] = m.K[0][1];
    m.K[2][0] = m.K[0][2];
    m.K[2][1] = m.K[1][2];
  } else if constexpr (D == 1) {
    double t;
    const int64_t c0 = medium_cell_of(gd, 0, x[0], t);
    const double2* cell = reinterpret_cast<const double2*>(gd.tab) + c0 * 2;
    const double2 p01 = __ldg(cell), p23 = __ldg(cell + 1);
    double hh;
    horner3(p01.x, p01.y, p23.x, p23.y, t, m.c, m.g[0], hh);
    m.K[0][0] = 2.0 * hh;
  } else {
    double tx, tz;
    const int64_t cx = medium_cell_of(gd, 0, x[0], tx);
    const int64_t cz = medium_cell_of(gd, 1, x[1], tz);
    const double2* cell = reinterpret_cast<const double2*>(gd.tab) + (cx * (gd.n[1] + 2) + cz) * 8;
    // row k (power k of tx): its cubic in tz, with d/dz and (d2/dz2)/2
    double r[4], rz[4], hz[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const double2 a01 = __ldg(cell + 2 * k), a23 = __ldg(cell + 2 * k + 1);
      horner3(a01.x, a01.y, a23.x, a23.y, tz, r[k], rz[k], hz[k]);
    }
    double cxx_h, czz_h;
    horner3(r[0], r[1], r[2], r[3], tx, m.c, m.g[0], cxx_h);
    // d/dz and d2/dxdz: value and derivative in tx of the rz cubic
    double w = fma(rz[3], tx, rz[2]);
    double d = fma(rz[3], tx, w);
    w = fma(w, tx, rz[1]);
    d = fma(d, tx, w);
    m.g[1] = fma(w, tx, rz[0]);
    m.K[0][1] = d;
    m.K[1][0] = d;
    czz_h = fma(fma(fma(hz[3], tx, hz[2]), tx, hz[1]), tx, hz[0]);
    m.K[0][0] = 2.0 * cxx_h;
    m.K[1][1] = 2.0 * czz_h;
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
  } else if constexpr (D == 3) {
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const double* row = C + (idx[0][a] * gd.n[1] + idx[1][b]) * gd.n[2];
        double s0 = 0;
#pragma unroll
        for (int e = 0; e < 4; ++e) s0 += w[2][e] * __ldg(row + idx[2][e]);
        c += w[0][a] * w[1][b] * s0;
      }
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
