// Vector-Jacobian product of the FGA ray right-hand side (rhs in fga_ray_rhs.cuh) and
// the transposed spline evaluation, used by the adjoint kernel.
#pragma once

#include "fga_internal.cuh"
#include "fga_medium.cuh"
#include "fga_ray_rhs.cuh"

namespace fga {
namespace adj {

struct cx {
  double r, i;
};
__device__ __forceinline__ cx mk(double r, double i) { return cx{r, i}; }
__device__ __forceinline__ cx operator+(cx a, cx b) { return cx{a.r + b.r, a.i + b.i}; }
__device__ __forceinline__ cx operator-(cx a, cx b) { return cx{a.r - b.r, a.i - b.i}; }
__device__ __forceinline__ cx operator*(cx a, cx b) {
  return cx{a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r};
}
__device__ __forceinline__ cx operator*(double s, cx a) { return cx{s * a.r, s * a.i}; }
__device__ __forceinline__ cx conj(cx a) { return cx{a.r, -a.i}; }
// a * conj(b)
__device__ __forceinline__ cx mulc(cx a, cx b) { return cx{a.r * b.r + a.i * b.i, a.i * b.r - a.r * b.i}; }
// Re(a * conj(b)): the adjoint of a real factor x in w = x b given w's adjoint a
__device__ __forceinline__ double rdot(cx a, cx b) { return a.r * b.r + a.i * b.i; }

// c, grad c, Hessian and third derivatives of the spline at x, with the tap indices and
// weights kept for the transposed scatter.
template <int D>
struct MedAD {
  // third derivatives: 2D xxx, xxz, xzz, zzz; 3D the ten of t3_index
  double c, g[D], K[D][D], T3[D == 3 ? 10 : 4];
  int64_t idx[D][4];
  double w[D][4], dw[D][4], ddw[D][4], dddw[D][4];
};

// Index of the third derivative d^3 c / dx_i dx_j dx_k (3D) among the ten distinct ones,
// ordered by the derivative orders (nx, ny, nz) as xxx, xxy, xxz, xyy, xyz, xzz, yyy,
// yyz, yzz, zzz.
__host__ __device__ constexpr int t3_index(int i, int j, int k) {
  const int nx = (i == 0) + (j == 0) + (k == 0), ny = (i == 1) + (j == 1) + (k == 1);
  // position of (nx, ny, nz) in the list above: orders with larger nx first, then larger ny
  return nx == 3 ? 0 : nx == 2 ? (ny == 1 ? 1 : 2) : nx == 1 ? (ny == 2 ? 3 : ny == 1 ? 4 : 5)
                                                             : (ny == 3 ? 6 : ny == 2 ? 7 : ny == 1 ? 8 : 9);
}

template <int D>
__device__ __forceinline__ void medium_ad(const GridDev& gd, const double* __restrict__ C,
                                          const double* x, MedAD<D>& m) {
#pragma unroll
  for (int k = 0; k < D; ++k) {
    double u = (x[k] - gd.o[k]) * gd.inv_h[k];
    double fl = floor(u);
    spline_taps(u - fl, m.w[k], m.dw[k], m.ddw[k]);
    m.dddw[k][0] = -1.0;
    m.dddw[k][1] = 3.0;
    m.dddw[k][2] = -3.0;
    m.dddw[k][3] = 1.0;
    int64_t i0 = (int64_t)fl - 1;
#pragma unroll
    for (int a = 0; a < 4; ++a) m.idx[k][a] = tap_index(i0 + a, gd.n[k], gd.periodic[k]);
  }
  if constexpr (D == 1) {
    double c = 0, c1 = 0, c2 = 0, c3 = 0;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      double v = __ldg(C + m.idx[0][a]);
      c += m.w[0][a] * v;
      c1 += m.dw[0][a] * v;
      c2 += m.ddw[0][a] * v;
      c3 += m.dddw[0][a] * v;
    }
    double ih = gd.inv_h[0];
    m.c = c;
    m.g[0] = c1 * ih;
    m.K[0][0] = c2 * ih * ih;
    m.T3[0] = c3 * ih * ih * ih;
    m.T3[1] = m.T3[2] = m.T3[3] = 0.0;
  } else if constexpr (D == 3) {
    // contract z (orders 0..3), then y, then x, keeping every combination of total order <= 3
    double t[4][10];  // [x tap][(ny, nz) with ny + nz <= 3]: 00 01 02 03 10 11 12 20 21 30
#pragma unroll
    for (int a = 0; a < 4; ++a) {
#pragma unroll
      for (int e = 0; e < 10; ++e) t[a][e] = 0.0;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const double* row = C + (m.idx[0][a] * gd.n[1] + m.idx[1][b]) * gd.n[2];
        double sz[4] = {0, 0, 0, 0};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const double v = __ldg(row + m.idx[2][e]);
          sz[0] += m.w[2][e] * v;
          sz[1] += m.dw[2][e] * v;
          sz[2] += m.ddw[2][e] * v;
          sz[3] += m.dddw[2][e] * v;
        }
        const double wy[4] = {m.w[1][b], m.dw[1][b], m.ddw[1][b], m.dddw[1][b]};
        t[a][0] += wy[0] * sz[0];
        t[a][1] += wy[0] * sz[1];
        t[a][2] += wy[0] * sz[2];
        t[a][3] += wy[0] * sz[3];
        t[a][4] += wy[1] * sz[0];
        t[a][5] += wy[1] * sz[1];
        t[a][6] += wy[1] * sz[2];
        t[a][7] += wy[2] * sz[0];
        t[a][8] += wy[2] * sz[1];
        t[a][9] += wy[3] * sz[0];
      }
    }
    // out[(nx, ny, nz)] = sum_a wx^(nx)_a t[a][(ny, nz)]
    auto contract = [&](int nx, int e) {
      double v = 0.0;
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const double wx = nx == 0 ? m.w[0][a] : nx == 1 ? m.dw[0][a] : nx == 2 ? m.ddw[0][a] : m.dddw[0][a];
        v += wx * t[a][e];
      }
      return v;
    };
    const double ix = gd.inv_h[0], iy = gd.inv_h[1], iz = gd.inv_h[2];
    m.c = contract(0, 0);
    m.g[0] = contract(1, 0) * ix;
    m.g[1] = contract(0, 4) * iy;
    m.g[2] = contract(0, 1) * iz;
    m.K[0][0] = contract(2, 0) * ix * ix;
    m.K[1][1] = contract(0, 7) * iy * iy;
    m.K[2][2] = contract(0, 2) * iz * iz;
    m.K[0][1] = m.K[1][0] = contract(1, 4) * ix * iy;
    m.K[0][2] = m.K[2][0] = contract(1, 1) * ix * iz;
    m.K[1][2] = m.K[2][1] = contract(0, 5) * iy * iz;
    m.T3[0] = contract(3, 0) * ix * ix * ix;  // xxx
    m.T3[1] = contract(2, 4) * ix * ix * iy;  // xxy
    m.T3[2] = contract(2, 1) * ix * ix * iz;  // xxz
    m.T3[3] = contract(1, 7) * ix * iy * iy;  // xyy
    m.T3[4] = contract(1, 5) * ix * iy * iz;  // xyz
    m.T3[5] = contract(1, 2) * ix * iz * iz;  // xzz
    m.T3[6] = contract(0, 9) * iy * iy * iy;  // yyy
    m.T3[7] = contract(0, 8) * iy * iy * iz;  // yyz
    m.T3[8] = contract(0, 6) * iy * iz * iz;  // yzz
    m.T3[9] = contract(0, 3) * iz * iz * iz;  // zzz
  } else {
    double r[4][4];  // row sums along z: value, d, dd, ddd
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const double* row = C + m.idx[0][a] * gd.n[1];
      double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        double v = __ldg(row + m.idx[1][b]);
        s0 += m.w[1][b] * v;
        s1 += m.dw[1][b] * v;
        s2 += m.ddw[1][b] * v;
        s3 += m.dddw[1][b] * v;
      }
      r[a][0] = s0;
      r[a][1] = s1;
      r[a][2] = s2;
      r[a][3] = s3;
    }
    double c = 0, cx_ = 0, cz = 0, cxx = 0, cxz = 0, czz = 0, cxxx = 0, cxxz = 0, cxzz = 0, czzz = 0;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      c += m.w[0][a] * r[a][0];
      cx_ += m.dw[0][a] * r[a][0];
      cz += m.w[0][a] * r[a][1];
      cxx += m.ddw[0][a] * r[a][0];
      cxz += m.dw[0][a] * r[a][1];
      czz += m.w[0][a] * r[a][2];
      cxxx += m.dddw[0][a] * r[a][0];
      cxxz += m.ddw[0][a] * r[a][1];
      cxzz += m.dw[0][a] * r[a][2];
      czzz += m.w[0][a] * r[a][3];
    }
    double ix = gd.inv_h[0], iz = gd.inv_h[1];
    m.c = c;
    m.g[0] = cx_ * ix;
    m.g[1] = cz * iz;
    m.K[0][0] = cxx * ix * ix;
    m.K[0][1] = m.K[1][0] = cxz * ix * iz;
    m.K[1][1] = czz * iz * iz;
    m.T3[0] = cxxx * ix * ix * ix;
    m.T3[1] = cxxz * ix * ix * iz;
    m.T3[2] = cxzz * ix * iz * iz;
    m.T3[3] = czzz * iz * iz * iz;
  }
}

// Transposed spline: adjoints (cb, gb, Kb) of (c, grad c, Hessian) at a point -> the
// coefficient gradient (added without waiting for the result) and the point's adjoint Qb.
template <int D>
__device__ __forceinline__ void medium_ad_transpose(const GridDev& gd, const MedAD<D>& m, double cb,
                                                    const double* gb, const double (*Kb)[D],
                                                    double* Qb, double* __restrict__ gradC) {
  if constexpr (D == 3) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      double q = cb * m.g[k];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        q += gb[i] * m.K[i][k];
#pragma unroll
        for (int j = 0; j < 3; ++j) q += Kb[i][j] * m.T3[t3_index(i, j, k)];
      }
      Qb[k] += q;
    }
    // coefficient (a, b, e) receives al w_e + be w'_e + ga w''_e, the x and y factors of
    // the ten terms gathered per (a, b)
    const double ix = gd.inv_h[0], iy = gd.inv_h[1], iz = gd.inv_h[2];
    const double kxy = (Kb[0][1] + Kb[1][0]) * ix * iy, kxz = (Kb[0][2] + Kb[2][0]) * ix * iz,
                 kyz = (Kb[1][2] + Kb[2][1]) * iy * iz;
    const double kxx = Kb[0][0] * ix * ix, kyy = Kb[1][1] * iy * iy, kzz = Kb[2][2] * iz * iz;
    const double gx = gb[0] * ix, gy = gb[1] * iy, gz = gb[2] * iz;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const double wa = m.w[0][a], da = m.dw[0][a], dda = m.ddw[0][a];
        const double wb = m.w[1][b], db = m.dw[1][b], ddb = m.ddw[1][b];
        const double ww = wa * wb;
        const double al = cb * ww + gx * da * wb + gy * wa * db + kxx * dda * wb + kyy * wa * ddb +
                          kxy * da * db;
        const double be = gz * ww + kxz * da * wb + kyz * wa * db;
        const double ga = kzz * ww;
        double* row = gradC + (m.idx[0][a] * gd.n[1] + m.idx[1][b]) * gd.n[2];
#pragma unroll
        for (int e = 0; e < 4; ++e)
          red_add_f64(row + m.idx[2][e], al * m.w[2][e] + be * m.dw[2][e] + ga * m.ddw[2][e]);
      }
  } else if constexpr (D == 1) {
    Qb[0] += cb * m.g[0] + gb[0] * m.K[0][0] + Kb[0][0] * m.T3[0];
    double ih = gd.inv_h[0];
#pragma unroll
    for (int a = 0; a < 4; ++a)
      red_add_f64(gradC + m.idx[0][a],
                  cb * m.w[0][a] + gb[0] * m.dw[0][a] * ih + Kb[0][0] * m.ddw[0][a] * ih * ih);
  } else {
    const double kxz = Kb[0][1] + Kb[1][0];
    Qb[0] += cb * m.g[0] + gb[0] * m.K[0][0] + gb[1] * m.K[0][1] + Kb[0][0] * m.T3[0] +
             kxz * m.T3[1] + Kb[1][1] * m.T3[2];
    Qb[1] += cb * m.g[1] + gb[0] * m.K[0][1] + gb[1] * m.K[1][1] + Kb[0][0] * m.T3[1] +
             kxz * m.T3[2] + Kb[1][1] * m.T3[3];
    const double ix = gd.inv_h[0], iz = gd.inv_h[1];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const double wa = m.w[0][a], da = m.dw[0][a] * ix, dda = m.ddw[0][a] * ix * ix;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const double wb = m.w[1][b], db = m.dw[1][b] * iz, ddb = m.ddw[1][b] * iz * iz;
        red_add_f64(gradC + m.idx[0][a] * gd.n[1] + m.idx[1][b],
                    cb * wa * wb + gb[0] * da * wb + gb[1] * wa * db + Kb[0][0] * dda * wb +
                        kxz * da * db + Kb[1][1] * wa * ddb);
      }
    }
  }
}

// yb += (d f/d y)^T kb and gradC += (d f/d C)^T kb for the right-hand side f of rhs<D>
// (1D and 3D; 2D uses rhs2_vjp below).
template <int D>
__device__ void rhs_vjp(const GridDev& gd, const double* __restrict__ C, const double* y,
                        const double* kb, double* yb, double* __restrict__ gradC) {
  using Lo = Layout<D>;
  // ---- forward intermediates ----
  MedAD<D> m;
  medium_ad<D>(gd, C, y + Lo::Q, m);
  double P[D], n[D];
  double pn2 = 0;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    P[i] = y[Lo::P + i];
    pn2 += P[i] * P[i];
  }
  const double rinv = rsqrt_nr(pn2), pn = pn2 * rinv, cop = m.c * rinv;
  double ng = 0;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    n[i] = P[i] * rinv;
    ng += n[i] * m.g[i];
  }
  cx A[D][D], B[D][D], ag[D], bn[D], ak[D][D], Ad[D][D], Bd[D][D];
#pragma unroll
  for (int j = 0; j < D; ++j)
#pragma unroll
    for (int k = 0; k < D; ++k) {
      A[j][k] = mk(y[Lo::AR + j * D + k], y[Lo::AI + j * D + k]);
      B[j][k] = mk(y[Lo::BR + j * D + k], y[Lo::BI + j * D + k]);
    }
#pragma unroll
  for (int j = 0; j < D; ++j) {
    ag[j] = mk(0, 0);
    bn[j] = mk(0, 0);
#pragma unroll
    for (int l = 0; l < D; ++l) {
      ag[j] = ag[j] + m.g[l] * A[j][l];
      bn[j] = bn[j] + n[l] * B[j][l];
    }
#pragma unroll
    for (int k = 0; k < D; ++k) {
      ak[j][k] = mk(0, 0);
#pragma unroll
      for (int l = 0; l < D; ++l) ak[j][k] = ak[j][k] + m.K[l][k] * A[j][l];
      Ad[j][k] = n[k] * ag[j] + cop * (B[j][k] - n[k] * bn[j]);
      Bd[j][k] = -1.0 * (pn * ak[j][k] + m.g[k] * bn[j]);
    }
  }
  cx Z[D][D], Zd[D][D];
#pragma unroll
  for (int j = 0; j < D; ++j)
#pragma unroll
    for (int k = 0; k < D; ++k) {
      Z[j][k] = A[j][k] + mk(-B[j][k].i, B[j][k].r);
      Zd[j][k] = Ad[j][k] + mk(-Bd[j][k].i, Bd[j][k].r);
    }
  cx N, Dt;
  cx Cf[D == 3 ? 3 : 1][D == 3 ? 3 : 1];  // 3D: the cofactors of Z
  if constexpr (D == 1) {
    N = Zd[0][0];
    Dt = Z[0][0];
  } else if constexpr (D == 3) {
    // cofactor C[i][j] = (-1)^{i+j} det(minor ij) (cyclic minors carry the sign);
    // N = tr(adj(Z) dZ) = sum C[i][j] dZ[i][j], det Z = sum_j Z[0][j] C[0][j]
    N = mk(0, 0);
    Dt = mk(0, 0);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const int r0 = (i + 1) % 3, r1 = (i + 2) % 3, c0 = (j + 1) % 3, c1 = (j + 2) % 3;
        Cf[i][j] = Z[r0][c0] * Z[r1][c1] - Z[r0][c1] * Z[r1][c0];
        N = N + Cf[i][j] * Zd[i][j];
      }
#pragma unroll
    for (int j = 0; j < 3; ++j) Dt = Dt + Z[0][j] * Cf[0][j];
  } else {
    N = Z[1][1] * Zd[0][0] - Z[0][1] * Zd[1][0] - Z[1][0] * Zd[0][1] + Z[0][0] * Zd[1][1];
    Dt = Z[0][0] * Z[1][1] - Z[0][1] * Z[1][0];
  }
  const double dd = Dt.r * Dt.r + Dt.i * Dt.i;
  const double idd = rcp_nr(dd);
  const cx rD = mk(Dt.r * idd, -Dt.i * idd);
  const cx q = N * rD;
  const cx F = mk(ng + 0.5 * q.r, 0.5 * q.i);
  const cx a = mk(y[Lo::aR], y[Lo::aI]);
  // ---- reverse ----
  double Pb[D], nb[D], gb[D], Kb[D][D], Qb[D];
#pragma unroll
  for (int i = 0; i < D; ++i) {
    Pb[i] = 0;
    nb[i] = 0;
    gb[i] = 0;
    Qb[i] = 0;
#pragma unroll
    for (int k = 0; k < D; ++k) Kb[i][k] = 0;
  }
  double cb = 0, pnb = 0, copb = 0, rinvb = 0, pn2b = 0, ngb = 0;
  cx Ab[D][D], Bb[D][D], Adb[D][D], Bdb[D][D], agb[D], bnb[D], akb[D][D], Zb[D][D], Zdb[D][D];
#pragma unroll
  for (int j = 0; j < D; ++j) {
    agb[j] = mk(0, 0);
    bnb[j] = mk(0, 0);
#pragma unroll
    for (int k = 0; k < D; ++k) {
      Ab[j][k] = mk(0, 0);
      Bb[j][k] = mk(0, 0);
      Adb[j][k] = mk(kb[Lo::AR + j * D + k], kb[Lo::AI + j * D + k]);
      Bdb[j][k] = mk(kb[Lo::BR + j * D + k], kb[Lo::BI + j * D + k]);
      akb[j][k] = mk(0, 0);
      Zb[j][k] = mk(0, 0);
      Zdb[j][k] = mk(0, 0);
    }
  }
  // da/dt = a F
  const cx adb = mk(kb[Lo::aR], kb[Lo::aI]);
  const cx ab = mulc(adb, F);
  const cx Fb = mulc(adb, a);
  // F = ng + q/2
  ngb += Fb.r;
  const cx qb = 0.5 * Fb;
  // q = N rD, rD = 1/Dt
  const cx Nb = mulc(qb, rD);
  const cx rDb = mulc(qb, N);
  const cx Dtb = -1.0 * mulc(rDb, rD * rD);
  if constexpr (D == 1) {
    Zdb[0][0] = Zdb[0][0] + Nb;
    Zb[0][0] = Zb[0][0] + Dtb;
  } else if constexpr (D == 3) {
    // N = sum C dZ; det Z = sum_j Z[0][j] C[0][j]; C[i][j] = Z[r0][c0] Z[r1][c1] - Z[r0][c1] Z[r1][c0]
    cx Cb[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        Zdb[i][j] = Zdb[i][j] + mulc(Nb, Cf[i][j]);
        Cb[i][j] = mulc(Nb, Zd[i][j]);
      }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      Zb[0][j] = Zb[0][j] + mulc(Dtb, Cf[0][j]);
      Cb[0][j] = Cb[0][j] + mulc(Dtb, Z[0][j]);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const int r0 = (i + 1) % 3, r1 = (i + 2) % 3, c0 = (j + 1) % 3, c1 = (j + 2) % 3;
        Zb[r0][c0] = Zb[r0][c0] + mulc(Cb[i][j], Z[r1][c1]);
        Zb[r1][c1] = Zb[r1][c1] + mulc(Cb[i][j], Z[r0][c0]);
        Zb[r0][c1] = Zb[r0][c1] - mulc(Cb[i][j], Z[r1][c0]);
        Zb[r1][c0] = Zb[r1][c0] - mulc(Cb[i][j], Z[r0][c1]);
      }
  } else {
    Zb[0][0] = Zb[0][0] + mulc(Dtb, Z[1][1]);
    Zb[1][1] = Zb[1][1] + mulc(Dtb, Z[0][0]);
    Zb[0][1] = Zb[0][1] - mulc(Dtb, Z[1][0]);
    Zb[1][0] = Zb[1][0] - mulc(Dtb, Z[0][1]);
    Zb[1][1] = Zb[1][1] + mulc(Nb, Zd[0][0]);
    Zdb[0][0] = Zdb[0][0] + mulc(Nb, Z[1][1]);
    Zb[0][1] = Zb[0][1] - mulc(Nb, Zd[1][0]);
    Zdb[1][0] = Zdb[1][0] - mulc(Nb, Z[0][1]);
    Zb[1][0] = Zb[1][0] - mulc(Nb, Zd[0][1]);
    Zdb[0][1] = Zdb[0][1] - mulc(Nb, Z[1][0]);
    Zb[0][0] = Zb[0][0] + mulc(Nb, Zd[1][1]);
    Zdb[1][1] = Zdb[1][1] + mulc(Nb, Z[0][0]);
  }
  // Zd = Ad + i Bd, Z = A + i B  (adjoint of i w is -i times the adjoint)
#pragma unroll
  for (int j = 0; j < D; ++j)
#pragma unroll
    for (int k = 0; k < D; ++k) {
      Adb[j][k] = Adb[j][k] + Zdb[j][k];
      Bdb[j][k] = Bdb[j][k] + mk(Zdb[j][k].i, -Zdb[j][k].r);
      Ab[j][k] = Ab[j][k] + Zb[j][k];
      Bb[j][k] = Bb[j][k] + mk(Zb[j][k].i, -Zb[j][k].r);
    }
  // (S has no right-hand side: Layout)
  double Qdb[D];
#pragma unroll
  for (int i = 0; i < D; ++i) Qdb[i] = kb[Lo::Q + i];
  // Bd_jk = -(pn ak_jk + g_k bn_j);  Ad_jk = n_k ag_j + cop (B_jk - n_k bn_j)
#pragma unroll
  for (int j = 0; j < D; ++j)
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const cx bdb = Bdb[j][k];
      pnb += -rdot(bdb, ak[j][k]);
      akb[j][k] = akb[j][k] + (-pn) * bdb;
      bnb[j] = bnb[j] + (-m.g[k]) * bdb;
      gb[k] += -rdot(bdb, bn[j]);
      const cx adbk = Adb[j][k];
      agb[j] = agb[j] + n[k] * adbk;
      nb[k] += rdot(adbk, ag[j]) - cop * rdot(adbk, bn[j]);
      copb += rdot(adbk, B[j][k] - n[k] * bn[j]);
      Bb[j][k] = Bb[j][k] + cop * adbk;
      bnb[j] = bnb[j] + (-cop * n[k]) * adbk;
    }
  // ak_jk = sum_l A_jl K_lk; bn_j = sum_l B_jl n_l; ag_j = sum_l A_jl g_l
#pragma unroll
  for (int j = 0; j < D; ++j)
#pragma unroll
    for (int l = 0; l < D; ++l) {
#pragma unroll
      for (int k = 0; k < D; ++k) {
        Ab[j][l] = Ab[j][l] + m.K[l][k] * akb[j][k];
        Kb[l][k] += rdot(akb[j][k], A[j][l]);
      }
      Bb[j][l] = Bb[j][l] + n[l] * bnb[j];
      nb[l] += rdot(bnb[j], B[j][l]);
      Ab[j][l] = Ab[j][l] + m.g[l] * agb[j];
      gb[l] += rdot(agb[j], A[j][l]);
    }
  // ng = n.g; dP/dt = -pn g; dQ/dt = c n
  const double* Pdb = kb + Lo::P;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    nb[i] += ngb * m.g[i] + Qdb[i] * m.c;
    gb[i] += ngb * n[i] - Pdb[i] * pn;
    pnb += -Pdb[i] * m.g[i];
    cb += Qdb[i] * n[i];
  }
  // cop = c rinv; n = P rinv; pn = pn2 rinv; rinv = pn2^{-1/2}; pn2 = |P|^2
  cb += copb * rinv;
  rinvb += copb * m.c;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    Pb[i] += nb[i] * rinv;
    rinvb += nb[i] * P[i];
  }
  pn2b += pnb * rinv;
  rinvb += pnb * pn2;
  pn2b += rinvb * (-0.5 * rinv * rinv * rinv);
#pragma unroll
  for (int i = 0; i < D; ++i) Pb[i] += 2.0 * P[i] * pn2b;
  // medium
  medium_ad_transpose<D>(gd, m, cb, gb, Kb, Qb, gradC);
  // ---- accumulate into yb ----
#pragma unroll
  for (int i = 0; i < D; ++i) {
    yb[Lo::Q + i] += Qb[i];
    yb[Lo::P + i] += Pb[i];
  }
#pragma unroll
  for (int j = 0; j < D; ++j)
#pragma unroll
    for (int k = 0; k < D; ++k) {
      yb[Lo::AR + j * D + k] += Ab[j][k].r;
      yb[Lo::AI + j * D + k] += Ab[j][k].i;
      yb[Lo::BR + j * D + k] += Bb[j][k].r;
      yb[Lo::BI + j * D + k] += Bb[j][k].i;
    }
  yb[Lo::aR] += ab.r;
  yb[Lo::aI] += ab.i;
  // S does not enter f
}

// Scatter of the adjoints (cb, gb, Kb) of (c, grad c, Hessian) at x to the 16 spline
// coefficients around x (2D); the tap weights are computed again from x rather than
// kept from the forward evaluation (they would hold 48 registers through the whole
// vector-Jacobian product). kxz is the adjoint of the mixed derivative (both K entries).
// Coefficient (a, b) receives al_a w_b + be_a w'_b + ga_a w''_b with
// al_a = cb w_a + gx w'_a + kxx' w''_a, be_a = gz w_a + kxz' w'_a, ga_a = kzz' w_a (the
// 1/h factors of the derivative weights folded into the adjoints).
__device__ __forceinline__ void medium_scatter2(const GridDev& gd, const double* x, double cb,
                                                double gb0, double gb1, double kxx, double kxz,
                                                double kzz, double* __restrict__ gradC) {
  double w[2][4], dw[2][4], ddw[2][4];
  int64_t idx[2][4];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const double u = (x[k] - gd.o[k]) * gd.inv_h[k];
    const double fl = floor(u);
    spline_taps(u - fl, w[k], dw[k], ddw[k]);
    const int64_t i0 = (int64_t)fl - 1;
#pragma unroll
    for (int a = 0; a < 4; ++a) idx[k][a] = tap_index(i0 + a, gd.n[k], gd.periodic[k]);
  }
  const double ix = gd.inv_h[0], iz = gd.inv_h[1];
  const double gx = gb0 * ix, gz = gb1 * iz;
  const double kx2 = kxx * (ix * ix), kxz2 = kxz * (ix * iz), kz2 = kzz * (iz * iz);
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const double al = fma(kx2, ddw[0][a], fma(gx, dw[0][a], cb * w[0][a]));
    const double be = fma(kxz2, dw[0][a], gz * w[0][a]);
    const double ga = kz2 * w[0][a];
    double* row = gradC + idx[0][a] * gd.n[1];
#pragma unroll
    for (int b = 0; b < 4; ++b)
      red_add_f64(row + idx[1][b], fma(ga, ddw[1][b], fma(be, dw[1][b], al * w[1][b])));
  }
}

// c, grad c, Hessian and the third derivatives (xxx, xxz, xzz, zzz) of c at x (2D) from
// the per-cell polynomial table gd.tab, by Horner's scheme with derivatives: the same
// cell and arithmetic as the ray kernels' medium_eval_tab for c, grad c and the Hessian.
__device__ __forceinline__ void medium_tab3(const GridDev& gd, const double* x, double& c,
                                            double& g0, double& g1, double& K00, double& K01,
                                            double& K11, double& T0, double& T1, double& T2,
                                            double& T3) {
  double tx, tz;
  bool clx, clz;
  const int64_t cx = medium_cell_of(gd, 0, x[0], tx, clx);
  const int64_t cz = medium_cell_of(gd, 1, x[1], tz, clz);
  const double2* cell = reinterpret_cast<const double2*>(gd.tab) + (cx * (gd.n[1] + 2) + cz) * 8;
  // row k (power k of tx): its cubic in tz with d/dz and (d2/dz2)/2, and its tz^3 coefficient
  double r[4], rz[4], hz[4], a3[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const double2 a01 = __ldg(cell + 2 * k), a23 = __ldg(cell + 2 * k + 1);
    horner3(a01.x, a01.y, a23.x, a23.y, tz, r[k], rz[k], hz[k]);
    a3[k] = a23.y;
  }
  double cxx_h, cxxz_h, czz_h, cxzz, dummy;
  horner3(r[0], r[1], r[2], r[3], tx, c, g0, cxx_h);
  horner3(rz[0], rz[1], rz[2], rz[3], tx, g1, K01, cxxz_h);
  horner3(hz[0], hz[1], hz[2], hz[3], tx, czz_h, cxzz, dummy);
  K00 = 2.0 * cxx_h;
  K11 = 2.0 * czz_h;
  // beyond the clamped edge of an open axis c is constant along it: the pure third
  // derivative along that axis is 0 (the mixed ones vanish there with the cell's first and
  // second derivative coefficients)
  T0 = clx ? 0.0 : 6.0 * r[3];
  T1 = 2.0 * cxxz_h;
  T2 = 2.0 * cxzz;
  T3 = clz ? 0.0 : 6.0 * fma(fma(fma(a3[3], tx, a3[2]), tx, a3[1]), tx, a3[0]);
}

// The vector-Jacobian product of rhs2 (the 2D right-hand side) written out with scalars,
// the same derivative as the generic rhs_vjp term by term (the reverse of
//   dQ/dt = c n, dP/dt = -|P| g, dA_jk/dt = n_k u_j + (c/|P|) B_jk with
//   u_j = (A g)_j - (c/|P|)(B n)_j, dB_jk/dt = (A Km)_jk - g_k (B n)_j with Km = -|P| K,
//   da/dt = a (n.g + N conj(det Z)/(2 |det Z|^2)), N = tr(adj(Z) dZ/dt),
//   dS/dt = P.dQ/dt - c |P|),
// arranged so that far fewer values are live at once.
__device__ __forceinline__ void rhs2_vjp(const GridDev& gd, const double* __restrict__ C,
                                         const double* y, const double* kb, double* yb,
                                         double* __restrict__ gradC) {
  using Lo = Layout<2>;
  // ---- forward intermediates ----
  double c, g0, g1, K00, K01, K11, T0, T1, T2, T3;
  medium_tab3(gd, y + Lo::Q, c, g0, g1, K00, K01, K11, T0, T1, T2, T3);
  const double P0 = y[Lo::P], P1 = y[Lo::P + 1];
  const double pn2 = fma(P0, P0, P1 * P1);
  const double rinv = rsqrt_nr(pn2), pn = pn2 * rinv, cop = c * rinv;
  const double n0 = P0 * rinv, n1 = P1 * rinv;
  const double ng = fma(n0, g0, n1 * g1);
  const double km00 = -pn * K00, km01 = -pn * K01, km11 = -pn * K11;
  auto Aj = [&](int j, int k) { return mk(y[Lo::AR + 2 * j + k], y[Lo::AI + 2 * j + k]); };
  auto Bj = [&](int j, int k) { return mk(y[Lo::BR + 2 * j + k], y[Lo::BI + 2 * j + k]); };
  auto Zj = [&](int j, int k) {  // A + i B
    return mk(y[Lo::AR + 2 * j + k] - y[Lo::BI + 2 * j + k], y[Lo::AI + 2 * j + k] + y[Lo::BR + 2 * j + k]);
  };
  cx bn[2], u[2], Zd[2][2];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const cx A0 = Aj(j, 0), A1 = Aj(j, 1), B0 = Bj(j, 0), B1 = Bj(j, 1);
    bn[j] = n0 * B0 + n1 * B1;
    u[j] = (g0 * A0 + g1 * A1) - cop * bn[j];
    const cx Ad0 = n0 * u[j] + cop * B0, Ad1 = n1 * u[j] + cop * B1;
    const cx Bd0 = (km00 * A0 + km01 * A1) - g0 * bn[j];
    const cx Bd1 = (km01 * A0 + km11 * A1) - g1 * bn[j];
    Zd[j][0] = Ad0 + mk(-Bd0.i, Bd0.r);
    Zd[j][1] = Ad1 + mk(-Bd1.i, Bd1.r);
  }
  const cx Z00 = Zj(0, 0), Z01 = Zj(0, 1), Z10 = Zj(1, 0), Z11 = Zj(1, 1);
  const cx N = Z11 * Zd[0][0] - Z01 * Zd[1][0] - Z10 * Zd[0][1] + Z00 * Zd[1][1];
  const cx Dt = Z00 * Z11 - Z01 * Z10;
  const double idd = rcp_nr(fma(Dt.r, Dt.r, Dt.i * Dt.i));
  const cx rD = mk(Dt.r * idd, -Dt.i * idd);
  const cx q = N * rD;
  const cx F = mk(ng + 0.5 * q.r, 0.5 * q.i);
  // ---- reverse ----
  const cx a = mk(y[Lo::aR], y[Lo::aI]);
  const cx kab = mk(kb[Lo::aR], kb[Lo::aI]);
  const cx ab = mulc(kab, F);
  yb[Lo::aR] += ab.r;
  yb[Lo::aI] += ab.i;
  const cx Fb = mulc(kab, a);
  const double ngb = Fb.r;
  const cx qb = 0.5 * Fb;
  const cx Nb = mulc(qb, rD);
  const cx Dtb = -1.0 * mulc(mulc(qb, N), rD * rD);
  // adjoints of Z (det and N) and of dZ/dt (N)
  cx Zb[2][2], Zdb[2][2];
  Zb[0][0] = mulc(Dtb, Z11) + mulc(Nb, Zd[1][1]);
  Zb[1][1] = mulc(Dtb, Z00) + mulc(Nb, Zd[0][0]);
  Zb[0][1] = -1.0 * (mulc(Dtb, Z10) + mulc(Nb, Zd[1][0]));
  Zb[1][0] = -1.0 * (mulc(Dtb, Z01) + mulc(Nb, Zd[0][1]));
  Zdb[0][0] = mulc(Nb, Z11);
  Zdb[1][1] = mulc(Nb, Z00);
  Zdb[1][0] = -1.0 * mulc(Nb, Z01);
  Zdb[0][1] = -1.0 * mulc(Nb, Z10);
  // (S has no right-hand side: Layout)
  const double Qdb0 = kb[Lo::Q], Qdb1 = kb[Lo::Q + 1];
  double Pb0 = 0.0, Pb1 = 0.0;
  double cb = 0.0, pnb = 0.0;
  double nb0 = 0, nb1 = 0, gb0 = 0, gb1 = 0, copb = 0, kmb00 = 0, kmb01 = 0, kmb11 = 0;
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const cx A0 = Aj(j, 0), A1 = Aj(j, 1), B0 = Bj(j, 0), B1 = Bj(j, 1);
    // dZ/dt = dA/dt + i dB/dt, Z = A + i B (the adjoint of i w is -i times w's adjoint)
    const cx Adb0 = mk(kb[Lo::AR + 2 * j], kb[Lo::AI + 2 * j]) + Zdb[j][0];
    const cx Adb1 = mk(kb[Lo::AR + 2 * j + 1], kb[Lo::AI + 2 * j + 1]) + Zdb[j][1];
    const cx Bdb0 = mk(kb[Lo::BR + 2 * j], kb[Lo::BI + 2 * j]) + mk(Zdb[j][0].i, -Zdb[j][0].r);
    const cx Bdb1 = mk(kb[Lo::BR + 2 * j + 1], kb[Lo::BI + 2 * j + 1]) + mk(Zdb[j][1].i, -Zdb[j][1].r);
    cx Ab0 = Zb[j][0], Ab1 = Zb[j][1];
    cx Bb0 = mk(Zb[j][0].i, -Zb[j][0].r), Bb1 = mk(Zb[j][1].i, -Zb[j][1].r);
    // dB_jk/dt = km_0k A_j0 + km_1k A_j1 - g_k bn_j
    Ab0 = Ab0 + (km00 * Bdb0 + km01 * Bdb1);
    Ab1 = Ab1 + (km01 * Bdb0 + km11 * Bdb1);
    kmb00 += rdot(Bdb0, A0);
    kmb01 += rdot(Bdb0, A1) + rdot(Bdb1, A0);
    kmb11 += rdot(Bdb1, A1);
    gb0 -= rdot(Bdb0, bn[j]);
    gb1 -= rdot(Bdb1, bn[j]);
    cx bnb = -1.0 * (g0 * Bdb0 + g1 * Bdb1);
    // dA_jk/dt = n_k u_j + cop B_jk
    const cx ub = n0 * Adb0 + n1 * Adb1;
    nb0 += rdot(Adb0, u[j]);
    nb1 += rdot(Adb1, u[j]);
    copb += rdot(Adb0, B0) + rdot(Adb1, B1);
    Bb0 = Bb0 + cop * Adb0;
    Bb1 = Bb1 + cop * Adb1;
    // u_j = ag_j - cop bn_j, ag_j = g0 A_j0 + g1 A_j1
    bnb = bnb - cop * ub;
    copb -= rdot(ub, bn[j]);
    Ab0 = Ab0 + g0 * ub;
    Ab1 = Ab1 + g1 * ub;
    gb0 += rdot(ub, A0);
    gb1 += rdot(ub, A1);
    // bn_j = n0 B_j0 + n1 B_j1
    Bb0 = Bb0 + n0 * bnb;
    Bb1 = Bb1 + n1 * bnb;
    nb0 += rdot(bnb, B0);
    nb1 += rdot(bnb, B1);
    yb[Lo::AR + 2 * j] += Ab0.r;
    yb[Lo::AI + 2 * j] += Ab0.i;
    yb[Lo::AR + 2 * j + 1] += Ab1.r;
    yb[Lo::AI + 2 * j + 1] += Ab1.i;
    yb[Lo::BR + 2 * j] += Bb0.r;
    yb[Lo::BI + 2 * j] += Bb0.i;
    yb[Lo::BR + 2 * j + 1] += Bb1.r;
    yb[Lo::BI + 2 * j + 1] += Bb1.i;
  }
  // km = -pn K (K symmetric: kmb01 collects both of its uses)
  const double Kb00 = -pn * kmb00, Kbxz = -pn * kmb01, Kb11 = -pn * kmb11;
  pnb -= K00 * kmb00 + K01 * kmb01 + K11 * kmb11;
  // ng = n.g; dQ/dt = c n; dP/dt = -pn g
  const double Pdb0 = kb[Lo::P], Pdb1 = kb[Lo::P + 1];
  nb0 += ngb * g0 + Qdb0 * c;
  nb1 += ngb * g1 + Qdb1 * c;
  gb0 += ngb * n0 - Pdb0 * pn;
  gb1 += ngb * n1 - Pdb1 * pn;
  pnb -= Pdb0 * g0 + Pdb1 * g1;
  cb += Qdb0 * n0 + Qdb1 * n1;
  // cop = c rinv; n = P rinv; pn = pn2 rinv; rinv = pn2^{-1/2}; pn2 = |P|^2
  cb += copb * rinv;
  double rinvb = copb * c + nb0 * P0 + nb1 * P1 + pnb * pn2;
  Pb0 += nb0 * rinv;
  Pb1 += nb1 * rinv;
  const double pn2b = pnb * rinv + rinvb * (-0.5 * rinv * rinv * rinv);
  Pb0 += 2.0 * P0 * pn2b;
  Pb1 += 2.0 * P1 * pn2b;
  // medium at Q
  yb[Lo::Q] += cb * g0 + gb0 * K00 + gb1 * K01 + Kb00 * T0 + Kbxz * T1 + Kb11 * T2;
  yb[Lo::Q + 1] += cb * g1 + gb0 * K01 + gb1 * K11 + Kb00 * T1 + Kbxz * T2 + Kb11 * T3;
  yb[Lo::P] += Pb0;
  yb[Lo::P + 1] += Pb1;
  medium_scatter2(gd, y + Lo::Q, cb, gb0, gb1, Kb00, Kbxz, Kb11, gradC);
  // S does not enter f
}

// One RK4 step that also hands its stage states z2 = y + h/2 k1, z3 = y + h/2 k2,
// z4 = y + h k3 to put(stage, z) (the same arithmetic as rk4_step).
template <int D, typename Put>
__device__ __forceinline__ void rk4_step_record(const GridDev& gd, double* y, double dt, Put put) {
  using Lo = Layout<D>;
  constexpr int NF = Lo::NF;
  constexpr int NI = Lo::NI;  // S is not integrated (Layout)
  double acc[NF], tmp[NF], k[NF];
  tmp[Lo::S] = y[Lo::S];
  const double h2 = 0.5 * dt, h6 = dt / 6.0, h3 = dt / 3.0;
  rhs<D>(gd, y, k);
#pragma unroll
  for (int i = 0; i < NI; ++i) {
    acc[i] = fma(h6, k[i], y[i]);
    tmp[i] = fma(h2, k[i], y[i]);
  }
  put(0, tmp);
  rhs<D>(gd, tmp, k);
#pragma unroll
  for (int i = 0; i < NI; ++i) {
    acc[i] = fma(h3, k[i], acc[i]);
    tmp[i] = fma(h2, k[i], y[i]);
  }
  put(1, tmp);
  rhs<D>(gd, tmp, k);
#pragma unroll
  for (int i = 0; i < NI; ++i) {
    acc[i] = fma(h3, k[i], acc[i]);
    tmp[i] = fma(dt, k[i], y[i]);
  }
  put(2, tmp);
  rhs<D>(gd, tmp, k);
#pragma unroll
  for (int i = 0; i < NI; ++i) y[i] = fma(h6, k[i], acc[i]);
#pragma unroll
  for (int i = 0; i < D; ++i) {
    if (gd.periodic[i]) {
      double r = fmod(y[Lo::Q + i] - gd.o[i], gd.L[i]);
      if (r < 0) r += gd.L[i];
      y[Lo::Q + i] = gd.o[i] + r;
    }
  }
}

// One RK4 step y -> y + dt/6 (k1 + 2 k2 + 2 k3 + k4) (the periodic wrap is a shift).
template <int D>
__device__ __forceinline__ void rk4_step(const GridDev& gd, const double* __restrict__ C, double* y,
                                         double dt) {
  using Lo = Layout<D>;
  constexpr int NF = Lo::NF;
  constexpr int NI = Lo::NI;  // S is not integrated (Layout)
  double acc[NF], tmp[NF], k[NF];
  tmp[Lo::S] = y[Lo::S];
  const double h2 = 0.5 * dt, h6 = dt / 6.0, h3 = dt / 3.0;
  rhs<D>(gd, y, k);
#pragma unroll
  for (int i = 0; i < NI; ++i) {
    acc[i] = fma(h6, k[i], y[i]);
    tmp[i] = fma(h2, k[i], y[i]);
  }
  rhs<D>(gd, tmp, k);
#pragma unroll
  for (int i = 0; i < NI; ++i) {
    acc[i] = fma(h3, k[i], acc[i]);
    tmp[i] = fma(h2, k[i], y[i]);
  }
  rhs<D>(gd, tmp, k);
#pragma unroll
  for (int i = 0; i < NI; ++i) {
    acc[i] = fma(h3, k[i], acc[i]);
    tmp[i] = fma(dt, k[i], y[i]);
  }
  rhs<D>(gd, tmp, k);
#pragma unroll
  for (int i = 0; i < NI; ++i) y[i] = fma(h6, k[i], acc[i]);
#pragma unroll
  for (int i = 0; i < D; ++i) {
    if (gd.periodic[i]) {
      double r = fmod(y[Lo::Q + i] - gd.o[i], gd.L[i]);
      if (r < 0) r += gd.L[i];
      y[Lo::Q + i] = gd.o[i] + r;
    }
  }
}

template <int D>
__device__ __forceinline__ void vjp(const GridDev& gd, const double* __restrict__ C, const double* y,
                                    const double* kb, double* yb, double* __restrict__ gradC) {
  if constexpr (D == 2)
    rhs2_vjp(gd, C, y, kb, yb, gradC);
  else
    rhs_vjp<D>(gd, C, y, kb, yb, gradC);
}

// lambda <- (d step/d y)^T lambda at the state y (start of the step), gradC accumulated.
// The three stage states and the incoming lambda live in the caller's shared-memory
// slots zs[(slot * NF + field) * nt + lane] (4 * NF values per thread) rather than in
// registers, which the vector-Jacobian products need.
// The step's stage states z2, z3, z4 come from stage(s, f) (recorded by rk4_step_record
// when the segment was recomputed).
template <int D, typename Stage>
__device__ void rk4_step_adjoint(const GridDev& gd, const double* __restrict__ C, const double* y,
                                 double dt, double* lam, double* __restrict__ gradC, double* zs,
                                 int nt, int lane, Stage stage) {
  using Lo = Layout<D>;
  constexpr int NF = Lo::NF;
  auto Z = [&](int s, int f) -> double& { return zs[(s * NF + f) * nt + lane]; };
  const double h2 = 0.5 * dt, h6 = dt / 6.0, h3 = dt / 3.0;
#pragma unroll
  for (int s = 0; s < 3; ++s)
#pragma unroll
    for (int i = 0; i < NF; ++i) Z(s, i) = stage(s, i);
#pragma unroll
  for (int i = 0; i < NF; ++i) Z(3, i) = lam[i];  // lambda in
  double kb[NF], zb[NF], z[NF];
  // S is not integrated (Layout): its stage cotangents are 0 and lambda_S passes through
  constexpr int NI = Lo::NI;
  kb[Lo::S] = zb[Lo::S] = 0.0;
  z[Lo::S] = Z(2, Lo::S);
  // stage 4: k4 bar = h/6 lambda
#pragma unroll
  for (int i = 0; i < NI; ++i) {
    kb[i] = h6 * Z(3, i);
    zb[i] = 0.0;
    z[i] = Z(2, i);
  }
  vjp<D>(gd, C, z, kb, zb, gradC);
  // stage 3: k3 bar = h/3 lambda + h z4 bar
#pragma unroll
  for (int i = 0; i < NI; ++i) {
    lam[i] += zb[i];
    kb[i] = fma(dt, zb[i], h3 * Z(3, i));
    zb[i] = 0.0;
    z[i] = Z(1, i);
  }
  vjp<D>(gd, C, z, kb, zb, gradC);
  // stage 2: k2 bar = h/3 lambda + h/2 z3 bar
#pragma unroll
  for (int i = 0; i < NI; ++i) {
    lam[i] += zb[i];
    kb[i] = fma(h2, zb[i], h3 * Z(3, i));
    zb[i] = 0.0;
    z[i] = Z(0, i);
  }
  vjp<D>(gd, C, z, kb, zb, gradC);
  // stage 1: k1 bar = h/6 lambda + h/2 z2 bar, at y itself
#pragma unroll
  for (int i = 0; i < NI; ++i) {
    lam[i] += zb[i];
    kb[i] = fma(h2, zb[i], h6 * Z(3, i));
  }
  vjp<D>(gd, C, y, kb, lam, gradC);
}

}  // namespace adj
}  // namespace fga
