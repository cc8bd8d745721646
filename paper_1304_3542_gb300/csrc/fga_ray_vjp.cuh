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
  double c, g[D], K[D][D], T3[4];  // 2D third derivatives: xxx, xxz, xzz, zzz
  int64_t idx[D][4];
  double w[D][4], dw[D][4], ddw[D][4], dddw[D][4];
};

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
  if constexpr (D == 1) {
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

// yb += (d f/d y)^T kb and gradC += (d f/d C)^T kb for the right-hand side f of rhs<D>.
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
  const double rinv = rsqrt(pn2), pn = pn2 * rinv, cop = m.c * rinv;
  double ng = 0, Qd[D];
#pragma unroll
  for (int i = 0; i < D; ++i) {
    n[i] = P[i] * rinv;
    Qd[i] = m.c * n[i];
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
  if constexpr (D == 1) {
    N = Zd[0][0];
    Dt = Z[0][0];
  } else {
    N = Z[1][1] * Zd[0][0] - Z[0][1] * Zd[1][0] - Z[1][0] * Zd[0][1] + Z[0][0] * Zd[1][1];
    Dt = Z[0][0] * Z[1][1] - Z[0][1] * Z[1][0];
  }
  const double dd = Dt.r * Dt.r + Dt.i * Dt.i;
  const cx rD = mk(Dt.r / dd, -Dt.i / dd);
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
  // dS/dt = P.Qd - c pn
  const double Sdb = kb[Lo::S];
  double Qdb[D];
#pragma unroll
  for (int i = 0; i < D; ++i) {
    Qdb[i] = kb[Lo::Q + i] + Sdb * P[i];
    Pb[i] += Sdb * Qd[i];
  }
  cb += -Sdb * pn;
  pnb += -Sdb * m.c;
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

// One RK4 step that also hands its stage states z2 = y + h/2 k1, z3 = y + h/2 k2,
// z4 = y + h k3 to put(stage, z) (the same arithmetic as rk4_step).
template <int D, typename Put>
__device__ __forceinline__ void rk4_step_record(const GridDev& gd, double* y, double dt, Put put) {
  using Lo = Layout<D>;
  constexpr int NF = Lo::NF;
  double acc[NF], tmp[NF], k[NF];
  const double h2 = 0.5 * dt, h6 = dt / 6.0, h3 = dt / 3.0;
  rhs<D>(gd, y, k);
#pragma unroll
  for (int i = 0; i < NF; ++i) {
    acc[i] = fma(h6, k[i], y[i]);
    tmp[i] = fma(h2, k[i], y[i]);
  }
  put(0, tmp);
  rhs<D>(gd, tmp, k);
#pragma unroll
  for (int i = 0; i < NF; ++i) {
    acc[i] = fma(h3, k[i], acc[i]);
    tmp[i] = fma(h2, k[i], y[i]);
  }
  put(1, tmp);
  rhs<D>(gd, tmp, k);
#pragma unroll
  for (int i = 0; i < NF; ++i) {
    acc[i] = fma(h3, k[i], acc[i]);
    tmp[i] = fma(dt, k[i], y[i]);
  }
  put(2, tmp);
  rhs<D>(gd, tmp, k);
#pragma unroll
  for (int i = 0; i < NF; ++i) y[i] = fma(h6, k[i], acc[i]);
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
  double acc[NF], tmp[NF], k[NF];
  const double h2 = 0.5 * dt, h6 = dt / 6.0, h3 = dt / 3.0;
  rhs<D>(gd, y, k);
#pragma unroll
  for (int i = 0; i < NF; ++i) {
    acc[i] = fma(h6, k[i], y[i]);
    tmp[i] = fma(h2, k[i], y[i]);
  }
  rhs<D>(gd, tmp, k);
#pragma unroll
  for (int i = 0; i < NF; ++i) {
    acc[i] = fma(h3, k[i], acc[i]);
    tmp[i] = fma(h2, k[i], y[i]);
  }
  rhs<D>(gd, tmp, k);
#pragma unroll
  for (int i = 0; i < NF; ++i) {
    acc[i] = fma(h3, k[i], acc[i]);
    tmp[i] = fma(dt, k[i], y[i]);
  }
  rhs<D>(gd, tmp, k);
#pragma unroll
  for (int i = 0; i < NF; ++i) y[i] = fma(h6, k[i], acc[i]);
#pragma unroll
  for (int i = 0; i < D; ++i) {
    if (gd.periodic[i]) {
      double r = fmod(y[Lo::Q + i] - gd.o[i], gd.L[i]);
      if (r < 0) r += gd.L[i];
      y[Lo::Q + i] = gd.o[i] + r;
    }
  }
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
  // stage 4: k4 bar = h/6 lambda
#pragma unroll
  for (int i = 0; i < NF; ++i) {
    kb[i] = h6 * Z(3, i);
    zb[i] = 0.0;
    z[i] = Z(2, i);
  }
  rhs_vjp<D>(gd, C, z, kb, zb, gradC);
  // stage 3: k3 bar = h/3 lambda + h z4 bar
#pragma unroll
  for (int i = 0; i < NF; ++i) {
    lam[i] += zb[i];
    kb[i] = fma(dt, zb[i], h3 * Z(3, i));
    zb[i] = 0.0;
    z[i] = Z(1, i);
  }
  rhs_vjp<D>(gd, C, z, kb, zb, gradC);
  // stage 2: k2 bar = h/3 lambda + h/2 z3 bar
#pragma unroll
  for (int i = 0; i < NF; ++i) {
    lam[i] += zb[i];
    kb[i] = fma(h2, zb[i], h3 * Z(3, i));
    zb[i] = 0.0;
    z[i] = Z(0, i);
  }
  rhs_vjp<D>(gd, C, z, kb, zb, gradC);
  // stage 1: k1 bar = h/6 lambda + h/2 z2 bar, at y itself
#pragma unroll
  for (int i = 0; i < NF; ++i) {
    lam[i] += zb[i];
    kb[i] = fma(h2, zb[i], h6 * Z(3, i));
  }
  rhs_vjp<D>(gd, C, y, kb, lam, gradC);
}

}  // namespace adj
}  // namespace fga
