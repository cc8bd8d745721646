// Right-hand side of the FGA ray system shared by the forward integrator and the
// adjoint: Eqs. characline, dzQ, dzP, a_formu (Z of Eq. op_zZ) and dS/dt = P.dQ/dt - H
// for the + branch, H = c(Q)|P|; plus the initial state and the stored outputs.
#pragma once

#include "fga_internal.cuh"
#include "fga_medium.cuh"

namespace fga {

// State of one ray: Q, P, A = dQ/dz, B = dP/dz (real and imaginary parts), a, S. S is
// carried but not integrated: for H = c(Q)|P|, homogeneous of degree 1 in P,
// P.dH/dP = H, so dS/dt = P.dQ/dt - H vanishes identically and S keeps its initial
// value 0 (RK4 on a zero right-hand side is the identity). The RK4 scheme integrates the
// first NI = NF - 1 fields.
template <int D>
struct Layout {
  static constexpr int NF = 2 * D + 4 * D * D + 3;
  static constexpr int NI = NF - 1;
  static constexpr int Q = 0, P = D, AR = 2 * D, AI = 2 * D + D * D, BR = 2 * D + 2 * D * D,
                       BI = 2 * D + 3 * D * D, aR = 2 * D + 4 * D * D, aI = aR + 1, S = aR + 2;
};

// Order in which the persistent ray kernels take Gaussians: work item w -> Gaussian
// (w * mult) mod G, mult coprime with G and near G/golden ratio. Consecutive Gaussians
// share q (and so, early on, position and receivers); spreading them over the list keeps
// the threads running at the same time from adding into the same few trace or
// gradient entries at once.
__device__ __forceinline__ int64_t work_order(unsigned long long w, int64_t G, unsigned long long mult) {
  return (int64_t)((w * mult) % (unsigned long long)G);
}

// The right-hand side in 2D with the algebra arranged for fused multiply-adds (the same
// equations as the generic form below; only the rounding differs):
//   dQ/dt = (c/|P|) P,  dP/dt = -|P| g,
//   dA_jk/dt = ((A g)_j - (c/|P|)(B n)_j) n_k + (c/|P|) B_jk,
//   dB_jk/dt = (A Km)_jk - (B n)_j g_k,  Km = -|P| K  (H_QQ = |P| K),
//   da/dt = a (n.g + tr(adj(Z) dZ/dt) conj(det Z)/(2 |det Z|^2)),  dS/dt = P.dQ/dt - c|P|.
__device__ __forceinline__ bool rhs2(const GridDev& gd, const double* y, double* k) {
  using Lo = Layout<2>;
  Med m;
  medium_eval_tab<2>(gd, y + Lo::Q, m);
  const double p0 = y[Lo::P], p1 = y[Lo::P + 1];
  const double pn2 = fma(p0, p0, p1 * p1);
  const double rinv = rsqrt_nr(pn2);
  const double pn = pn2 * rinv;
  const double n0 = p0 * rinv, n1 = p1 * rinv;
  const double cop = m.c * rinv;  // c/|P|
  const double g0 = m.g[0], g1 = m.g[1];
  k[Lo::Q] = cop * p0;
  k[Lo::Q + 1] = cop * p1;
  k[Lo::P] = -pn * g0;
  k[Lo::P + 1] = -pn * g1;
  const double ng = fma(n0, g0, n1 * g1);
  const double km00 = -pn * m.K[0][0], km01 = -pn * m.K[0][1], km11 = -pn * m.K[1][1];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const double ar0 = y[Lo::AR + 2 * j], ar1 = y[Lo::AR + 2 * j + 1];
    const double ai0 = y[Lo::AI + 2 * j], ai1 = y[Lo::AI + 2 * j + 1];
    const double br0 = y[Lo::BR + 2 * j], br1 = y[Lo::BR + 2 * j + 1];
    const double bi0 = y[Lo::BI + 2 * j], bi1 = y[Lo::BI + 2 * j + 1];
    const double bnr = fma(br0, n0, br1 * n1), bni = fma(bi0, n0, bi1 * n1);
    const double ur = fma(-cop, bnr, fma(ar0, g0, ar1 * g1));
    const double ui = fma(-cop, bni, fma(ai0, g0, ai1 * g1));
    k[Lo::AR + 2 * j] = fma(ur, n0, cop * br0);
    k[Lo::AR + 2 * j + 1] = fma(ur, n1, cop * br1);
    k[Lo::AI + 2 * j] = fma(ui, n0, cop * bi0);
    k[Lo::AI + 2 * j + 1] = fma(ui, n1, cop * bi1);
    k[Lo::BR + 2 * j] = fma(ar0, km00, fma(ar1, km01, -bnr * g0));
    k[Lo::BR + 2 * j + 1] = fma(ar0, km01, fma(ar1, km11, -bnr * g1));
    k[Lo::BI + 2 * j] = fma(ai0, km00, fma(ai1, km01, -bni * g0));
    k[Lo::BI + 2 * j + 1] = fma(ai0, km01, fma(ai1, km11, -bni * g1));
  }
  // Z = A + iB, dZ/dt; tr(adj(Z) dZ) = Z11 dZ00 - Z01 dZ10 - Z10 dZ01 + Z00 dZ11
  double zr[4], zi[4], dzr[4], dzi[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    zr[e] = y[Lo::AR + e] - y[Lo::BI + e];
    zi[e] = y[Lo::AI + e] + y[Lo::BR + e];
    dzr[e] = k[Lo::AR + e] - k[Lo::BI + e];
    dzi[e] = k[Lo::AI + e] + k[Lo::BR + e];
  }
  double trr = zr[3] * dzr[0];
  trr = fma(-zi[3], dzi[0], trr);
  trr = fma(-zr[1], dzr[2], trr);
  trr = fma(zi[1], dzi[2], trr);
  trr = fma(-zr[2], dzr[1], trr);
  trr = fma(zi[2], dzi[1], trr);
  trr = fma(zr[0], dzr[3], trr);
  trr = fma(-zi[0], dzi[3], trr);
  double tri = zr[3] * dzi[0];
  tri = fma(zi[3], dzr[0], tri);
  tri = fma(-zr[1], dzi[2], tri);
  tri = fma(-zi[1], dzr[2], tri);
  tri = fma(-zr[2], dzi[1], tri);
  tri = fma(-zi[2], dzr[1], tri);
  tri = fma(zr[0], dzi[3], tri);
  tri = fma(zi[0], dzr[3], tri);
  const double detr = fma(zr[0], zr[3], fma(-zi[0], zi[3], fma(-zr[1], zr[2], zi[1] * zi[2])));
  const double deti = fma(zr[0], zi[3], fma(zi[0], zr[3], fma(-zr[1], zi[2], -zi[1] * zr[2])));
  const double dd = fma(detr, detr, deti * deti);
  const double ih = 0.5 * rcp_nr(dd);  // 1/(2 |det Z|^2)
  const double qr = fma(trr, detr, tri * deti) * ih, qi = fma(tri, detr, -trr * deti) * ih;
  const double fr = ng + qr;
  const double ar = y[Lo::aR], ai = y[Lo::aI];
  k[Lo::aR] = fma(ar, fr, -ai * qi);
  k[Lo::aI] = fma(ar, qi, ai * fr);
  return pn2 > 0.0 && dd > 0.0;
}

// The right-hand side in 3D, arranged like rhs2 (the same equations; only the rounding
// differs from a literal transcription):
//   dA_jk/dt = ((A g)_j - (c/|P|)(B n)_j) n_k + (c/|P|) B_jk,
//   dB_jk/dt = (A Km)_jk - (B n)_j g_k,  Km = -|P| K,
//   da/dt = a (n.g + tr(adj(Z) dZ/dt) conj(det Z)/(2 |det Z|^2)),
// with adj(Z) from the cofactors of the 3 x 3 complex Z = A + iB.
__device__ __forceinline__ bool rhs3(const GridDev& gd, const double* y, double* k) {
  using Lo = Layout<3>;
  Med m;
  medium_eval_tab<3>(gd, y + Lo::Q, m);
  const double p0 = y[Lo::P], p1 = y[Lo::P + 1], p2 = y[Lo::P + 2];
  const double pn2 = fma(p0, p0, fma(p1, p1, p2 * p2));
  const double rinv = rsqrt_nr(pn2);
  const double pn = pn2 * rinv;
  const double n[3] = {p0 * rinv, p1 * rinv, p2 * rinv};
  const double cop = m.c * rinv;  // c/|P|
  k[Lo::Q] = cop * p0;
  k[Lo::Q + 1] = cop * p1;
  k[Lo::Q + 2] = cop * p2;
#pragma unroll
  for (int i = 0; i < 3; ++i) k[Lo::P + i] = -pn * m.g[i];
  const double ng = fma(n[0], m.g[0], fma(n[1], m.g[1], n[2] * m.g[2]));
  double km[3][3];
#pragma unroll
  for (int l = 0; l < 3; ++l)
#pragma unroll
    for (int kk = l; kk < 3; ++kk) {
      km[l][kk] = -pn * m.K[l][kk];
      km[kk][l] = km[l][kk];
    }
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const double* ar = y + Lo::AR + 3 * j;
    const double* ai = y + Lo::AI + 3 * j;
    const double* br = y + Lo::BR + 3 * j;
    const double* bi = y + Lo::BI + 3 * j;
    const double bnr = fma(br[0], n[0], fma(br[1], n[1], br[2] * n[2]));
    const double bni = fma(bi[0], n[0], fma(bi[1], n[1], bi[2] * n[2]));
    const double ur = fma(-cop, bnr, fma(ar[0], m.g[0], fma(ar[1], m.g[1], ar[2] * m.g[2])));
    const double ui = fma(-cop, bni, fma(ai[0], m.g[0], fma(ai[1], m.g[1], ai[2] * m.g[2])));
#pragma unroll
    for (int kk = 0; kk < 3; ++kk) {
      k[Lo::AR + 3 * j + kk] = fma(ur, n[kk], cop * br[kk]);
      k[Lo::AI + 3 * j + kk] = fma(ui, n[kk], cop * bi[kk]);
      k[Lo::BR + 3 * j + kk] = fma(ar[0], km[0][kk], fma(ar[1], km[1][kk], fma(ar[2], km[2][kk], -bnr * m.g[kk])));
      k[Lo::BI + 3 * j + kk] = fma(ai[0], km[0][kk], fma(ai[1], km[1][kk], fma(ai[2], km[2][kk], -bni * m.g[kk])));
    }
  }
  // Z = A + iB and dZ/dt; cofactor C[i][j] = (-1)^{i+j} det(minor ij) (the cyclic minors
  // carry the sign), adj(Z)[j][i] = C[i][j]; tr(adj(Z) dZ) = sum C[i][j] dZ[i][j] and
  // det Z = sum_j Z[0][j] C[0][j]
  double zr[9], zi[9], dzr[9], dzi[9];
#pragma unroll
  for (int e = 0; e < 9; ++e) {
    zr[e] = y[Lo::AR + e] - y[Lo::BI + e];
    zi[e] = y[Lo::AI + e] + y[Lo::BR + e];
    dzr[e] = k[Lo::AR + e] - k[Lo::BI + e];
    dzi[e] = k[Lo::AI + e] + k[Lo::BR + e];
  }
  double trr = 0.0, tri = 0.0, detr = 0.0, deti = 0.0;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int r0 = (i + 1) % 3, r1 = (i + 2) % 3, c0 = (j + 1) % 3, c1 = (j + 2) % 3;
      const double ar = zr[r0 * 3 + c0], ai = zi[r0 * 3 + c0], br = zr[r1 * 3 + c1], bi = zi[r1 * 3 + c1];
      const double er = zr[r0 * 3 + c1], ei = zi[r0 * 3 + c1], fr = zr[r1 * 3 + c0], fi = zi[r1 * 3 + c0];
      const double cr = fma(ar, br, fma(-ai, bi, fma(-er, fr, ei * fi)));
      const double ci = fma(ar, bi, fma(ai, br, fma(-er, fi, -ei * fr)));
      const int e = i * 3 + j;
      trr = fma(cr, dzr[e], fma(-ci, dzi[e], trr));
      tri = fma(cr, dzi[e], fma(ci, dzr[e], tri));
      if (i == 0) {
        detr = fma(zr[j], cr, fma(-zi[j], ci, detr));
        deti = fma(zr[j], ci, fma(zi[j], cr, deti));
      }
    }
  const double dd = fma(detr, detr, deti * deti);
  const double ih = 0.5 * rcp_nr(dd);  // 1/(2 |det Z|^2)
  const double qr = fma(trr, detr, tri * deti) * ih, qi = fma(tri, detr, -trr * deti) * ih;
  const double fr = ng + qr;
  const double ar = y[Lo::aR], ai = y[Lo::aI];
  k[Lo::aR] = fma(ar, fr, -ai * qi);
  k[Lo::aI] = fma(ar, qi, ai * fr);
  return pn2 > 0.0 && dd > 0.0;
}

// The right-hand side in 1D (Z = A + iB is a scalar: tr(Z^{-1} dZ/dt) = dZ/Z), and the
// dispatch to the 2D and 3D forms. The medium comes from the per-cell polynomial table
// gd.tab.
template <int D>
__device__ __forceinline__ bool rhs(const GridDev& gd, const double* y, double* k) {
  if constexpr (D == 2) {
    return rhs2(gd, y, k);
  } else if constexpr (D == 3) {
    return rhs3(gd, y, k);
  } else {
    using Lo = Layout<1>;
    Med m;
    medium_eval_tab<1>(gd, y + Lo::Q, m);
    const double p = y[Lo::P];
    const double pn2 = p * p;
    const double rinv = rsqrt_nr(pn2);
    const double pn = pn2 * rinv, n = p * rinv;
    const double cop = m.c * rinv;  // c/|P|
    const double g = m.g[0], K = m.K[0][0];
    k[Lo::Q] = m.c * n;
    k[Lo::P] = -pn * g;
    const double ng = n * g;
    // dA/dt = (A g) n + (c/|P|)(B - (B n) n) (the second term vanishes for n = +-1, kept
    // as written), dB/dt = -(|P| A K + (B n) g)
    const double bnr = y[Lo::BR] * n, bni = y[Lo::BI] * n;
    k[Lo::AR] = fma(y[Lo::AR] * g, n, cop * fma(-bnr, n, y[Lo::BR]));
    k[Lo::AI] = fma(y[Lo::AI] * g, n, cop * fma(-bni, n, y[Lo::BI]));
    k[Lo::BR] = -fma(pn, y[Lo::AR] * K, bnr * g);
    k[Lo::BI] = -fma(pn, y[Lo::AI] * K, bni * g);
    const double zr = y[Lo::AR] - y[Lo::BI], zi = y[Lo::AI] + y[Lo::BR];
    const double dzr = k[Lo::AR] - k[Lo::BI], dzi = k[Lo::AI] + k[Lo::BR];
    const double dd = fma(zr, zr, zi * zi);
    const double ih = 0.5 * rcp_nr(dd);
    const double qr = fma(dzr, zr, dzi * zi) * ih, qi = fma(dzi, zr, -dzr * zi) * ih;
    const double fr = ng + qr;
    const double ar = y[Lo::aR], ai = y[Lo::aI];
    k[Lo::aR] = fma(ar, fr, -ai * qi);
    k[Lo::aI] = fma(ar, qi, ai * fr);
    return pn2 > 0.0 && dd > 0.0;
  }
}

// Initial state of Gaussian (q index qf, p index pj): Q = q, P = p, A = I, B = -iI,
// a = 2^{d/2}, S = 0.
template <int D>
__device__ __forceinline__ void ray_init(const GridDev& gd, const ShotDev& sh, int64_t qf, int64_t pj,
                                         double* y) {
  using Lo = Layout<D>;
#pragma unroll
  for (int i = 0; i < Lo::NF; ++i) y[i] = 0.0;
  int64_t qm[D], pm[D];
  if constexpr (D == 1) {
    qm[0] = qf;
    pm[0] = pj - sh.nb[0] / 2;
  } else if constexpr (D == 3) {
    const int64_t nq12 = sh.nq[1] * sh.nq[2];
    qm[0] = qf / nq12;
    qm[1] = (qf - qm[0] * nq12) / sh.nq[2];
    qm[2] = qf - qm[0] * nq12 - qm[1] * sh.nq[2];
    const int64_t nb12 = (int64_t)sh.nb[1] * sh.nb[2];
    const int64_t j0 = pj / nb12, j1 = (pj - j0 * nb12) / sh.nb[2], j2 = pj - j0 * nb12 - j1 * sh.nb[2];
    pm[0] = j0 - sh.nb[0] / 2;
    pm[1] = j1 - sh.nb[1] / 2;
    pm[2] = j2 - sh.nb[2] / 2;
  } else {
    qm[0] = qf / sh.nq[1];
    qm[1] = qf - qm[0] * sh.nq[1];
    int64_t j0 = pj / sh.nb[1];
    pm[0] = j0 - sh.nb[0] / 2;
    pm[1] = (pj - j0 * sh.nb[1]) - sh.nb[1] / 2;
  }
#pragma unroll
  for (int i = 0; i < D; ++i) {
    y[Lo::Q + i] = gd.o[i] + (double)(sh.s[i] * qm[i]) * gd.h[i];
    y[Lo::P + i] = (double)pm[i] * sh.pscale[i];
    y[Lo::AR + i * D + i] = 1.0;
    y[Lo::BI + i * D + i] = -1.0;
  }
  y[Lo::aR] = D == 1 ? 1.4142135623730951 : (D == 2 ? 2.0 : 2.8284271247461903);  // 2^{d/2}
}

// Final state (structure of arrays) and coefficient 2 W a psi (2 pi eps)^{-3d/2} e^{iS/eps}.
template <int D>
__device__ __forceinline__ bool ray_store(const ShotDev& sh, int64_t g, const double* y,
                                          const double2* __restrict__ gpsi, double* __restrict__ state,
                                          int64_t ld, double2* __restrict__ coef) {
  using Lo = Layout<D>;
#pragma unroll
  for (int i = 0; i < Lo::NF; ++i) state[i * ld + g] = y[i];
  double2 ps = gpsi[g];
  double sc = 2.0 * sh.W * sh.norm;
  double ar = y[Lo::aR], ai = y[Lo::aI];
  double pr = (ar * ps.x - ai * ps.y) * sc, pi = (ar * ps.y + ai * ps.x) * sc;
  double sn, cs;
  sincos(y[Lo::S] * sh.inv_eps, &sn, &cs);
  coef[g] = make_double2(pr * cs - pi * sn, pr * sn + pi * cs);
  bool fin = isfinite(y[Lo::aR]) && isfinite(y[Lo::aI]) && isfinite(y[Lo::S]);
#pragma unroll
  for (int i = 0; i < D; ++i) fin = fin && isfinite(y[Lo::Q + i]) && isfinite(y[Lo::P + i]);
  return fin;
}

// Calls fn(r, d[], X) for every receiver r (internal index) inside the window
// |x_r,k - Q_k| <= cut of the Gaussian with centre Q and momentum P (open axes), with
// d = x_r - Q and X = exp(i P.d/eps - |d|^2/(2 eps)) (complex, as double2). Receivers on
// runs get X by the recurrence X_{k+1} = X_k R_k, R_{k+1} = R_k exp(-dl^2/eps) along the
// run (dl the spacing: two exponentials and two sine/cosine pairs per run instead of one
// pair per receiver) and their positions from the run's geometry (within a few ulps of
// the given coordinates, checked when the runs are formed); the other receivers are
// evaluated one by one from their coordinates.
template <int D, typename Fn>
__device__ __forceinline__ void for_receivers_X(const GridDev& gd, const RxDev& rx, const double* Q,
                                                const double* P, double cut, double inv_eps, Fn fn) {
  // runs (1D and 2D: in 3D every receiver is evaluated from its coordinates)
  if constexpr (D <= 2) for (int64_t j = 0; j < rx.nruns; ++j) {
    // the run's axis is a runtime value: select with conditionals rather than index Q
    // and P with it (a runtime index would move the ray state to local memory)
    const bool a1 = D == 2 && rx.run_axis[j] == 1;
    const double qa = a1 ? Q[D - 1] : Q[0], pa = a1 ? P[D - 1] : P[0];
    const double x0 = rx.run_geo[3 * j], dl = rx.run_geo[3 * j + 1];
    double fr = 1.0, fi = 0.0;  // factor of the coordinate across the run
    double e = 0.0;
    if constexpr (D == 2) {
      const double qb = a1 ? Q[0] : Q[1], pb = a1 ? P[0] : P[1];
      e = rx.run_geo[3 * j + 2] - qb;
      if (fabs(e) > cut) continue;
      double s, c;
      sincos(pb * e * inv_eps, &s, &c);
      const double g = exp(-0.5 * e * e * inv_eps);
      fr = g * c;
      fi = g * s;
    }
    const int64_t r0 = rx.run_off[j], n = rx.run_off[j + 1] - r0;
    // candidates, one beyond each end of the window
    int64_t k0 = (int64_t)ceil((qa - cut - x0) / dl) - 1;
    int64_t k1 = (int64_t)floor((qa + cut - x0) / dl) + 1;
    k0 = k0 < 0 ? 0 : k0;
    k1 = k1 > n - 1 ? n - 1 : k1;
    if (k0 > k1) continue;
    double u = fma((double)k0, dl, x0) - qa;
    double s, c;
    sincos(pa * u * inv_eps, &s, &c);
    double g = exp(-0.5 * u * u * inv_eps);
    double xr = g * c * fr - g * s * fi, xi = g * c * fi + g * s * fr;
    sincos(pa * dl * inv_eps, &s, &c);
    g = exp(-(u * dl + 0.5 * dl * dl) * inv_eps);
    double rr = g * c, ri = g * s;
    const double rho = exp(-dl * dl * inv_eps);
    for (int64_t k = k0; k <= k1; ++k) {
      u = fma((double)k, dl, x0) - qa;
      if (fabs(u) <= cut) {
        double d[D];
        if constexpr (D == 2) {
          d[0] = a1 ? e : u;
          d[1] = a1 ? u : e;
        } else {
          d[0] = u;
        }
        fn(r0 + k, d, make_double2(xr, xi));
      }
      const double nr = xr * rr - xi * ri, ni = xr * ri + xi * rr;
      xr = nr;
      xi = ni;
      rr *= rho;
      ri *= rho;
    }
  }
  // the other receivers, by output tile
  int64_t tlo[D], thi[D];
#pragma unroll
  for (int k = 0; k < D; ++k) {
    int64_t lo = (int64_t)floor((Q[k] - cut - gd.o[k]) * gd.inv_h[k]) - 1;
    int64_t hi = (int64_t)ceil((Q[k] + cut - gd.o[k]) * gd.inv_h[k]) + 1;
    if (hi < 0 || lo > gd.n[k] - 1) return;
    lo = lo < 0 ? 0 : lo;
    hi = hi > gd.n[k] - 1 ? gd.n[k] - 1 : hi;
    tlo[k] = lo / gd.tile[k];
    thi[k] = hi / gd.tile[k];
  }
  auto direct = [&](int64_t r) {
    double d[D], ph = 0.0, r2 = 0.0;
    bool in = true;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      d[k] = rx.x[r * D + k] - Q[k];
      in = in && fabs(d[k]) <= cut;
      ph = fma(P[k], d[k], ph);
      r2 = fma(d[k], d[k], r2);
    }
    if (!in) return;
    const double g = exp(-0.5 * r2 * inv_eps);
    double s, c;
    sincos(ph * inv_eps, &s, &c);
    fn(r, d, make_double2(g * c, g * s));
  };
  if constexpr (D == 1) {
    for (int64_t t0 = tlo[0]; t0 <= thi[0]; ++t0)
      for (int64_t r = rx.off[t0]; r < rx.off[t0 + 1]; ++r) direct(r);
  } else if constexpr (D == 2) {
    for (int64_t t0 = tlo[0]; t0 <= thi[0]; ++t0)
      for (int64_t t1 = tlo[1]; t1 <= thi[1]; ++t1) {
        const int64_t bin = t0 * rx.ntile[1] + t1;
        for (int64_t r = rx.off[bin]; r < rx.off[bin + 1]; ++r) direct(r);
      }
  } else {
    for (int64_t t0 = tlo[0]; t0 <= thi[0]; ++t0)
      for (int64_t t1 = tlo[1]; t1 <= thi[1]; ++t1)
        for (int64_t t2 = tlo[2]; t2 <= thi[2]; ++t2) {
          const int64_t bin = (t0 * rx.ntile[1] + t1) * rx.ntile[2] + t2;
          for (int64_t r = rx.off[bin]; r < rx.off[bin + 1]; ++r) direct(r);
        }
  }
}

// Adds Re(e X(x_r)) to tr[r] for the receivers in the window of the Gaussian at (Q, P),
// with reductions the thread does not wait for (an atomic add whose result is awaited
// made trace recording about 8x slower).
template <int D>
__device__ __forceinline__ void add_traces(const GridDev& gd, const RxDev& rx, double cut, double inv_eps,
                                        const double* Q, const double* P, double er, double ei,
                                        double* __restrict__ tr) {
  for_receivers_X<D>(gd, rx, Q, P, cut, inv_eps, [&](int64_t r, const double*, double2 X) {
    red_add_f64(tr + r, er * X.x - ei * X.y);
  });
}

// Contribution of one Gaussian (state y, weight psi) to the traces at record m:
// Re(2 W a psi (2 pi eps)^{-3d/2} e^{iS/eps} exp(i P.d/eps - |d|^2/(2 eps))).
template <int D>
__device__ __forceinline__ void record_traces(const GridDev& gd, const ShotDev& sh, const RxDev& rx,
                                              double kappa, const double* y, double2 psi, int s,
                                              int64_t m, double* __restrict__ traces) {
  using Lo = Layout<D>;
  const double cut = kappa * sh.sqrt_eps;
  double sc = 2.0 * sh.W * sh.norm;
  double ar = y[Lo::aR], ai = y[Lo::aI];
  double pr = (ar * psi.x - ai * psi.y) * sc, pi = (ar * psi.y + ai * psi.x) * sc;
  double sn, cs;
  sincos(y[Lo::S] * sh.inv_eps, &sn, &cs);
  const double er = pr * cs - pi * sn, ei = pr * sn + pi * cs;
  double* tr = traces + ((int64_t)s * rx.nrec + m) * rx.nrx;
  add_traces<D>(gd, rx, cut, sh.inv_eps, y + Lo::Q, y + Lo::P, er, ei, tr);
}

}  // namespace fga
