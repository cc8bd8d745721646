// Right-hand side of the FGA ray system shared by the forward integrator and the
// adjoint: Eqs. characline, dzQ, dzP, a_formu (Z of Eq. op_zZ) and dS/dt = P.dQ/dt - H
// for the + branch, H = c(Q)|P|; plus the initial state and the stored outputs.
#pragma once

#include "fga_internal.cuh"
#include "fga_medium.cuh"

namespace fga {

template <int D>
struct Layout {
  static constexpr int NF = 2 * D + 4 * D * D + 3;
  static constexpr int Q = 0, P = D, AR = 2 * D, AI = 2 * D + D * D, BR = 2 * D + 2 * D * D,
                       BI = 2 * D + 3 * D * D, aR = 2 * D + 4 * D * D, aI = aR + 1, S = aR + 2;
};

template <int D>
__device__ __forceinline__ bool rhs(const GridDev& gd, const double* __restrict__ C, const double* y,
                                    double* k) {
  using Lo = Layout<D>;
  Med m;
  medium_eval<D>(gd, C, y + Lo::Q, m);
  double pn2 = 0;
#pragma unroll
  for (int i = 0; i < D; ++i) pn2 = fma(y[Lo::P + i], y[Lo::P + i], pn2);
  double rinv = rsqrt(pn2);
  double pn = pn2 * rinv;
  double n[D];
#pragma unroll
  for (int i = 0; i < D; ++i) n[i] = y[Lo::P + i] * rinv;
  double cop = m.c * rinv;  // c/|P|
  double ng = 0;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    k[Lo::Q + i] = m.c * n[i];
    k[Lo::P + i] = -pn * m.g[i];
    ng = fma(n[i], m.g[i], ng);
  }
  // dynamic rays
#pragma unroll
  for (int j = 0; j < D; ++j) {
    double agr = 0, agi = 0, bnr = 0, bni = 0;
#pragma unroll
    for (int l = 0; l < D; ++l) {
      agr = fma(y[Lo::AR + j * D + l], m.g[l], agr);
      agi = fma(y[Lo::AI + j * D + l], m.g[l], agi);
      bnr = fma(y[Lo::BR + j * D + l], n[l], bnr);
      bni = fma(y[Lo::BI + j * D + l], n[l], bni);
    }
#pragma unroll
    for (int kk = 0; kk < D; ++kk) {
      double akr = 0, aki = 0;
#pragma unroll
      for (int l = 0; l < D; ++l) {
        akr = fma(y[Lo::AR + j * D + l], m.K[l][kk], akr);
        aki = fma(y[Lo::AI + j * D + l], m.K[l][kk], aki);
      }
      k[Lo::AR + j * D + kk] = fma(agr, n[kk], cop * fma(-bnr, n[kk], y[Lo::BR + j * D + kk]));
      k[Lo::AI + j * D + kk] = fma(agi, n[kk], cop * fma(-bni, n[kk], y[Lo::BI + j * D + kk]));
      k[Lo::BR + j * D + kk] = -fma(pn, akr, bnr * m.g[kk]);
      k[Lo::BI + j * D + kk] = -fma(pn, aki, bni * m.g[kk]);
    }
  }
  // tr(Z^{-1} dZ/dt), Z = A + iB, dZ/dt = dA + i dB
  double trr, tri, detr, deti;
  if constexpr (D == 1) {
    double zr = y[Lo::AR] - y[Lo::BI], zi = y[Lo::AI] + y[Lo::BR];
    double dzr = k[Lo::AR] - k[Lo::BI], dzi = k[Lo::AI] + k[Lo::BR];
    trr = dzr;
    tri = dzi;
    detr = zr;
    deti = zi;
  } else {
    double zr[4], zi[4], dzr[4], dzi[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      zr[e] = y[Lo::AR + e] - y[Lo::BI + e];
      zi[e] = y[Lo::AI + e] + y[Lo::BR + e];
      dzr[e] = k[Lo::AR + e] - k[Lo::BI + e];
      dzi[e] = k[Lo::AI + e] + k[Lo::BR + e];
    }
    // adj(Z) : dZ = Z11 dZ00 - Z01 dZ10 - Z10 dZ01 + Z00 dZ11
    trr = zr[3] * dzr[0] - zi[3] * dzi[0] - (zr[1] * dzr[2] - zi[1] * dzi[2]) -
          (zr[2] * dzr[1] - zi[2] * dzi[1]) + zr[0] * dzr[3] - zi[0] * dzi[3];
    tri = zr[3] * dzi[0] + zi[3] * dzr[0] - (zr[1] * dzi[2] + zi[1] * dzr[2]) -
          (zr[2] * dzi[1] + zi[2] * dzr[1]) + zr[0] * dzi[3] + zi[0] * dzr[3];
    detr = zr[0] * zr[3] - zi[0] * zi[3] - (zr[1] * zr[2] - zi[1] * zi[2]);
    deti = zr[0] * zi[3] + zi[0] * zr[3] - (zr[1] * zi[2] + zi[1] * zr[2]);
  }
  double dd = fma(detr, detr, deti * deti);
  double idd = 1.0 / dd;
  double qr = (trr * detr + tri * deti) * idd, qi = (tri * detr - trr * deti) * idd;
  double fr = ng + 0.5 * qr, fi = 0.5 * qi;
  double ar = y[Lo::aR], ai = y[Lo::aI];
  k[Lo::aR] = ar * fr - ai * fi;
  k[Lo::aI] = ar * fi + ai * fr;
  double pq = 0;
#pragma unroll
  for (int i = 0; i < D; ++i) pq = fma(y[Lo::P + i], k[Lo::Q + i], pq);
  k[Lo::S] = pq - m.c * pn;
  return pn2 > 0.0 && dd > 0.0;
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
  y[Lo::aR] = (D == 1) ? 1.4142135623730951 : 2.0;
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

// Calls fn(r, d[]) for every receiver r inside the window |x_r,k - Q_k| <= cut of the
// Gaussian with centre Q (open axes), d = x_r - Q.
template <int D, typename Fn>
__device__ __forceinline__ void for_receivers_in_window(const GridDev& gd, const RxDev& rx,
                                                        const double* Q, double cut, Fn fn) {
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
  if constexpr (D == 1) {
    for (int64_t t0 = tlo[0]; t0 <= thi[0]; ++t0)
      for (int64_t e = rx.off[t0]; e < rx.off[t0 + 1]; ++e) {
        int32_t r = rx.list[e];
        double d[1] = {rx.x[r] - Q[0]};
        if (fabs(d[0]) <= cut) fn(r, d);
      }
  } else {
    for (int64_t t0 = tlo[0]; t0 <= thi[0]; ++t0)
      for (int64_t t1 = tlo[1]; t1 <= thi[1]; ++t1) {
        int64_t bin = t0 * rx.ntile[1] + t1;
        for (int64_t e = rx.off[bin]; e < rx.off[bin + 1]; ++e) {
          int32_t r = rx.list[e];
          double d[2] = {rx.x[2 * r] - Q[0], rx.x[2 * r + 1] - Q[1]};
          if (fabs(d[0]) <= cut && fabs(d[1]) <= cut) fn(r, d);
        }
      }
  }
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
  for_receivers_in_window<D>(gd, rx, y + Lo::Q, cut, [&](int32_t r, const double* d) {
    double ph = 0.0, r2 = 0.0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      ph = fma(y[Lo::P + k], d[k], ph);
      r2 = fma(d[k], d[k], r2);
    }
    double gs = exp(-0.5 * r2 * sh.inv_eps);
    double s2, c2;
    sincos(ph * sh.inv_eps, &s2, &c2);
    atomicAdd(tr + r, gs * (er * c2 - ei * s2));
  });
}

}  // namespace fga
