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

// 1/x for x > 0: the hardware's approximate reciprocal (PTX rcp.approx.ftz.f64, about
// 20 correct bits) refined by two Newton-Raphson steps r <- r + r (1 - x r), each
// doubling the correct bits (within an ulp of 1/x; measured on GB300 over x in
// [2^-40, 2^40]).
__device__ __forceinline__ double rcp_nr(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}

// 1/sqrt(x) for x > 0: the hardware's approximation (PTX rsqrt.approx.ftz.f64, about
// 20 correct bits) refined by one third-order Householder step for x^{-1/2}: with
// e = 1 - x y^2, y <- y (1 + e/2 + 3 e^2/8), which cubes the relative error (about one
// ulp remains; measured on GB300 over x in [2^-40, 2^40]).
__device__ __forceinline__ double rsqrt_nr(double x) {
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  const double e = fma(-x * y, y, 1.0);
  return fma(y * e, fma(0.375, e, 0.5), y);
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

// The medium comes from the per-cell polynomial table gd.tab.
template <int D>
__device__ __forceinline__ bool rhs(const GridDev& gd, const double* y, double* k) {
  if constexpr (D == 2) return rhs2(gd, y, k);
  using Lo = Layout<D>;
  Med m;
  medium_eval_tab<D>(gd, y + Lo::Q, m);
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
  } else if constexpr (D == 3) {
    // Z = A + iB and dZ/dt (3 x 3 complex); tr(adj(Z) dZ) and det Z by cofactors
    double zr[9], zi[9], dzr[9], dzi[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      zr[e] = y[Lo::AR + e] - y[Lo::BI + e];
      zi[e] = y[Lo::AI + e] + y[Lo::BR + e];
      dzr[e] = k[Lo::AR + e] - k[Lo::BI + e];
      dzi[e] = k[Lo::AI + e] + k[Lo::BR + e];
    }
    // cofactor C[i][j] = (-1)^{i+j} det(minor ij); adj(Z)[j][i] = C[i][j]
    double cr[9], ci[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const int r0 = (i + 1) % 3, r1 = (i + 2) % 3, c0 = (j + 1) % 3, c1 = (j + 2) % 3;
        // cyclic minors carry the sign (-1)^{i+j} already
        const double ar = zr[r0 * 3 + c0], ai = zi[r0 * 3 + c0], br = zr[r1 * 3 + c1], bi = zi[r1 * 3 + c1];
        const double er = zr[r0 * 3 + c1], ei = zi[r0 * 3 + c1], fr = zr[r1 * 3 + c0], fi = zi[r1 * 3 + c0];
        cr[i * 3 + j] = (ar * br - ai * bi) - (er * fr - ei * fi);
        ci[i * 3 + j] = (ar * bi + ai * br) - (er * fi + ei * fr);
      }
    // tr(adj(Z) dZ) = sum_{i,j} C[i][j] dZ[i][j];  det Z = sum_j Z[0][j] C[0][j]
    trr = 0.0;
    tri = 0.0;
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      trr += cr[e] * dzr[e] - ci[e] * dzi[e];
      tri += cr[e] * dzi[e] + ci[e] * dzr[e];
    }
    detr = 0.0;
    deti = 0.0;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      detr += zr[j] * cr[j] - zi[j] * ci[j];
      deti += zr[j] * ci[j] + zi[j] * cr[j];
    }
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
