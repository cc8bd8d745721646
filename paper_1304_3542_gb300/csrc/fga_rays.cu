// Step 2 of the method: time propagation of every kept Gaussian of the + branch.
//
// State per Gaussian (FP64, in registers for the whole trajectory):
//   Q, P (Eq. characline with H = c(Q)|P|, Eq. hamiltonian),
//   A = d_zQ, B = d_zP, (j,k) entry d_{z_j} Q_k (Eqs. dzQ, dzP),
//   a (Eq. a_formu, Z = A + iB from Eq. op_zZ) and the action S (dS/dt = P.dQ/dt - H).
// With n = P/|P|, g = grad c(Q), K = Hessian of c(Q), the second derivatives of H
// are H_QP[l][k] = g_l n_k, H_PQ[l][k] = n_l g_k, H_PP = c (I - n n^T)/|P| and
// H_QQ = |P| K, so the dynamic ray equations collapse to
//   dA_jk/dt = (A g)_j n_k + (c/|P|) (B_jk - (B n)_j n_k),
//   dB_jk/dt = -(|P| (A K)_jk + (B n)_j g_k),
// and (dP_H . dQ_H)/H = n . g. One thread integrates one Gaussian with classical
// RK4 (Numerical test section) for all T/dt steps; the velocity is read through the
// read-only cache (its spline coefficients stay resident in L2). The epilogue stores
// the state (structure of arrays, coalesced) and the complex coefficient of the
// reconstruction sum, 2 W a psi (2 pi eps)^{-3d/2} e^{i S/eps} (the 2 accounts for the
// conjugate - branch). Unless asked to integrate every ray to T, a ray stops once its
// window has left an open axis for good (see fga_config.integrate_exited); the kernel
// is persistent (one grid of resident blocks pulling Gaussians from a counter) so that
// lanes whose ray stopped early pick up new work instead of idling in their warp.
#include <algorithm>

#include "fga_internal.cuh"
#include "fga_medium.cuh"

namespace fga {

int state_fields(int dim) { return 2 * dim + 4 * dim * dim + 3; }

namespace {

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

// Persistent integrator: every lane takes the next Gaussian from a global counter as
// soon as its ray has reached T (or left the grid for good), so the warps stay full
// whatever the mix of ray lifetimes. Each ray's arithmetic does not depend on which
// lane runs it, so the results are the same as with one thread per Gaussian.
template <int D>
__global__ void __launch_bounds__(128) k_rays(GridDev gd, const ShotDev* __restrict__ shots,
                                              const double* __restrict__ C, int64_t G,
                                              const int32_t* __restrict__ gshot,
                                              const int64_t* __restrict__ gq,
                                              const int32_t* __restrict__ gp,
                                              const double2* __restrict__ gpsi, int64_t nsteps,
                                              double dt, double kappa, int integrate_exited,
                                              double* __restrict__ state, int64_t ld,
                                              double2* __restrict__ coef, int* status,
                                              unsigned long long* steps_done,
                                              unsigned long long* next) {
  using Lo = Layout<D>;
  constexpr int NF = Lo::NF;
  int64_t g = (int64_t)atomicAdd(next, 1ull);
  unsigned long long my_steps = 0;
  bool ok = true;
  if (g < G) {
    int s = gshot[g];
    double y[NF];
    ray_init<D>(gd, shots[s], gq[g], gp[g], y);
    // exit box: beyond these bounds on an open axis the window misses the grid and the
    // spline's taps are all clamped, so c does not depend on Q_k there
    double lo[D], hi[D];
#pragma unroll
    for (int i = 0; i < D; ++i) {
      double reach = kappa * shots[s].sqrt_eps + 2.0 * gd.h[i];
      lo[i] = gd.o[i] - reach;
      hi[i] = gd.o[i] + (double)(gd.n[i] - 1) * gd.h[i] + reach;
    }
    const double h2 = 0.5 * dt, h6 = dt / 6.0, h3 = dt / 3.0;
    int64_t step = 0;
    while (true) {
      bool done = step >= nsteps;
      if (!done && !integrate_exited) {
#pragma unroll
        for (int i = 0; i < D; ++i)
          done = done || (!gd.periodic[i] && ((y[Lo::Q + i] < lo[i] && y[Lo::P + i] <= 0.0) ||
                                              (y[Lo::Q + i] > hi[i] && y[Lo::P + i] >= 0.0)));
      }
      if (done) {
        ok &= ray_store<D>(shots[s], g, y, gpsi, state, ld, coef);
        my_steps += (unsigned long long)step;
        g = (int64_t)atomicAdd(next, 1ull);
        if (g >= G) break;
        s = gshot[g];
        ray_init<D>(gd, shots[s], gq[g], gp[g], y);
#pragma unroll
        for (int i = 0; i < D; ++i) {
          double reach = kappa * shots[s].sqrt_eps + 2.0 * gd.h[i];
          lo[i] = gd.o[i] - reach;
          hi[i] = gd.o[i] + (double)(gd.n[i] - 1) * gd.h[i] + reach;
        }
        step = 0;
        continue;
      }
      double acc[NF], tmp[NF], k[NF];
      ok &= rhs<D>(gd, C, y, k);
#pragma unroll
      for (int i = 0; i < NF; ++i) {
        acc[i] = fma(h6, k[i], y[i]);
        tmp[i] = fma(h2, k[i], y[i]);
      }
      ok &= rhs<D>(gd, C, tmp, k);
#pragma unroll
      for (int i = 0; i < NF; ++i) {
        acc[i] = fma(h3, k[i], acc[i]);
        tmp[i] = fma(h2, k[i], y[i]);
      }
      ok &= rhs<D>(gd, C, tmp, k);
#pragma unroll
      for (int i = 0; i < NF; ++i) {
        acc[i] = fma(h3, k[i], acc[i]);
        tmp[i] = fma(dt, k[i], y[i]);
      }
      ok &= rhs<D>(gd, C, tmp, k);
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
      ++step;
    }
  }
  if (!ok) atomicOr(status, kStatusNumeric);
  // steps integrated (one atomic per resident thread)
  if (my_steps) atomicAdd(steps_done, my_steps);
}

}  // namespace

cudaError_t launch_rays(fga_plan_s* p) {
  // d_steps[0]: steps integrated; d_steps[1]: the work counter of the persistent kernel
  cudaError_t e = cudaMemsetAsync(p->d_steps, 0, 2 * sizeof(unsigned long long), p->stream);
  if (e != cudaSuccess) return e;
  if (p->G == 0) return cudaSuccess;
  if (p->ray_blocks == 0) {
    int dev = 0, sms = 0, per_sm = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
      e = p->grid.dim == 1
              ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rays<1>, 128, 0)
              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rays<2>, 128, 0);
    if (e != cudaSuccess) return e;
    p->ray_blocks = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
  }
  unsigned blocks = (unsigned)std::min<int64_t>(p->ray_blocks, (p->G + 127) / 128);
  if (p->grid.dim == 1)
    k_rays<1><<<blocks, 128, 0, p->stream>>>(p->grid, p->d_shots, p->d_coef, p->G, p->d_gshot,
                                             p->d_gq, p->d_gp, p->d_gpsi, p->nsteps, p->dt, p->kappa,
                                             p->integrate_exited, p->d_state, (int64_t)p->g_cap,
                                             p->d_gcoef, p->d_status, p->d_steps, p->d_steps + 1);
  else
    k_rays<2><<<blocks, 128, 0, p->stream>>>(p->grid, p->d_shots, p->d_coef, p->G, p->d_gshot,
                                             p->d_gq, p->d_gp, p->d_gpsi, p->nsteps, p->dt, p->kappa,
                                             p->integrate_exited, p->d_state, (int64_t)p->g_cap,
                                             p->d_gcoef, p->d_status, p->d_steps, p->d_steps + 1);
  p->launches += 1;
  return cudaGetLastError();
}

}  // namespace fga
