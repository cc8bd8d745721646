// Step 2 of the method with Z from divided differences (FGA_Z_DIVIDED; the alternative
// to Eqs. dzQ, dzP named after Eq. op_zZ). The ray, amplitude and action equations are
// those of fga_rays.cu; only the way d_zQ, d_zP enter Eq. a_formu differs.
#include <algorithm>

#include "fga_internal.cuh"
#include "fga_medium.cuh"
#include "fga_ray_rhs.cuh"

namespace fga {

namespace {

// FGA_Z_DIVIDED: d_zQ and d_zP by divided differences (the alternative named after
// Eq. op_zZ). A Gaussian carries its ray (Q, P), 4D auxiliary rays r = 4j + m started at
// q +- dq_j e_j (m = 0, 1) and p +- dp_j e_j (m = 2, 3), a and S, all integrated by the
// same RK4. With d_z = d_q - i d_p and central differences Dq_j, Dp_j across the pairs,
//   Z_jk = (Dq_j Q_k + Dp_j P_k) + i (Dq_j P_k - Dp_j Q_k),
// dZ/dt is the same combination of the auxiliary rays' rates, and both enter Eq.
// a_formu as in rhs<D>. Only c and grad c are needed (no Hessian), but at 1 + 4D points.
template <int D>
struct LayoutDD {
  static constexpr int NR = 4 * D;                   // auxiliary rays
  static constexpr int AUX = 2 * D;                  // first auxiliary value
  static constexpr int aR = AUX + NR * 2 * D, aI = aR + 1, S = aR + 2;
  static constexpr int NF = S + 1;                   // 13 (1D), 39 (2D)
};

// Eq. characline for H = c(Q)|P| at one ray; n.grad c and H for Eq. a_formu and dS/dt.
template <int D>
__device__ __forceinline__ bool ray_rates(const GridDev& gd, const double* y, double* k, double& ng,
                                          double& H) {
  Med m;
  medium_eval_tab<D>(gd, y, m);
  double pn2 = 0;
#pragma unroll
  for (int i = 0; i < D; ++i) pn2 = fma(y[D + i], y[D + i], pn2);
  const double rinv = rsqrt(pn2), pn = pn2 * rinv;
  double g = 0;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    const double n = y[D + i] * rinv;
    k[i] = m.c * n;
    k[D + i] = -pn * m.g[i];
    g = fma(n, m.g[i], g);
  }
  ng = g;
  H = m.c * pn;
  return pn2 > 0.0;
}

// Central differences of the auxiliary rays' values v (Q, P of ray r at v + 2 D r) into
// Z = zr + i zi, entry (j, k) at j D + k.
template <int D>
__device__ __forceinline__ void dd_matrix(const double* v, const double* i2dq, const double* i2dp,
                                          double* zr, double* zi) {
#pragma unroll
  for (int j = 0; j < D; ++j)
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const double* r0 = v + (4 * j) * 2 * D;
      const double* r1 = r0 + 2 * D;
      const double* r2 = r1 + 2 * D;
      const double* r3 = r2 + 2 * D;
      const double DqQ = (r0[k] - r1[k]) * i2dq[j], DqP = (r0[D + k] - r1[D + k]) * i2dq[j];
      const double DpQ = (r2[k] - r3[k]) * i2dp[j], DpP = (r2[D + k] - r3[D + k]) * i2dp[j];
      zr[j * D + k] = DqQ + DpP;
      zi[j * D + k] = DqP - DpQ;
    }
}

template <int D>
__device__ __forceinline__ bool rhs_dd(const GridDev& gd, const double* y, double* k,
                                       const double* i2dq, const double* i2dp) {
  using Lo = LayoutDD<D>;
  double ng, H, ngr, Hr;
  bool ok = ray_rates<D>(gd, y, k, ng, H);
#pragma unroll
  for (int r = 0; r < Lo::NR; ++r) ok &= ray_rates<D>(gd, y + Lo::AUX + 2 * D * r, k + Lo::AUX + 2 * D * r, ngr, Hr);
  double zr[D * D], zi[D * D], dzr[D * D], dzi[D * D];
  dd_matrix<D>(y + Lo::AUX, i2dq, i2dp, zr, zi);
  dd_matrix<D>(k + Lo::AUX, i2dq, i2dp, dzr, dzi);
  // tr(Z^{-1} dZ/dt) = tr(adj(Z) dZ/dt)/det Z
  double trr, tri, detr, deti;
  if constexpr (D == 1) {
    trr = dzr[0];
    tri = dzi[0];
    detr = zr[0];
    deti = zi[0];
  } else {
    trr = zr[3] * dzr[0] - zi[3] * dzi[0] - (zr[1] * dzr[2] - zi[1] * dzi[2]) -
          (zr[2] * dzr[1] - zi[2] * dzi[1]) + zr[0] * dzr[3] - zi[0] * dzi[3];
    tri = zr[3] * dzi[0] + zi[3] * dzr[0] - (zr[1] * dzi[2] + zi[1] * dzr[2]) -
          (zr[2] * dzi[1] + zi[2] * dzr[1]) + zr[0] * dzi[3] + zi[0] * dzr[3];
    detr = zr[0] * zr[3] - zi[0] * zi[3] - (zr[1] * zr[2] - zi[1] * zi[2]);
    deti = zr[0] * zi[3] + zi[0] * zr[3] - (zr[1] * zi[2] + zi[1] * zr[2]);
  }
  const double dd = fma(detr, detr, deti * deti);
  const double idd = 1.0 / dd;
  const double qr = (trr * detr + tri * deti) * idd, qi = (tri * detr - trr * deti) * idd;
  const double fr = ng + 0.5 * qr, fi = 0.5 * qi;
  const double ar = y[Lo::aR], ai = y[Lo::aI];
  k[Lo::aR] = ar * fr - ai * fi;
  k[Lo::aI] = ar * fi + ai * fr;
  double pq = 0;
#pragma unroll
  for (int i = 0; i < D; ++i) pq = fma(y[D + i], k[i], pq);
  k[Lo::S] = pq - H;
  return ok && dd > 0.0;
}

// Persistent like k_rays (no receivers): a thread takes the next Gaussian from the
// counter when its ray is done. The stored state has the layout of the dynamic-ray
// kernels, with A = Dq Q - i Dp Q and B = Dq P - i Dp P at the final time.
template <int D>
__global__ void __launch_bounds__(128) k_rays_dd(GridDev gd, const ShotDev* __restrict__ shots, int64_t G,
                                                 const int32_t* __restrict__ gshot,
                                                 const int64_t* __restrict__ gq,
                                                 const int32_t* __restrict__ gp,
                                                 const double2* __restrict__ gpsi, int64_t nsteps,
                                                 double dt, double kappa, int integrate_exited,
                                                 double eta, double* __restrict__ state, int64_t ld,
                                                 double2* __restrict__ coef, int* status,
                                                 unsigned long long* steps_done,
                                                 unsigned long long* next, unsigned long long mult,
                                                 int32_t* __restrict__ gsteps) {
  using Lo = LayoutDD<D>;
  using Ls = Layout<D>;
  constexpr int NF = Lo::NF;
  unsigned long long my_steps = 0;
  bool ok = true;
  while (true) {
    const unsigned long long w = atomicAdd(next, 1ull);
    if (w >= (unsigned long long)G) break;
    const int64_t g = work_order(w, G, mult);
    const ShotDev& sh = shots[gshot[g]];
    double y[NF];
    {
      double y0[Ls::NF];
      ray_init<D>(gd, sh, gq[g], gp[g], y0);
#pragma unroll
      for (int i = 0; i < D; ++i) {
        y[i] = y0[Ls::Q + i];
        y[D + i] = y0[Ls::P + i];
      }
      y[Lo::aR] = y0[Ls::aR];
      y[Lo::aI] = 0.0;
      y[Lo::S] = 0.0;
    }
    double i2dq[D], i2dp[D];
#pragma unroll
    for (int j = 0; j < D; ++j) {
      const double dq = eta * (double)sh.s[j] * gd.h[j], dp = eta * sh.pscale[j];
      i2dq[j] = 0.5 / dq;
      i2dp[j] = 0.5 / dp;
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        double* r = y + Lo::AUX + 2 * D * (4 * j + m);
#pragma unroll
        for (int i = 0; i < 2 * D; ++i) r[i] = y[i];
        if (m == 0) r[j] += dq;
        if (m == 1) r[j] -= dq;
        if (m == 2) r[D + j] += dp;
        if (m == 3) r[D + j] -= dp;
      }
    }
    double lo[D], hi[D];
#pragma unroll
    for (int i = 0; i < D; ++i) {
      const double reach = kappa * sh.sqrt_eps + 2.0 * gd.h[i];
      lo[i] = gd.o[i] - reach;
      hi[i] = gd.o[i] + (double)(gd.n[i] - 1) * gd.h[i] + reach;
    }
    const double h2 = 0.5 * dt, h6 = dt / 6.0, h3 = dt / 3.0;
    int64_t step = 0;
    while (step < nsteps) {
      if (!integrate_exited) {
        bool gone = false;
#pragma unroll
        for (int i = 0; i < D; ++i)
          gone = gone || (!gd.periodic[i] && ((y[i] < lo[i] && y[D + i] <= 0.0) ||
                                              (y[i] > hi[i] && y[D + i] >= 0.0)));
        if (gone) break;
      }
      double acc[NF], tmp[NF], k[NF];
      ok &= rhs_dd<D>(gd, y, k, i2dq, i2dp);
#pragma unroll
      for (int i = 0; i < NF; ++i) {
        acc[i] = fma(h6, k[i], y[i]);
        tmp[i] = fma(h2, k[i], y[i]);
      }
      ok &= rhs_dd<D>(gd, tmp, k, i2dq, i2dp);
#pragma unroll
      for (int i = 0; i < NF; ++i) {
        acc[i] = fma(h3, k[i], acc[i]);
        tmp[i] = fma(h2, k[i], y[i]);
      }
      ok &= rhs_dd<D>(gd, tmp, k, i2dq, i2dp);
#pragma unroll
      for (int i = 0; i < NF; ++i) {
        acc[i] = fma(h3, k[i], acc[i]);
        tmp[i] = fma(dt, k[i], y[i]);
      }
      ok &= rhs_dd<D>(gd, tmp, k, i2dq, i2dp);
#pragma unroll
      for (int i = 0; i < NF; ++i) y[i] = fma(h6, k[i], acc[i]);
      // the Gaussian's own centre wraps on periodic axes; the auxiliary rays do not (the
      // medium is periodic, and their differences must not jump by a period)
#pragma unroll
      for (int i = 0; i < D; ++i) {
        if (gd.periodic[i]) {
          double r = fmod(y[i] - gd.o[i], gd.L[i]);
          if (r < 0) r += gd.L[i];
          y[i] = gd.o[i] + r;
        }
      }
      ++step;
    }
    double out[Ls::NF];
#pragma unroll
    for (int i = 0; i < D; ++i) {
      out[Ls::Q + i] = y[i];
      out[Ls::P + i] = y[D + i];
    }
#pragma unroll
    for (int j = 0; j < D; ++j)
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const double* r0 = y + Lo::AUX + (4 * j) * 2 * D;
        const double* r1 = r0 + 2 * D;
        const double* r2 = r1 + 2 * D;
        const double* r3 = r2 + 2 * D;
        out[Ls::AR + j * D + k] = (r0[k] - r1[k]) * i2dq[j];
        out[Ls::AI + j * D + k] = -(r2[k] - r3[k]) * i2dp[j];
        out[Ls::BR + j * D + k] = (r0[D + k] - r1[D + k]) * i2dq[j];
        out[Ls::BI + j * D + k] = -(r2[D + k] - r3[D + k]) * i2dp[j];
      }
    out[Ls::aR] = y[Lo::aR];
    out[Ls::aI] = y[Lo::aI];
    out[Ls::S] = y[Lo::S];
    ok &= ray_store<D>(sh, g, out, gpsi, state, ld, coef);
    gsteps[g] = (int32_t)step;
    my_steps += (unsigned long long)step;
  }
  if (!ok) atomicOr(status, kStatusNumeric);
  if (my_steps) atomicAdd(steps_done, my_steps);
}

}  // namespace

// Persistent launch over all Gaussians: the occupancy limit of blocks per SM on every SM
// (no tuning), at most one thread per Gaussian.
cudaError_t launch_rays_dd(fga_plan_s* p, int64_t nsteps) {
  cudaError_t e = cudaMemsetAsync(p->d_steps, 0, 2 * sizeof(unsigned long long), p->stream);
  if (e != cudaSuccess || p->G == 0) return e;
  auto kern = p->grid.dim == 1 ? k_rays_dd<1> : k_rays_dd<2>;
  int dev = 0, sms = 0, per_sm = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 128, 0);
  if (e != cudaSuccess) return e;
  const int64_t blocks = std::max<int64_t>(
      1, std::min<int64_t>((int64_t)sms * std::max(per_sm, 1), (p->G + 127) / 128));
  kern<<<(unsigned)blocks, 128, 0, p->stream>>>(p->grid, p->d_shots, p->G, p->d_gshot, p->d_gq,
                                                p->d_gp, p->d_gpsi, nsteps, p->dt, p->kappa,
                                                p->integrate_exited, p->dz_eta, p->d_state,
                                                (int64_t)p->g_cap, p->d_gcoef, p->d_status,
                                                p->d_steps, p->d_steps + 1,
                                                work_order_mult(p->G), p->d_gsteps);
  p->launches += 1;
  return cudaGetLastError();
}

}  // namespace fga
