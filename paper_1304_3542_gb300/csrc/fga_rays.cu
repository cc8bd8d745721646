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
#include "fga_ray_rhs.cuh"

namespace fga {

int state_fields(int dim) { return 2 * dim + 4 * dim * dim + 3; }

namespace {

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
                                              unsigned long long* next, RxDev rx,
                                              double* __restrict__ traces) {
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
    double2 psi = rx.every > 0 ? gpsi[g] : make_double2(0.0, 0.0);
    while (true) {
      if (rx.every > 0 && step % rx.every == 0)
        record_traces<D>(gd, shots[s], rx, kappa, y, psi, s, step / rx.every, traces);
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
        if (rx.every > 0) psi = gpsi[g];
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
  RxDev rx = p->rx;
  if (p->nrx > 0) {
    e = cudaMemsetAsync(p->d_traces, 0, sizeof(double) * p->nshots * rx.nrec * rx.nrx, p->stream);
    if (e != cudaSuccess) return e;
  } else {
    rx.every = 0;
  }
  if (p->grid.dim == 1)
    k_rays<1><<<blocks, 128, 0, p->stream>>>(p->grid, p->d_shots, p->d_coef, p->G, p->d_gshot,
                                             p->d_gq, p->d_gp, p->d_gpsi, p->nsteps, p->dt, p->kappa,
                                             p->integrate_exited, p->d_state, (int64_t)p->g_cap,
                                             p->d_gcoef, p->d_status, p->d_steps, p->d_steps + 1,
                                             rx, p->d_traces);
  else
    k_rays<2><<<blocks, 128, 0, p->stream>>>(p->grid, p->d_shots, p->d_coef, p->G, p->d_gshot,
                                             p->d_gq, p->d_gp, p->d_gpsi, p->nsteps, p->dt, p->kappa,
                                             p->integrate_exited, p->d_state, (int64_t)p->g_cap,
                                             p->d_gcoef, p->d_status, p->d_steps, p->d_steps + 1,
                                             rx, p->d_traces);
  p->launches += 1;
  return cudaGetLastError();
}

}  // namespace fga
