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
// MINB = 1 lets the compiler use up to 255 registers per thread (2 blocks of 128 per SM
// for the 2D kernel); MINB = 3 caps them at 168 for 3 resident blocks (no spills in 2D,
// many in 3D). The autotuner picks one.
template <int D, int MINB>
__global__ void __launch_bounds__(128, MINB) k_rays(GridDev gd, const ShotDev* __restrict__ shots,
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
                                              double* __restrict__ trace_part, int64_t slice_len,
                                              int slices, unsigned long long mult,
                                              int32_t* __restrict__ gsteps,
                                              const int64_t* __restrict__ gm,
                                              const int32_t* __restrict__ order) {
  using Lo = Layout<D>;
  constexpr int NF = Lo::NF;
  if (gm) {  // counts kept on the device (pipeline graph)
    G = gm[0];
    mult = (unsigned long long)gm[1];
  }
  // this block's private slice of the trace sums (no other block adds into it)
  double* traces = rx.every > 0 ? trace_part + (int64_t)(blockIdx.x % slices) * slice_len : nullptr;
  unsigned long long w = atomicAdd(next, 1ull);
  // the w-th Gaussian to integrate: longest estimated ray first when an order is given
  auto nth = [&](unsigned long long w) -> int64_t {
    return order ? (int64_t)order[w] : work_order(w, G, mult);
  };
  int64_t g = w < (unsigned long long)G ? nth(w) : G;
  unsigned long long my_steps = 0;
  bool ok = true;
  if (g < G) {
    int s = gshot[g];
    // In 2D and 3D the step's starting state (23 or 45 values) lives in shared memory, a
    // thread's values NF (odd) doubles apart, which keeps a warp's accesses free of bank
    // conflicts. In 3D the stage state, the accumulator and the right-hand side would not
    // fit in 255 registers beside it; in 2D it frees registers (212 instead of 244; 166
    // without spills for three blocks per SM), 0.4 % faster on the layered workload.
    __shared__ double y_sm[D >= 2 ? 128 * NF : 1];
    double y_reg[D >= 2 ? 1 : NF];
    double* const y = D >= 2 ? y_sm + threadIdx.x * NF : y_reg;
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
    // With receivers, every ray's step 0 falls on a loop trip that is a multiple of the
    // record interval, so all lanes of a warp record on the same trips (a lane that
    // picks up a new ray idles until then, at most every - 1 trips).
    int64_t trip = 0, wait = 0;
    double2 psi = rx.every > 0 ? gpsi[g] : make_double2(0.0, 0.0);
    while (true) {
      if (wait > 0) {
        --wait;
        ++trip;
        continue;
      }
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
        gsteps[g] = (int32_t)step;
        my_steps += (unsigned long long)step;
        w = atomicAdd(next, 1ull);
        if (w >= (unsigned long long)G) break;
        g = nth(w);
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
        if (rx.every > 0) wait = (rx.every - (trip + 1) % rx.every) % rx.every;
        ++trip;
        continue;
      }
      // S (the last field) is not integrated: its right-hand side vanishes (Layout)
      constexpr int NI = Lo::NI;
      double acc[NF], tmp[NF], k[NF];
      tmp[Lo::S] = y[Lo::S];
      if constexpr (D == 3) {
        // the four stages as a loop around one copy of the (long) 3D right-hand side, so
        // that the kernel's code fits the instruction cache; the same operations in the
        // same order as the unrolled form
#pragma unroll
        for (int i = 0; i < NI; ++i) tmp[i] = y[i];
#pragma unroll 1
        for (int st = 0; st < 4; ++st) {
          ok &= rhs<D>(gd, tmp, k);
          if (st == 0) {
#pragma unroll
            for (int i = 0; i < NI; ++i) {
              acc[i] = fma(h6, k[i], y[i]);
              tmp[i] = fma(h2, k[i], y[i]);
            }
          } else if (st < 3) {
            const double wt = st == 1 ? h2 : dt;
#pragma unroll
            for (int i = 0; i < NI; ++i) {
              acc[i] = fma(h3, k[i], acc[i]);
              tmp[i] = fma(wt, k[i], y[i]);
            }
          } else {
#pragma unroll
            for (int i = 0; i < NI; ++i) y[i] = fma(h6, k[i], acc[i]);
          }
        }
      } else {
        ok &= rhs<D>(gd, y, k);
#pragma unroll
        for (int i = 0; i < NI; ++i) {
          acc[i] = fma(h6, k[i], y[i]);
          tmp[i] = fma(h2, k[i], y[i]);
        }
        ok &= rhs<D>(gd, tmp, k);
#pragma unroll
        for (int i = 0; i < NI; ++i) {
          acc[i] = fma(h3, k[i], acc[i]);
          tmp[i] = fma(h2, k[i], y[i]);
        }
        ok &= rhs<D>(gd, tmp, k);
#pragma unroll
        for (int i = 0; i < NI; ++i) {
          acc[i] = fma(h3, k[i], acc[i]);
          tmp[i] = fma(dt, k[i], y[i]);
        }
        ok &= rhs<D>(gd, tmp, k);
#pragma unroll
        for (int i = 0; i < NI; ++i) y[i] = fma(h6, k[i], acc[i]);
      }
#pragma unroll
      for (int i = 0; i < D; ++i) {
        if (gd.periodic[i]) {
          double r = fmod(y[Lo::Q + i] - gd.o[i], gd.L[i]);
          if (r < 0) r += gd.L[i];
          y[Lo::Q + i] = gd.o[i] + r;
        }
      }
      ++step;
      ++trip;
    }
  }
  if (!ok) atomicOr(status, kStatusNumeric);
  // steps integrated (one atomic per resident thread)
  if (my_steps) atomicAdd(steps_done, my_steps);
}

}  // namespace

namespace {

// Longest-first order of the rays (the persistent kernel's tail: the rays taken last
// should be the short ones). The length of a ray is estimated from its initial state as
// the straight-line time to the exit box of the ray kernel (the grid widened by
// kappa sqrt(eps) + 2h on every open axis) at the speed c(q): exact for a constant medium
// and a ray that leaves, a ranking heuristic otherwise (the integrated rays do not depend
// on the order). est[g] receives the estimated steps (overwritten by the ray kernel with
// the steps taken); cnt[b] counts the rays of bucket b = (nsteps - est) / width.
template <int D>
__global__ void k_ray_estimate(GridDev gd, const ShotDev* __restrict__ shots, const double* __restrict__ C,
                               int64_t G, const int64_t* __restrict__ gm, const int32_t* __restrict__ gshot,
                               const int64_t* __restrict__ gq, const int32_t* __restrict__ gp,
                               int64_t nsteps, double dt, double kappa, int32_t* __restrict__ est,
                               int64_t width, unsigned long long* __restrict__ cnt) {
  using Lo = Layout<D>;
  if (gm) G = gm[0];
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < G;
       g += (int64_t)gridDim.x * blockDim.x) {
    const ShotDev& sh = shots[gshot[g]];
    double y[Lo::NF];
    ray_init<D>(gd, sh, gq[g], gp[g], y);
    const double c = medium_value<D>(gd, C, y + Lo::Q);
    double pn2 = 0.0;
#pragma unroll
    for (int k = 0; k < D; ++k) pn2 = fma(y[Lo::P + k], y[Lo::P + k], pn2);
    const double cop = pn2 > 0.0 ? c / sqrt(pn2) : 0.0;
    double t = (double)nsteps * dt;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      if (gd.periodic[k]) continue;
      const double reach = kappa * sh.sqrt_eps + 2.0 * gd.h[k];
      const double lo = gd.o[k] - reach, hi = gd.o[k] + (double)(gd.n[k] - 1) * gd.h[k] + reach;
      const double v = cop * y[Lo::P + k], q = y[Lo::Q + k];
      if (v > 0.0) t = fmin(t, (hi - q) / v);
      if (v < 0.0) t = fmin(t, (lo - q) / v);
    }
    const double st = t / dt;
    const int64_t e = st >= (double)nsteps ? nsteps : (st > 0.0 ? (int64_t)st : 0);
    est[g] = (int32_t)e;
    atomicAdd(cnt + (nsteps - e) / width, 1ull);
  }
}

// Scatter of the Gaussians into the buckets' ranges (offsets fill[b] after the scan).
// With spread set (traces recorded), in the spread order work_order(w) within a bucket,
// so that rays running at the same time still come from all over the list and add into
// different trace entries. Without traces, in index order within a bucket: neighbouring
// Gaussians (one q, adjacent p) then run at the same time and end at about the same
// step, so the 8-byte state stores of the four rays that share a 32-byte sector of each
// state row meet in L2 and leave it as whole sectors instead of partial ones that are
// read back to be filled.
__global__ void k_ray_order(int64_t G, const int64_t* __restrict__ gm, unsigned long long mult,
                            int spread, const int32_t* __restrict__ est, int64_t nsteps,
                            int64_t width, unsigned long long* __restrict__ fill,
                            int32_t* __restrict__ order) {
  if (gm) {
    G = gm[0];
    mult = (unsigned long long)gm[1];
  }
  for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < G;
       w += (int64_t)gridDim.x * blockDim.x) {
    const int64_t g = spread ? work_order((unsigned long long)w, G, mult) : w;
    const int64_t b = (nsteps - est[g]) / width;
    order[atomicAdd(fill + b, 1ull)] = (int32_t)g;
  }
}

// One thread per table cell (cells -1 .. n per axis, stored at index + 1).
template <int D>
__global__ void k_medium_table(GridDev gd, const double* __restrict__ C, double* __restrict__ tab) {
  constexpr int NC = D == 1 ? 4 : (D == 2 ? 16 : 64);
  const int64_t n1 = D == 1 ? 1 : gd.n[1] + 2;
  const int64_t n2 = D == 3 ? gd.n[2] + 2 : 1;
  const int64_t cells = (gd.n[0] + 2) * n1 * n2;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < cells;
       c += (int64_t)gridDim.x * blockDim.x) {
    int64_t ci[3];
    if constexpr (D == 1) {
      ci[0] = c;
    } else if constexpr (D == 2) {
      ci[0] = c / n1;
      ci[1] = c % n1;
    } else {
      ci[0] = c / (n1 * n2);
      ci[1] = (c / n2) % n1;
      ci[2] = c % n2;
    }
    double a[NC];
    medium_cell<D>(gd, C, ci, a);
#pragma unroll
    for (int k = 0; k < NC; ++k) tab[c * NC + k] = a[k];
  }
}

// out[j] = sum_s part[s * len + i] in slice order (j: see launch_slice_sum).
__global__ void k_slice_sum(const double* __restrict__ part, int64_t slices, int64_t len,
                            double* __restrict__ out, const int32_t* __restrict__ perm,
                            int64_t row) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * blockDim.x) {
    double v = 0.0;
    for (int64_t s = 0; s < slices; ++s) v += part[s * len + i];
    const int64_t j = perm ? (i / row) * row + perm[i % row] : i;
    out[j] = v;
  }
}

__global__ void k_gather_rows(const double* __restrict__ in, const int32_t* __restrict__ perm,
                              int64_t len, int64_t row, double* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = in[(i / row) * row + perm[i % row]];
}

}  // namespace

size_t medium_table_doubles(const GridDev& gd) {
  size_t cells = 1;
  for (int k = 0; k < gd.dim; ++k) cells *= (size_t)(gd.n[k] + 2);
  return cells * ((size_t)1 << (2 * gd.dim));
}

cudaError_t launch_medium_table(fga_plan_s* p) {
  const size_t cells = medium_table_doubles(p->grid) >> (2 * p->grid.dim);
  const unsigned blocks = (unsigned)std::min<size_t>((cells + 255) / 256, 4096);
  if (p->grid.dim == 1)
    k_medium_table<1><<<blocks, 256, 0, p->stream>>>(p->grid, p->d_coef, p->d_medtab);
  else if (p->grid.dim == 2)
    k_medium_table<2><<<blocks, 256, 0, p->stream>>>(p->grid, p->d_coef, p->d_medtab);
  else
    k_medium_table<3><<<blocks, 256, 0, p->stream>>>(p->grid, p->d_coef, p->d_medtab);
  p->launches += 1;
  return cudaGetLastError();
}

unsigned long long work_order_mult(int64_t G) { return work_order_mult_of(G); }

int64_t ray_order_width(int64_t nsteps) { return std::max<int64_t>(1, std::min<int64_t>(16, nsteps / 64)); }

namespace {
using RayKernel = decltype(&k_rays<2, 1>);
RayKernel ray_kernel(const fga_plan_s* p) {
  const bool v3 = p->ray_variant == 1;
  if (p->grid.dim == 1) return v3 ? k_rays<1, 3> : k_rays<1, 1>;
  if (p->grid.dim == 2) return v3 ? k_rays<2, 3> : k_rays<2, 1>;
  return v3 ? k_rays<3, 3> : k_rays<3, 1>;
}
}  // namespace

int ray_max_per_sm(fga_plan_s* p) {
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ray_kernel(p), 128, 0);
  return (e == cudaSuccess && per_sm > 0) ? per_sm : 1;
}

cudaError_t ensure_ray_blocks(fga_plan_s* p) {
  if (p->ray_blocks > 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int max_sm = ray_max_per_sm(p);
  const int per_sm = p->ray_per_sm > 0 && p->ray_per_sm < max_sm ? p->ray_per_sm : max_sm;
  p->ray_blocks = (int64_t)sms * per_sm;
  return cudaSuccess;
}

int64_t ray_launch_blocks(fga_plan_s* p) {
  return std::max<int64_t>(1, std::min<int64_t>(p->ray_blocks, (p->G + 127) / 128));
}

int64_t part_slices(int64_t blocks, int64_t len) {
  const int64_t budget = ((int64_t)4 << 30) / 8;
  return std::max<int64_t>(1, std::min<int64_t>(blocks, budget / std::max<int64_t>(len, 1)));
}

int64_t trace_slices(fga_plan_s* p) {
  return part_slices(ray_launch_blocks(p), p->nshots * p->rx.nrec * p->rx.nrx);
}

cudaError_t launch_slice_sum(fga_plan_s* p, const double* part, int64_t slices, int64_t len,
                             double* out, const int32_t* perm, int64_t row) {
  const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((len + 255) / 256, 8192));
  k_slice_sum<<<blocks, 256, 0, p->stream>>>(part, slices, len, out, perm, row);
  p->launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_gather_rows(fga_plan_s* p, const double* in, const int32_t* perm, int64_t rows,
                               int64_t row, double* out) {
  const int64_t len = rows * row;
  const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((len + 255) / 256, 8192));
  k_gather_rows<<<blocks, 256, 0, p->stream>>>(in, perm, len, row, out);
  p->launches += 1;
  return cudaGetLastError();
}

// The caller has sized p->d_part for the trace slices when record is set and there
// are receivers.
cudaError_t launch_rays_steps(fga_plan_s* p, int64_t nsteps, bool record) {
  // d_steps[0]: steps integrated; d_steps[1]: the work counter of the persistent kernel
  cudaError_t e = cudaMemsetAsync(p->d_steps, 0, 2 * sizeof(unsigned long long), p->stream);
  if (e != cudaSuccess) return e;
  if (p->G == 0 && !p->dev_counts) {
    if (record && p->nrx > 0)
      return cudaMemsetAsync(p->d_traces, 0, sizeof(double) * p->nshots * p->rx.nrec * p->rx.nrx,
                             p->stream);
    return cudaSuccess;
  }
  e = ensure_ray_blocks(p);
  if (e != cudaSuccess) return e;
  const unsigned blocks = (unsigned)(p->dev_counts ? p->ray_blocks : ray_launch_blocks(p));
  RxDev rx = p->rx;
  int64_t len = 0, slices = 1;
  if (record && p->nrx > 0) {
    len = p->nshots * rx.nrec * rx.nrx;
    slices = trace_slices(p);
    if (p->part_cap < (size_t)(slices * len)) return cudaErrorInvalidValue;
    e = cudaMemsetAsync(p->d_part, 0, sizeof(double) * slices * len, p->stream);
    if (e != cudaSuccess) return e;
  } else {
    rx.every = 0;
  }
  const unsigned long long mult = work_order_mult(p->G);
  // longest estimated ray first (full integrations of rays that stop at the exit box)
  const int32_t* order = nullptr;
  if (!p->integrate_exited && nsteps == p->nsteps && p->d_ray_bucket) {
    const int64_t width = ray_order_width(p->nsteps), nb = p->nsteps / width + 1;
    e = cudaMemsetAsync(p->d_ray_bucket, 0, sizeof(int64_t) * (nb + 1), p->stream);
    if (e != cudaSuccess) return e;
    const int64_t Gl = p->dev_counts ? (int64_t)p->g_cap : p->G;
    const unsigned gb = (unsigned)std::max<int64_t>(1, std::min<int64_t>((Gl + 255) / 256, 4096));
    const int64_t* gm = p->dev_counts ? p->d_gm : nullptr;
    unsigned long long* cnt = reinterpret_cast<unsigned long long*>(p->d_ray_bucket);
    if (p->grid.dim == 1)
      k_ray_estimate<1><<<gb, 256, 0, p->stream>>>(p->grid, p->d_shots, p->d_coef, p->G, gm, p->d_gshot,
                                                  p->d_gq, p->d_gp, nsteps, p->dt, p->kappa, p->d_gsteps,
                                                  width, cnt);
    else if (p->grid.dim == 2)
      k_ray_estimate<2><<<gb, 256, 0, p->stream>>>(p->grid, p->d_shots, p->d_coef, p->G, gm, p->d_gshot,
                                                  p->d_gq, p->d_gp, nsteps, p->dt, p->kappa, p->d_gsteps,
                                                  width, cnt);
    else
      k_ray_estimate<3><<<gb, 256, 0, p->stream>>>(p->grid, p->d_shots, p->d_coef, p->G, gm, p->d_gshot,
                                                  p->d_gq, p->d_gp, nsteps, p->dt, p->kappa, p->d_gsteps,
                                                  width, cnt);
    e = launch_scan(p, p->d_ray_bucket, nb);
    if (e != cudaSuccess) return e;
    k_ray_order<<<gb, 256, 0, p->stream>>>(p->G, gm, mult, rx.every > 0 ? 1 : 0, p->d_gsteps, nsteps,
                                           width, cnt, p->d_adj_order);
    p->launches += 2;
    order = p->d_adj_order;
  }
  auto kern = ray_kernel(p);
  kern<<<blocks, 128, 0, p->stream>>>(p->grid, p->d_shots, p->d_coef, p->G, p->d_gshot, p->d_gq,
                                      p->d_gp, p->d_gpsi, nsteps, p->dt, p->kappa,
                                      p->integrate_exited, p->d_state, (int64_t)p->g_cap,
                                      p->d_gcoef, p->d_status, p->d_steps, p->d_steps + 1, rx,
                                      p->d_part, len, (int)slices, mult, p->d_gsteps,
                                      p->dev_counts ? p->d_gm : nullptr, order);
  p->launches += 1;
  e = cudaGetLastError();
  if (e != cudaSuccess || len == 0) return e;
  return launch_slice_sum(p, p->d_part, slices, len, p->d_traces, p->d_rx_perm, rx.nrx);
}

cudaError_t launch_rays(fga_plan_s* p) { return launch_rays_steps(p, p->nsteps, true); }

}  // namespace fga
