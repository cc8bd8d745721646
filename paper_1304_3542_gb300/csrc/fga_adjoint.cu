// Adjoint of the traces with respect to the velocity samples (the spline
// coefficients): given the cotangent of the traces (for the misfit
// J = 1/2 sum (trace - data)^2 it is the residual), accumulate
//   grad_c = (d traces / d c)^T residual
// with the set of Gaussians held fixed. c enters the traces through the rays (c, grad c
// and the Hessian of c at Q in the right-hand side of Eqs. characline, dzQ, dzP,
// a_formu) and through the branch split psi+ = 1/2 (psi_0 + i eps psi_1/(c(q)|p|))
// (Eq. psi).
//
// Discrete adjoint of the RK4 scheme (the exact gradient of the computed traces):
// every ray is integrated forward again storing a checkpoint every K ~ sqrt(T/dt)
// steps; the reverse sweep recomputes one segment of K states (and the RK4 stage states
// of its steps) at a time from its checkpoint and runs the transposed RK4 stages, each through the hand-written
// vector-Jacobian product of the right-hand side below (rhs_vjp). The coefficient
// gradient of each evaluation of c, grad c, Hessian of c is scattered to its 4^d
// spline taps with atomic additions. Like the forward integrator the kernel is
// persistent (lanes take the next Gaussian from a counter); each resident thread owns
// a slice of a scratch buffer for its checkpoints and segment states.
#include <algorithm>

#include "fga_internal.cuh"
#include "fga_medium.cuh"
#include "fga_ray_rhs.cuh"
#include "fga_ray_vjp.cuh"

namespace fga {

namespace {

using adj::cx;
using adj::MedAD;
using adj::conj;
using adj::medium_ad;
using adj::medium_ad_transpose;
using adj::mk;
using adj::mulc;
using adj::rdot;
using adj::rhs_vjp;
using adj::rk4_step;
using adj::rk4_step_adjoint;
using adj::rk4_step_record;
using adj::operator+;
using adj::operator-;
using adj::operator*;

// Adjoint of the record at state y: lam += d(sum_r res_r trace contribution)/dy and
// psib += the same derivative with respect to (Re psi, Im psi).
template <int D>
__device__ __forceinline__ void record_vjp(const GridDev& gd, const ShotDev& sh, const RxDev& rx,
                                           double kappa, const double* y, double2 psi,
                                           const double* __restrict__ res_row, double* lam,
                                           double* psib) {
  using Lo = Layout<D>;
  const double cut = kappa * sh.sqrt_eps;
  const double c0 = 2.0 * sh.W * sh.norm;
  double sn, cs;
  sincos(y[Lo::S] * sh.inv_eps, &sn, &cs);
  const cx eS = mk(cs, sn);
  const cx a = mk(y[Lo::aR], y[Lo::aI]);
  const cx ps = mk(psi.x, psi.y);
  const cx pref = c0 * (a * ps * eS);
  cx prefb = mk(0, 0);
  double Qb[D], Pb[D];
#pragma unroll
  for (int k = 0; k < D; ++k) Qb[k] = Pb[k] = 0.0;
  for_receivers_X<D>(gd, rx, y + Lo::Q, y + Lo::P, cut, sh.inv_eps,
                     [&](int64_t r, const double* d, double2 Xv) {
    const double w = res_row[r];
    const cx X = mk(Xv.x, Xv.y);
    // value = Re(pref X); adjoint of the complex product with a real cotangent w
    prefb = prefb + w * conj(X);
    const cx Xb = w * conj(pref);
    const cx zeta_b = mulc(Xb, X);  // X = exp(zeta), zeta = -|d|^2/(2 eps) + i P.d/eps
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const double db = zeta_b.r * (-d[k] * sh.inv_eps) + zeta_b.i * y[Lo::P + k] * sh.inv_eps;
      Pb[k] += zeta_b.i * d[k] * sh.inv_eps;
      Qb[k] -= db;  // d = x_r - Q
    }
  });
  // pref = c0 a psi e^{iS/eps}
  const cx ab = mulc(prefb, c0 * (ps * eS));
  const cx psb = mulc(prefb, c0 * (a * eS));
  const double Sb = rdot(prefb, mk(-pref.i * sh.inv_eps, pref.r * sh.inv_eps));
#pragma unroll
  for (int k = 0; k < D; ++k) {
    lam[Lo::Q + k] += Qb[k];
    lam[Lo::P + k] += Pb[k];
  }
  lam[Lo::aR] += ab.r;
  lam[Lo::aI] += ab.i;
  lam[Lo::S] += Sb;
  psib[0] += psb.r;
  psib[1] += psb.i;
}

// Gaussians in order of decreasing stop step (counting sort by stop-step bucket), so
// that the 32 rays of a warp, which the adjoint runs in lockstep, have nearly the same
// length.
__global__ void k_order_count(const int32_t* __restrict__ gsteps, int64_t G, int64_t nsteps,
                              int64_t width, int64_t* __restrict__ cnt) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < G;
       g += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(reinterpret_cast<unsigned long long*>(cnt + (nsteps - gsteps[g]) / width), 1ull);
}

__global__ void k_order_scatter(const int32_t* __restrict__ gsteps, int64_t G, int64_t nsteps,
                                int64_t width, int64_t* __restrict__ fill, int32_t* __restrict__ order) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < G;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pos = (int64_t)atomicAdd(
        reinterpret_cast<unsigned long long*>(fill + (nsteps - gsteps[g]) / width), 1ull);
    order[pos] = (int32_t)g;
  }
}

// One warp runs 32 Gaussians in lockstep: the forward pass with checkpoints until the
// last of them stops, then the reverse sweep from the warp's longest ray down to step 0,
// each lane working only on steps its own ray reached (the others wait); so the segment
// recomputations of all lanes fall on the same trips.
template <int D>
__global__ void __launch_bounds__(128) k_adjoint(GridDev gd, const ShotDev* __restrict__ shots,
                                                 const double* __restrict__ C, int64_t G,
                                                 const int32_t* __restrict__ gshot,
                                                 const int64_t* __restrict__ gq,
                                                 const int32_t* __restrict__ gp,
                                                 const double2* __restrict__ gpsi,
                                                 const double2* __restrict__ gpsi_f1, int64_t nsteps,
                                                 double dt, double kappa, int integrate_exited,
                                                 RxDev rx, const double* __restrict__ residual,
                                                 double* __restrict__ grad_part, int64_t grad_len,
                                                 int slices, double* __restrict__ scratch,
                                                 int64_t kseg, int64_t ncheck,
                                                 unsigned long long* next,
                                                 const int32_t* __restrict__ order) {
  using Lo = Layout<D>;
  constexpr int NF = Lo::NF;
  constexpr unsigned kFull = 0xffffffffu;
  // this block's private slice of dJ/dc (no other block adds into it)
  double* gradC = grad_part + (int64_t)(blockIdx.x % slices) * grad_len;
  const int64_t nthr = (int64_t)gridDim.x * blockDim.x;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  // scratch: [slot][field][thread], slots 0..ncheck-1 checkpoints, then kseg segment states,
  // then 3 kseg stage states
  auto slot = [&](int64_t sidx, int f) -> double& { return scratch[(sidx * NF + f) * nthr + tid]; };
  extern __shared__ double zs[];  // [4][NF][blockDim.x]: RK4 stage states and lambda in
  while (true) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(next, 32ull);
    base = __shfl_sync(kFull, base, 0);
    const unsigned long long w = base + (unsigned long long)lane;
    const bool has = w < (unsigned long long)G;
    if (!__any_sync(kFull, has)) break;
    const int64_t g = has ? (int64_t)order[w] : 0;
    const int s = has ? gshot[g] : 0;
    const ShotDev& sh = shots[s];
    double lo[D], hi[D];
#pragma unroll
    for (int i = 0; i < D; ++i) {
      double reach = kappa * sh.sqrt_eps + 2.0 * gd.h[i];
      lo[i] = gd.o[i] - reach;
      hi[i] = gd.o[i] + (double)(gd.n[i] - 1) * gd.h[i] + reach;
    }
    double y[NF];
    ray_init<D>(gd, sh, has ? gq[g] : 0, has ? gp[g] : 0, y);
    // forward with checkpoints every kseg steps; nend = the step the ray stopped at. With
    // a single segment (kseg > nsteps) this pass records every state and the stage states
    // of every step directly, and the reverse sweep recomputes nothing.
    const bool single = kseg > nsteps;
    int64_t nend = 0;
    bool run = has;
    for (int64_t step = 0; __any_sync(kFull, run); ++step) {
      if (!run) continue;
      if (single) {
#pragma unroll
        for (int f = 0; f < NF; ++f) slot(ncheck + step, f) = y[f];
      } else if (step % kseg == 0) {
#pragma unroll
        for (int f = 0; f < NF; ++f) slot(step / kseg, f) = y[f];
      }
      bool done = step >= nsteps;
      if (!done && !integrate_exited) {
#pragma unroll
        for (int i = 0; i < D; ++i)
          done = done || (!gd.periodic[i] && ((y[Lo::Q + i] < lo[i] && y[Lo::P + i] <= 0.0) ||
                                              (y[Lo::Q + i] > hi[i] && y[Lo::P + i] >= 0.0)));
      }
      if (done) {
        nend = step;
        run = false;
      } else if (single) {
        rk4_step_record<D>(gd, y, dt, [&](int st, const double* zz) {
#pragma unroll
          for (int f = 0; f < NF; ++f) slot(ncheck + kseg + 3 * step + st, f) = zz[f];
        });
      } else {
        rk4_step<D>(gd, C, y, dt);
      }
    }
    int64_t nend_w = nend;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const int64_t o = __shfl_xor_sync(kFull, nend_w, off);
      nend_w = o > nend_w ? o : nend_w;
    }
    // reverse sweep
    double lam[NF], psib[2] = {0.0, 0.0};
#pragma unroll
    for (int f = 0; f < NF; ++f) lam[f] = 0.0;
    const double2 psi = has ? gpsi[g] : make_double2(0.0, 0.0);
    // states j*kseg .. of segment j into the segment slots (lanes whose ray reached them)
    // stage states of the step from segment state i: slots ncheck + kseg + 3 i + (0, 1, 2)
    auto load_segment = [&](int64_t j) {
      const bool mine = has && j * kseg <= nend;
      double z[NF];
#pragma unroll
      for (int f = 0; f < NF; ++f) z[f] = mine ? slot(j, f) : 0.0;
      for (int64_t i = 0; i < kseg && j * kseg + i <= nend_w; ++i) {
        if (!mine || j * kseg + i > nend) continue;
#pragma unroll
        for (int f = 0; f < NF; ++f) slot(ncheck + i, f) = z[f];
        if (j * kseg + i + 1 <= nend)
          rk4_step_record<D>(gd, z, dt, [&](int s, const double* zz) {
#pragma unroll
            for (int f = 0; f < NF; ++f) slot(ncheck + kseg + 3 * i + s, f) = zz[f];
          });
      }
    };
    int64_t seg_loaded = single ? 0 : -1;
    for (int64_t nn = nend_w;; --nn) {
      const bool act = has && nn <= nend;
      const int64_t j = nn / kseg;
      if (j != seg_loaded) {
        load_segment(j);
        seg_loaded = j;
      }
      double yn[NF];
      if (act && rx.every > 0 && nn % rx.every == 0) {
#pragma unroll
        for (int f = 0; f < NF; ++f) yn[f] = slot(ncheck + (nn - j * kseg), f);
        record_vjp<D>(gd, sh, rx, kappa, yn, psi,
                      residual + ((int64_t)s * rx.nrec + nn / rx.every) * rx.nrx, lam, psib);
      }
      if (nn == 0) break;
      // state at nn - 1
      const int64_t jp = (nn - 1) / kseg;
      if (jp != seg_loaded) {
        load_segment(jp);
        seg_loaded = jp;
      }
      if (act) {
#pragma unroll
        for (int f = 0; f < NF; ++f) yn[f] = slot(ncheck + (nn - 1 - jp * kseg), f);
        const int64_t i = nn - 1 - jp * kseg;
        rk4_step_adjoint<D>(gd, C, yn, dt, lam, gradC, zs, blockDim.x, threadIdx.x,
                            [&](int s, int f) { return slot(ncheck + kseg + 3 * i + s, f); });
      }
    }
    if (!has) continue;
    // branch split: psi+ = 1/2 psi_0 + t, t = 1/2 i eps psi_1/(c(q)|p|), so d psi+/d c(q) = -t/c(q)
    const double2 t1 = gpsi_f1[g];
    double q[D];
    {
      int64_t qf = gq[g];
      int64_t qm[D];
      if constexpr (D == 1) {
        qm[0] = qf;
      } else if constexpr (D == 3) {
        const int64_t nq12 = sh.nq[1] * sh.nq[2];
        qm[0] = qf / nq12;
        qm[1] = (qf - qm[0] * nq12) / sh.nq[2];
        qm[2] = qf - qm[0] * nq12 - qm[1] * sh.nq[2];
      } else {
        qm[0] = qf / sh.nq[1];
        qm[1] = qf - qm[0] * sh.nq[1];
      }
#pragma unroll
      for (int i = 0; i < D; ++i) q[i] = gd.o[i] + (double)(sh.s[i] * qm[i]) * gd.h[i];
    }
    MedAD<D> mq;
    medium_ad<D>(gd, C, q, mq);
    const double cqb = -(psib[0] * t1.x + psib[1] * t1.y) / mq.c;
    double zero_g[D], Qdummy[D];
    double zero_K[D][D];
#pragma unroll
    for (int i = 0; i < D; ++i) {
      zero_g[i] = 0.0;
      Qdummy[i] = 0.0;
#pragma unroll
      for (int k = 0; k < D; ++k) zero_K[i][k] = 0.0;
    }
    medium_ad_transpose<D>(gd, mq, cqb, zero_g, zero_K, Qdummy, gradC);
  }
}

}  // namespace

// Dynamic shared memory of the adjoint kernel: 4 * NF doubles per thread of 128.
size_t adjoint_smem(int dim) { return (size_t)4 * state_fields(dim) * 128 * sizeof(double); }

cudaError_t set_adjoint_smem(int dim) {
  if (dim == 1)
    return cudaFuncSetAttribute(k_adjoint<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)adjoint_smem(1));
  if (dim == 2)
    return cudaFuncSetAttribute(k_adjoint<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)adjoint_smem(2));
  return cudaFuncSetAttribute(k_adjoint<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)adjoint_smem(3));
}

// Resident threads of the adjoint kernel and the scratch doubles they need.
int64_t adjoint_threads(fga_plan_s* p) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (set_adjoint_smem(p->grid.dim) != cudaSuccess) return 0;
  const int d = p->grid.dim;
  cudaError_t e = d == 1 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_adjoint<1>, 128,
                                                                         adjoint_smem(1))
                  : d == 2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_adjoint<2>, 128,
                                                                           adjoint_smem(2))
                           : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_adjoint<3>, 128,
                                                                           adjoint_smem(3));
  if (e != cudaSuccess) return 0;
  int64_t blocks = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
  blocks = std::min<int64_t>(blocks, (p->G + 127) / 128);
  return std::max<int64_t>(blocks, 1) * 128;
}

// dJ/dc into gradC (device, npts): the kernel adds into block-private slices of
// p->d_part (sized by the caller for adjoint_slices(p, nthreads)), then the slices are
// summed in order into gradC.
int64_t adjoint_slices(fga_plan_s* p, int64_t nthreads) {
  return part_slices(std::max<int64_t>(nthreads / 128, 1), p->grid.npts);
}

// Width (in steps) of the stop-step buckets the Gaussians are sorted by.
int64_t adjoint_sort_width(int64_t nsteps) {
  return std::max<int64_t>(1, std::min<int64_t>(16, nsteps / 64));
}

cudaError_t launch_adjoint(fga_plan_s* p, const double* residual, double* gradC, double* scratch,
                           int64_t nthreads, int64_t kseg, int64_t ncheck) {
  cudaError_t e = cudaMemsetAsync(p->d_steps + 1, 0, sizeof(unsigned long long), p->stream);
  if (e != cudaSuccess) return e;
  const int64_t len = p->grid.npts;
  if (p->G == 0) return cudaMemsetAsync(gradC, 0, sizeof(double) * len, p->stream);
  const unsigned blocks = (unsigned)(nthreads / 128);
  const int64_t slices = adjoint_slices(p, nthreads);
  if (p->part_cap < (size_t)(slices * len)) return cudaErrorInvalidValue;
  // Gaussians by decreasing stop step
  const int64_t width = adjoint_sort_width(p->nsteps), nb = p->nsteps / width + 1;
  if (p->adj_bucket_cap < (size_t)(nb + 1)) return cudaErrorInvalidValue;
  e = cudaMemsetAsync(p->d_adj_bucket, 0, sizeof(int64_t) * (nb + 1), p->stream);
  if (e != cudaSuccess) return e;
  const unsigned gb = (unsigned)std::max<int64_t>(1, std::min<int64_t>((p->G + 255) / 256, 4096));
  k_order_count<<<gb, 256, 0, p->stream>>>(p->d_gsteps, p->G, p->nsteps, width, p->d_adj_bucket);
  e = launch_scan(p, p->d_adj_bucket, nb);
  if (e != cudaSuccess) return e;
  k_order_scatter<<<gb, 256, 0, p->stream>>>(p->d_gsteps, p->G, p->nsteps, width, p->d_adj_bucket,
                                             p->d_adj_order);
  p->launches += 2;
  e = cudaMemsetAsync(p->d_part, 0, sizeof(double) * slices * len, p->stream);
  if (e != cudaSuccess) return e;
  RxDev rx = p->rx;
  if (p->grid.dim == 1)
    k_adjoint<1><<<blocks, 128, adjoint_smem(1), p->stream>>>(p->grid, p->d_shots, p->d_coef, p->G, p->d_gshot,
                                                p->d_gq, p->d_gp, p->d_gpsi, p->d_gpsi_f1, p->nsteps,
                                                p->dt, p->kappa, p->integrate_exited, rx, residual,
                                                p->d_part, len, (int)slices, scratch, kseg, ncheck,
                                                p->d_steps + 1, p->d_adj_order);
  else if (p->grid.dim == 3)
    k_adjoint<3><<<blocks, 128, adjoint_smem(3), p->stream>>>(p->grid, p->d_shots, p->d_coef, p->G, p->d_gshot,
                                                p->d_gq, p->d_gp, p->d_gpsi, p->d_gpsi_f1, p->nsteps,
                                                p->dt, p->kappa, p->integrate_exited, rx, residual,
                                                p->d_part, len, (int)slices, scratch, kseg, ncheck,
                                                p->d_steps + 1, p->d_adj_order);
  else
    k_adjoint<2><<<blocks, 128, adjoint_smem(2), p->stream>>>(p->grid, p->d_shots, p->d_coef, p->G, p->d_gshot,
                                                p->d_gq, p->d_gp, p->d_gpsi, p->d_gpsi_f1, p->nsteps,
                                                p->dt, p->kappa, p->integrate_exited, rx, residual,
                                                p->d_part, len, (int)slices, scratch, kseg, ncheck,
                                                p->d_steps + 1, p->d_adj_order);
  p->launches += 1;
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_slice_sum(p, p->d_part, slices, len, gradC);
}

}  // namespace fga
