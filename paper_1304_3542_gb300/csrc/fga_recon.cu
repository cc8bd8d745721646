// Step 3 of the method: the Gaussian sum of Eq. recons on the output grid.
//
// Every term is cut to the window |x_k - Q_k| <= kappa sqrt(eps) on each axis and
// is a product over axes,
//   term(x) = coef * prod_k X_k(x_k),  X_k(xi) = sum_images exp(i P_k (xi - Q_k)/eps
//                                                          - (xi - Q_k)^2/(2 eps)),
// so the sum over the Gaussians that touch an output tile is a complex
// contraction U = X^T diag(coef) Z over the Gaussian index (a GEMM of rank one
// terms). Binning (K4) builds, per (shot, tile), the ordered list of Gaussians
// whose window meets the tile; the gather (K5) runs one CTA per (tile, segment of
// its list), generates the per-axis factors of a chunk of Gaussians into shared
// memory and accumulates a partial tile in registers, FP64 throughout; the
// partial tiles are then summed in a fixed order. The scatter-free form needs no
// atomics on the output and gives a deterministic summation order.
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "fga_internal.cuh"
#include "fga_tiles.cuh"

namespace fga {

namespace {

constexpr int NT = 256;
constexpr int T2 = 64;   // 2D tile edge (points)
constexpr int T3 = 16;   // 3D tile edge (points)
constexpr int CH3 = 16;  // Gaussians per chunk (3D)
constexpr int64_t SEG3 = 512;  // default Gaussians per work item (3D)
constexpr int T1 = 256;  // 1D tile length
constexpr int CH = 16;   // Gaussians per chunk (2D)
constexpr int CH1 = 32;  // Gaussians per chunk (1D)
constexpr int64_t SEG2 = 1024;  // default Gaussians per work item (2D)
constexpr int64_t SEG1 = 512;   // default Gaussians per work item (1D)
constexpr int64_t kPartialBudget = (int64_t)4 << 30;  // bytes of partial tiles at most
constexpr int64_t kBinChunk = 8192;  // Gaussians per binning split (at least)

// Pass 1 (FILL = false): number of Gaussians of each (tile, split), a split being a run
// of `chunk` consecutive Gaussians of the tile's shot. Pass 2 (FILL = true): the ordered
// list, each (tile, split) written at its own offset. One CTA per (tile, split),
// blockIdx.x = tile * nsplit + split, scans its run in order (block-wide ordered
// compaction per chunk of NT); with the splits' offsets in tile-major order every tile's
// list is ordered by Gaussian index, whatever nsplit is.
template <int D, bool FILL>
__global__ void __launch_bounds__(NT) k_bin(GridDev gd, const ShotDev* __restrict__ shots, int nshots,
                                            double kappa, const double* __restrict__ state,
                                            int64_t ld, int64_t* __restrict__ cnt,
                                            const int64_t* __restrict__ off,
                                            int32_t* __restrict__ list, int64_t list_cap,
                                            int nsplit, int64_t chunk, int* __restrict__ status) {
  const int64_t t = blockIdx.x / nsplit;
  const int64_t split = blockIdx.x - t * nsplit;
  const int s = shot_of_tile(shots, nshots, t);
  const ShotDev& sh = shots[s];
  int64_t a[D], b[D];
  tile_box<D>(gd, sh, t - sh.tile_off, a, b);
  const double cut = kappa * sh.sqrt_eps;
  __shared__ int warp_tot[NT / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t gend = sh.g_off + sh.g_cnt;
  const int64_t gb = sh.g_off + split * chunk;
  const int64_t ge = gb < gend && gend - gb > chunk ? gb + chunk : gend;
  int64_t base = FILL ? off[blockIdx.x] : 0;
  int64_t total = 0;
  for (int64_t g0 = gb; g0 < ge; g0 += NT) {
    int64_t g = g0 + threadIdx.x;
    bool f = false;
    if (g < ge) {
      double Q[D];
#pragma unroll
      for (int k = 0; k < D; ++k) Q[k] = state[k * ld + g];
      f = overlaps<D>(gd, Q, cut, a, b);
    }
    unsigned bal = __ballot_sync(0xffffffffu, f);
    if (lane == 0) warp_tot[warp] = __popc(bal);
    __syncthreads();
    int before = 0, all = 0;
    for (int w = 0; w < NT / 32; ++w) {
      if (w < warp) before += warp_tot[w];
      all += warp_tot[w];
    }
    if (FILL && f) {
      int64_t at = base + total + before + __popc(bal & ((1u << lane) - 1u));
      if (at < list_cap)
        list[at] = (int32_t)g;
      else
        atomicOr(status, kStatusCapacity);
    }
    total += all;
    __syncthreads();
  }
  if (!FILL && threadIdx.x == 0) cnt[blockIdx.x] = total;
}

// The conservative grid-index window [lo, hi] of every Gaussian along every axis (as
// window_range, once per Gaussian instead of once per (Gaussian, tile) in each binning
// pass): rng[(2 k) ld + g] = lo, rng[(2 k + 1) ld + g] = hi, clamped to +-2^30. G from the
// device when gm is given (pipeline graph).
template <int D>
__global__ void k_bin_ranges(GridDev gd, const ShotDev* __restrict__ shots,
                             const int32_t* __restrict__ gshot, double kappa,
                             const double* __restrict__ state, int64_t ld, int64_t G,
                             const int64_t* __restrict__ gm, int32_t* __restrict__ rng) {
  if (gm) G = gm[0];
  const double lim = 1073741824.0;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < G;
       g += (int64_t)gridDim.x * blockDim.x) {
    const double cut = kappa * shots[gshot[g]].sqrt_eps;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const double Q = state[k * ld + g];
      const double lo = floor((Q - cut - gd.o[k]) * gd.inv_h[k]) - 1.0;
      const double hi = ceil((Q + cut - gd.o[k]) * gd.inv_h[k]) + 1.0;
      rng[(2 * k) * ld + g] = (int32_t)fmin(fmax(lo, -lim), lim);
      rng[(2 * k + 1) * ld + g] = (int32_t)fmin(fmax(hi, -lim), lim);
    }
  }
}

// k_bin with the windows of k_bin_ranges: integer tests only (on a periodic axis the
// images l = -2 .. 2 shift the range by l n).
template <int D, bool FILL>
__global__ void __launch_bounds__(NT) k_bin_r(GridDev gd, const ShotDev* __restrict__ shots, int nshots,
                                              const int32_t* __restrict__ rng, int64_t ld,
                                              int64_t* __restrict__ cnt, const int64_t* __restrict__ off,
                                              int32_t* __restrict__ list, int64_t list_cap, int nsplit,
                                              int64_t chunk, int* __restrict__ status) {
  const int64_t t = blockIdx.x / nsplit;
  const int64_t split = blockIdx.x - t * nsplit;
  const int s = shot_of_tile(shots, nshots, t);
  const ShotDev& sh = shots[s];
  int64_t a[D], b[D];
  tile_box<D>(gd, sh, t - sh.tile_off, a, b);
  __shared__ int warp_tot[NT / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t gend = sh.g_off + sh.g_cnt;
  const int64_t gb = sh.g_off + split * chunk;
  const int64_t ge = gb < gend && gend - gb > chunk ? gb + chunk : gend;
  int64_t base = FILL ? off[blockIdx.x] : 0;
  int64_t total = 0;
  for (int64_t g0 = gb; g0 < ge; g0 += NT) {
    int64_t g = g0 + threadIdx.x;
    bool f = false;
    if (g < ge) {
      f = true;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const int64_t lo = rng[(2 * k) * ld + g], hi = rng[(2 * k + 1) * ld + g];
        bool any = lo <= b[k] && hi >= a[k];
        if (gd.periodic[k])
          for (int l = -2; l <= 2; ++l) any = any || (lo + l * gd.n[k] <= b[k] && hi + l * gd.n[k] >= a[k]);
        f = f && any;
      }
    }
    unsigned bal = __ballot_sync(0xffffffffu, f);
    if (lane == 0) warp_tot[warp] = __popc(bal);
    __syncthreads();
    int before = 0, all = 0;
    for (int w = 0; w < NT / 32; ++w) {
      if (w < warp) before += warp_tot[w];
      all += warp_tot[w];
    }
    if (FILL && f) {
      int64_t at = base + total + before + __popc(bal & ((1u << lane) - 1u));
      if (at < list_cap)
        list[at] = (int32_t)g;
      else
        atomicOr(status, kStatusCapacity);
    }
    total += all;
    __syncthreads();
  }
  if (!FILL && threadIdx.x == 0) cnt[blockIdx.x] = total;
}

// Offsets of the tiles' lists from the scanned (tile, split) offsets (entry ntiles: the
// total).
__global__ void k_tile_offsets(const int64_t* __restrict__ split_off, int nsplit, int64_t ntiles,
                               int64_t* __restrict__ tile_off) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t <= ntiles) tile_off[t] = split_off[t * nsplit];
}

// Per-axis factor of one Gaussian at grid index i (all images inside the window).
__device__ __forceinline__ double2 axis_factor(const Axis& ax, int64_t i, double Q, double P,
                                               double cut, double inv_eps) {
  double x = ax.o + (double)i * ax.h;
  double re = 0.0, im = 0.0;
  int lmax = ax.periodic ? 2 : 0;
  for (int l = -lmax; l <= lmax; ++l) {
    double d = x - Q + l * ax.L;
    if (fabs(d) <= cut) {
      double gs = exp(-0.5 * d * d * inv_eps);
      double sn, cs;
      sincos(P * d * inv_eps, &sn, &cs);
      re = fma(gs, cs, re);
      im = fma(gs, sn, im);
    }
  }
  return make_double2(re, im);
}

// Factors of one Gaussian along an open axis at the N grid points i0 .. i0+N-1,
// times cf: E_i = exp(-d_i^2/(2 eps)) exp(i P d_i/eps), d_i = x_i - Q, zero outside
// |d_i| <= cut. Evaluated directly at the first point inside the window and then by
// the exact recurrence E_{i+1} = E_i R_i rot, R_{i+1} = R_i rho with
// R_i = exp(-(d_i h + h^2/2)/eps), rot = exp(i P h/eps), rho = exp(-h^2/eps)
// (relative rounding growth below 1e-14 over 8 points, 2e-14 over 16).
template <int N>
__device__ __forceinline__ void axis_factors(double xi0, double h, double Q, double P, double cut,
                                             double inv_eps, double2 cf, double2* dst) {
  int r0 = 0;
  while (r0 < N && fabs(fma((double)r0, h, xi0) - Q) > cut) ++r0;
  for (int r = 0; r < r0; ++r) dst[r] = make_double2(0.0, 0.0);
  if (r0 == N) return;
  double d = fma((double)r0, h, xi0) - Q;
  double gs = exp(-0.5 * d * d * inv_eps);
  double sn, cs;
  sincos(P * d * inv_eps, &sn, &cs);
  double er = gs * cs, ei = gs * sn;
  double R = exp(-(d * h + 0.5 * h * h) * inv_eps);
  double rs, rc;
  sincos(P * h * inv_eps, &rs, &rc);
  const double rho = exp(-h * h * inv_eps);
  for (int r = r0; r < N; ++r) {
    double dr = fma((double)r, h, xi0) - Q;
    if (fabs(dr) <= cut)
      dst[r] = make_double2(cf.x * er - cf.y * ei, cf.x * ei + cf.y * er);
    else
      dst[r] = make_double2(0.0, 0.0);
    double tr = er * R, ti = ei * R;
    er = tr * rc - ti * rs;
    ei = tr * rs + ti * rc;
    R *= rho;
  }
}

// Number of list segments per tile (then scanned into seg_off).
__global__ void k_segments(const int64_t* __restrict__ off, int64_t ntiles, int64_t list_cap,
                           int64_t seg, int64_t* __restrict__ seg_cnt) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= ntiles) return;
  int64_t a = min(off[t], list_cap), b = min(off[t + 1], list_cap);
  seg_cnt[t] = (b - a + seg - 1) / seg;
}

// 1D gather of one work item: thread = grid point, partial[w][T1].
__global__ void __launch_bounds__(NT) k_gather1(GridDev gd, const ShotDev* __restrict__ shots,
                                                int nshots, double kappa,
                                                const double* __restrict__ state, int64_t ld,
                                                const double2* __restrict__ coef,
                                                const int64_t* __restrict__ off,
                                                const int32_t* __restrict__ list, int64_t list_cap,
                                                const int64_t* __restrict__ seg_off, int64_t ntiles,
                                                int64_t seg, double* __restrict__ partial) {
  const int64_t w = blockIdx.x;
  if (w >= seg_off[ntiles]) return;
  const int64_t t = tile_of_item(seg_off, ntiles, w);
  const int s = shot_of_tile(shots, nshots, t);
  const ShotDev& sh = shots[s];
  const double cut = kappa * sh.sqrt_eps, inv_eps = sh.inv_eps;
  const int64_t i = (t - sh.tile_off) * T1 + threadIdx.x;
  __shared__ double sQ[CH1], sP[CH1];
  __shared__ double2 sC[CH1];
  double re = 0.0;
  const int64_t l0 = min(off[t], list_cap) + (w - seg_off[t]) * seg;
  const int64_t l1 = min(min(off[t + 1], list_cap), l0 + seg);
  for (int64_t c0 = l0; c0 < l1; c0 += CH1) {
    int nc = (int)((l1 - c0) < CH1 ? (l1 - c0) : CH1);
    if (threadIdx.x < nc) {
      int32_t g = list[c0 + threadIdx.x];
      sQ[threadIdx.x] = state[0 * ld + g];
      sP[threadIdx.x] = state[1 * ld + g];
      sC[threadIdx.x] = coef[g];
    }
    __syncthreads();
    for (int j = 0; j < nc; ++j) {
      double2 x = axis_factor(grid_axis(gd, 0), i, sQ[j], sP[j], cut, inv_eps);
      re = fma(sC[j].x, x.x, fma(-sC[j].y, x.y, re));
    }
    __syncthreads();
  }
  partial[w * T1 + threadIdx.x] = re;
}

// 2D gather of one work item: 64 x 64 tile, 8 warps each covering a 16 x 32 patch
// (4 x 8 threads of 4 x 4 points); a warp skips a Gaussian whose window misses its
// patch. Writes the partial tile sum partial[w][64][64].
__global__ void __launch_bounds__(NT) k_gather2(GridDev gd, const ShotDev* __restrict__ shots,
                                                int nshots, double kappa,
                                                const double* __restrict__ state, int64_t ld,
                                                const double2* __restrict__ coef,
                                                const int64_t* __restrict__ off,
                                                const int32_t* __restrict__ list, int64_t list_cap,
                                                const int64_t* __restrict__ seg_off, int64_t ntiles,
                                                int64_t seg, double* __restrict__ partial) {
  const int64_t w = blockIdx.x;
  if (w >= seg_off[ntiles]) return;
  const int64_t t = tile_of_item(seg_off, ntiles, w);
  const int s = shot_of_tile(shots, nshots, t);
  const ShotDev& sh = shots[s];
  const double cut = kappa * sh.sqrt_eps, inv_eps = sh.inv_eps;
  int64_t a[2], b[2];
  tile_box<2>(gd, sh, t - sh.tile_off, a, b);
  __shared__ double2 Xs[CH][T2];
  __shared__ double2 Zs[CH][T2];
  __shared__ int win[CH][4];  // tile-local [xlo, xhi, zlo, zhi]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int wx = warp >> 1, wz = warp & 1;
  const int lx = lane >> 3, lz = lane & 7;
  const int x0 = wx * 16 + lx * 4, z0 = wz * 32 + lz * 4;
  const int px0 = wx * 16, px1 = wx * 16 + 15, pz0 = wz * 32, pz1 = wz * 32 + 31;
  // only Re(sum) is needed: u = 2 Re(...) and the 2 is inside coef
  double accr[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) accr[i][j] = 0.0;
  const int64_t l0 = min(off[t], list_cap) + (w - seg_off[t]) * seg;
  const int64_t l1 = min(min(off[t + 1], list_cap), l0 + seg);
  for (int64_t c0 = l0; c0 < l1; c0 += CH) {
    const int nc = (int)((l1 - c0) < CH ? (l1 - c0) : CH);
    // factor generation: thread -> (gaussian, axis, 8 consecutive points)
    {
      const int gi = threadIdx.x >> 4, axis = (threadIdx.x >> 3) & 1, part = threadIdx.x & 7;
      if (gi < nc) {
        int32_t g = list[c0 + gi];
        double Q = state[axis * ld + g], P = state[(2 + axis) * ld + g];
        double2 cf = axis == 0 ? coef[g] : make_double2(1.0, 0.0);
        double2* dst = (axis == 0 ? Xs[gi] : Zs[gi]) + part * 8;
        const Axis ax = grid_axis(gd, axis);
        const int64_t a_ax = axis == 0 ? a[0] : a[1];
        if (ax.periodic) {
          for (int r = 0; r < 8; ++r) {
            double2 f = axis_factor(ax, a_ax + part * 8 + r, Q, P, cut, inv_eps);
            dst[r] = make_double2(cf.x * f.x - cf.y * f.y, cf.x * f.y + cf.y * f.x);
          }
        } else {
          double xi0 = ax.o + (double)(a_ax + part * 8) * ax.h;
          axis_factors<8>(xi0, ax.h, Q, P, cut, inv_eps, cf, dst);
        }
        if (part == 0) {
          if (ax.periodic) {
            win[gi][2 * axis] = 0;
            win[gi][2 * axis + 1] = T2 - 1;
          } else {
            int64_t lo, hi;
            window_range_ax(ax, Q, cut, lo, hi);
            win[gi][2 * axis] = (int)((lo - a_ax) > -1 ? (lo - a_ax) : -1);
            win[gi][2 * axis + 1] = (int)((hi - a_ax) < T2 ? (hi - a_ax) : T2);
          }
        }
      }
    }
    __syncthreads();
    for (int gi = 0; gi < nc; ++gi) {
      if (win[gi][0] > px1 || win[gi][1] < px0 || win[gi][2] > pz1 || win[gi][3] < pz0) continue;
      double2 xv[4], zv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        xv[i] = Xs[gi][x0 + i];
        zv[i] = Zs[gi][z0 + i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          accr[i][j] = fma(xv[i].x, zv[j].x, fma(-xv[i].y, zv[j].y, accr[i][j]));
        }
    }
    __syncthreads();
  }
  double* dst = partial + w * (int64_t)(T2 * T2);
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) dst[(x0 + i) * T2 + z0 + j] = accr[i][j];
}

// Ordered sum of the partial tiles of every tile into the output grid.
// 3D gather of one work item: a 16^3 tile, thread = (x, y) column of 16 points along z;
// per chunk of 16 Gaussians the per-axis factors (16 points each, the x factor carrying
// the coefficient) and each window's range in the tile are made in shared memory, then
// every thread adds Re(X_g(x) Y_g(y) Z_g(z)) to its points inside the window (by
// quarters of 4 along z). Writes partial[w][16][16][16].
__global__ void __launch_bounds__(NT) k_gather3(GridDev gd, const ShotDev* __restrict__ shots,
                                                int nshots, double kappa,
                                                const double* __restrict__ state, int64_t ld,
                                                const double2* __restrict__ coef,
                                                const int64_t* __restrict__ off,
                                                const int32_t* __restrict__ list, int64_t list_cap,
                                                const int64_t* __restrict__ seg_off, int64_t ntiles,
                                                int64_t seg, double* __restrict__ partial) {
  const int64_t w = blockIdx.x;
  if (w >= seg_off[ntiles]) return;
  const int64_t t = tile_of_item(seg_off, ntiles, w);
  const int s = shot_of_tile(shots, nshots, t);
  const ShotDev& sh = shots[s];
  const double cut = kappa * sh.sqrt_eps, inv_eps = sh.inv_eps;
  int64_t a[3], b[3];
  tile_box<3>(gd, sh, t - sh.tile_off, a, b);
  __shared__ double2 F[3][CH3][T3];  // [axis][gaussian][point]
  // per Gaussian and axis: a range of tile points outside which its factor is zero
  // (conservative, clipped to the tile; empty when lo > hi)
  __shared__ int W[CH3][3][2];
  const int ix = threadIdx.x / T3, iy = threadIdx.x % T3;
  double acc[T3];
#pragma unroll
  for (int i = 0; i < T3; ++i) acc[i] = 0.0;
  const int64_t l0 = min(off[t], list_cap) + (w - seg_off[t]) * seg;
  const int64_t l1 = min(min(off[t + 1], list_cap), l0 + seg);
  for (int64_t c0 = l0; c0 < l1; c0 += CH3) {
    const int nc = (int)((l1 - c0) < CH3 ? (l1 - c0) : CH3);
    if (threadIdx.x < 3 * CH3) {
      const int gi = threadIdx.x / 3, axis = threadIdx.x % 3;
      double2* dst = F[axis][gi];
      if (gi < nc) {
        const int32_t g = list[c0 + gi];
        const double Q = state[axis * ld + g], P = state[(3 + axis) * ld + g];
        const double2 cf = axis == 0 ? coef[g] : make_double2(1.0, 0.0);
        const Axis ax = grid_axis(gd, axis);
        const int64_t a_ax = axis == 0 ? a[0] : (axis == 1 ? a[1] : a[2]);
        int wl = 0, wh = T3 - 1;
        if (ax.periodic) {
          for (int r = 0; r < T3; ++r) {
            const double2 f = axis_factor(ax, a_ax + r, Q, P, cut, inv_eps);
            dst[r] = make_double2(cf.x * f.x - cf.y * f.y, cf.x * f.y + cf.y * f.x);
          }
        } else {
          axis_factors<T3>(ax.o + (double)a_ax * ax.h, ax.h, Q, P, cut, inv_eps, cf, dst);
          int64_t lo, hi;
          window_range_ax(ax, Q, cut, lo, hi);
          lo -= a_ax;
          hi -= a_ax;
          wl = (int)(lo < 0 ? 0 : (lo > T3 ? T3 : lo));
          wh = (int)(hi > T3 - 1 ? T3 - 1 : (hi < -1 ? -1 : hi));
        }
        W[gi][axis][0] = wl;
        W[gi][axis][1] = wh;
      } else {
        for (int r = 0; r < T3; ++r) dst[r] = make_double2(0.0, 0.0);
        W[gi][axis][0] = T3;
        W[gi][axis][1] = -1;
      }
    }
    __syncthreads();
    for (int gi = 0; gi < nc; ++gi) {
      // outside the window the factors are exact zeros and add nothing: skip the column,
      // and the quarters of it (4 points) that miss the window along z
      if (ix < W[gi][0][0] || ix > W[gi][0][1] || iy < W[gi][1][0] || iy > W[gi][1][1]) continue;
      const int z0 = W[gi][2][0] >> 2, z1 = W[gi][2][1] >> 2;
      const double2 X = F[0][gi][ix], Y = F[1][gi][iy];
      const double xr = X.x * Y.x - X.y * Y.y, xi = X.x * Y.y + X.y * Y.x;
#pragma unroll
      for (int qz = 0; qz < T3 / 4; ++qz) {
        if (qz < z0 || qz > z1) continue;
#pragma unroll
        for (int i = 4 * qz; i < 4 * qz + 4; ++i) {
          const double2 Z = F[2][gi][i];
          acc[i] = fma(xr, Z.x, fma(-xi, Z.y, acc[i]));
        }
      }
    }
    __syncthreads();
  }
  double* dst = partial + w * (int64_t)(T3 * T3 * T3) + (int64_t)(ix * T3 + iy) * T3;
#pragma unroll
  for (int i = 0; i < T3; ++i) dst[i] = acc[i];
}

template <int D>
__global__ void __launch_bounds__(NT) k_reduce(GridDev gd, const ShotDev* __restrict__ shots,
                                               int nshots, const int64_t* __restrict__ seg_off,
                                               const double* __restrict__ partial,
                                               double* __restrict__ out) {
  const int64_t t = blockIdx.x;
  const int s = shot_of_tile(shots, nshots, t);
  const ShotDev& sh = shots[s];
  int64_t a[D], b[D];
  tile_box<D>(gd, sh, t - sh.tile_off, a, b);
  constexpr int TP = (D == 1) ? T1 : (D == 2 ? T2 * T2 : T3 * T3 * T3);
  const int64_t w0 = seg_off[t], w1 = seg_off[t + 1];
  for (int idx = threadIdx.x; idx < TP; idx += NT) {
    double v = 0.0;
    for (int64_t w = w0; w < w1; ++w) v += partial[w * TP + idx];
    if constexpr (D == 1) {
      int64_t i = a[0] + idx;
      if (i <= b[0]) out[(int64_t)s * gd.npts + i] = v;
    } else if constexpr (D == 2) {
      int64_t ix = a[0] + idx / T2, iz = a[1] + idx % T2;
      if (ix <= b[0] && iz <= b[1]) out[(int64_t)s * gd.npts + ix * gd.n[1] + iz] = v;
    } else {
      int64_t ix = a[0] + idx / (T3 * T3), iy = a[1] + (idx / T3) % T3, iz = a[2] + idx % T3;
      if (ix <= b[0] && iy <= b[1] && iz <= b[2])
        out[(int64_t)s * gd.npts + (ix * gd.n[1] + iy) * gd.n[2] + iz] = v;
    }
  }
}

}  // namespace

// Splits of the binning: runs of at least kBinChunk Gaussians, so that tiles x splits
// CTAs fill the GPU even when a shot has few tiles; at most 2^30 CTAs.
// With the counts on the device (pipeline graph) the splits cover the plan's whole
// Gaussian capacity.
void bin_splits(const fga_plan_s* p, int* nsplit, int64_t* chunk) {
  int64_t gmax = 1;
  if (p->dev_counts)
    gmax = std::max<int64_t>(gmax, (int64_t)p->g_cap);
  else
    for (const auto& sh : p->shots) gmax = std::max<int64_t>(gmax, sh.g_cnt);
  int64_t ns = (gmax + kBinChunk - 1) / kBinChunk;
  ns = std::max<int64_t>(1, std::min<int64_t>(ns, ((int64_t)1 << 30) / std::max<int64_t>(p->ntiles, 1)));
  *nsplit = (int)ns;
  *chunk = (gmax + ns - 1) / ns;
}

// Counts per (tile, split), their exclusive scan in tile-major order, and the tiles'
// list offsets d_tile_off (the total at d_tile_off[ntiles]).
cudaError_t launch_binning(fga_plan_s* p) {
  if (p->ntiles == 0) return cudaSuccess;
  int nsplit;
  int64_t chunk;
  bin_splits(p, &nsplit, &chunk);
  const int64_t items = p->ntiles * nsplit;
  if ((size_t)items + 1 > p->bin_cap) return cudaErrorInvalidValue;  // capacity not set up
  if (p->rng_cap < (size_t)p->grid.dim * 2 * p->g_cap) return cudaErrorInvalidValue;  // not set up
  const int64_t G = p->dev_counts ? (int64_t)p->g_cap : p->G;
  const int64_t* gm = p->dev_counts ? p->d_gm : nullptr;
  if (G > 0) {
    const unsigned gbk = (unsigned)std::max<int64_t>(1, std::min<int64_t>((G + 255) / 256, 4096));
    auto ranges = p->grid.dim == 1 ? k_bin_ranges<1> : (p->grid.dim == 2 ? k_bin_ranges<2> : k_bin_ranges<3>);
    ranges<<<gbk, 256, 0, p->stream>>>(p->grid, p->d_shots, p->d_gshot, p->kappa, p->d_state,
                                       (int64_t)p->g_cap, G, gm, p->d_rng);
    p->launches += 1;
  }
  auto bin = p->grid.dim == 1 ? k_bin_r<1, false> : (p->grid.dim == 2 ? k_bin_r<2, false> : k_bin_r<3, false>);
  bin<<<(unsigned)items, NT, 0, p->stream>>>(p->grid, p->d_shots, p->nshots, p->d_rng, (int64_t)p->g_cap,
                                             p->d_bin_off, nullptr, nullptr, 0, nsplit, chunk, p->d_status);
  p->launches += 1;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = launch_scan(p, p->d_bin_off, items);
  if (e != cudaSuccess) return e;
  k_tile_offsets<<<(unsigned)((p->ntiles + 256) / 256), 256, 0, p->stream>>>(p->d_bin_off, nsplit,
                                                                            p->ntiles, p->d_tile_off);
  p->launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_binning_fill(fga_plan_s* p) {
  if (p->ntiles == 0) return cudaSuccess;
  int nsplit;
  int64_t chunk;
  bin_splits(p, &nsplit, &chunk);
  const int64_t items = p->ntiles * nsplit;
  if ((size_t)items + 1 > p->bin_cap) return cudaErrorInvalidValue;
  if (p->rng_cap < (size_t)p->grid.dim * 2 * p->g_cap) return cudaErrorInvalidValue;
  auto fill = p->grid.dim == 1 ? k_bin_r<1, true> : (p->grid.dim == 2 ? k_bin_r<2, true> : k_bin_r<3, true>);
  fill<<<(unsigned)items, NT, 0, p->stream>>>(p->grid, p->d_shots, p->nshots, p->d_rng, (int64_t)p->g_cap,
                                              nullptr, p->d_bin_off, p->d_tile_list, (int64_t)p->list_cap,
                                              nsplit, chunk, p->d_status);
  p->launches += 1;
  return cudaGetLastError();
}

// Gaussians per work item: the tuned or default length, raised when needed so that the
// partial tiles (one per work item, sized for the tile lists' capacity) stay within
// kPartialBudget bytes.
int64_t segment_len(fga_plan_s* p) {
  const int64_t want = p->seg > 0 ? p->seg : (p->grid.dim == 1 ? SEG1 : (p->grid.dim == 2 ? SEG2 : SEG3));
  const int64_t tile_bytes = (int64_t)tile_points(p->grid.dim) * (int64_t)sizeof(double);
  const int64_t items = std::max<int64_t>(kPartialBudget / tile_bytes - p->ntiles, 1);
  const int64_t floor_len = ((int64_t)p->list_cap + items - 1) / items;
  return std::max<int64_t>(want, floor_len);
}

size_t partial_items(fga_plan_s* p) {
  const int64_t seg = segment_len(p);
  return (size_t)p->ntiles + (p->list_cap + seg - 1) / seg;
}

size_t tile_points(int dim) {
  return dim == 1 ? (size_t)T1 : (dim == 2 ? (size_t)T2 * T2 : (size_t)T3 * T3 * T3);
}

// Split of every tile's list into segments, one CTA per (tile, segment) writing a
// partial tile, then the ordered reduction into u_dev.
cudaError_t launch_reconstruct(fga_plan_s* p, double* u_dev) {
  if (p->ntiles == 0) return cudaSuccess;
  const int64_t seg = segment_len(p);
  k_segments<<<(unsigned)((p->ntiles + 255) / 256), 256, 0, p->stream>>>(
      p->d_tile_off, p->ntiles, (int64_t)p->list_cap, seg, p->d_seg_off);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  p->launches += 1;
  e = launch_scan(p, p->d_seg_off, p->ntiles);
  if (e != cudaSuccess) return e;
  const unsigned items = (unsigned)partial_items(p);
  if (p->grid.dim == 1) {
    k_gather1<<<items, NT, 0, p->stream>>>(p->grid, p->d_shots, p->nshots, p->kappa, p->d_state,
                                           (int64_t)p->g_cap, p->d_gcoef, p->d_tile_off,
                                           p->d_tile_list, (int64_t)p->list_cap, p->d_seg_off,
                                           p->ntiles, seg, p->d_partial);
    k_reduce<1><<<(unsigned)p->ntiles, NT, 0, p->stream>>>(p->grid, p->d_shots, p->nshots,
                                                           p->d_seg_off, p->d_partial, u_dev);
  } else if (p->grid.dim == 2) {
    k_gather2<<<items, NT, 0, p->stream>>>(p->grid, p->d_shots, p->nshots, p->kappa, p->d_state,
                                           (int64_t)p->g_cap, p->d_gcoef, p->d_tile_off,
                                           p->d_tile_list, (int64_t)p->list_cap, p->d_seg_off,
                                           p->ntiles, seg, p->d_partial);
    k_reduce<2><<<(unsigned)p->ntiles, NT, 0, p->stream>>>(p->grid, p->d_shots, p->nshots,
                                                           p->d_seg_off, p->d_partial, u_dev);
  } else {
    k_gather3<<<items, NT, 0, p->stream>>>(p->grid, p->d_shots, p->nshots, p->kappa, p->d_state,
                                           (int64_t)p->g_cap, p->d_gcoef, p->d_tile_off,
                                           p->d_tile_list, (int64_t)p->list_cap, p->d_seg_off,
                                           p->ntiles, seg, p->d_partial);
    k_reduce<3><<<(unsigned)p->ntiles, NT, 0, p->stream>>>(p->grid, p->d_shots, p->nshots,
                                                           p->d_seg_off, p->d_partial, u_dev);
  }
  p->launches += 2;
  return cudaGetLastError();
}

int tile_edge(int dim) { return dim == 1 ? T1 : (dim == 2 ? T2 : T3); }

}  // namespace fga

// ---------------------------------------------------------------------------
// Reconstruction that allocates nothing (fga_reconstruct_static in fga.h).
//
// For callers that cannot call cudaMalloc: code that runs where the allocator
// is off limits (for instance inside a host callback or a driver layer that owns
// all device memory), or a caller that has budgeted every byte of the device.
// The scratch that the plan-based path allocates per plan -- the shot record,
// the per-tile offsets and the per-tile Gaussian lists -- lives here in one
// file-scope device array of fixed size, which every GPU that loads this
// library holds until the process exits. The caller passes the inputs
// (centres, momenta and coefficients of the Gaussians) and the output grid.
// ---------------------------------------------------------------------------

namespace fga {
namespace {

constexpr int64_t kStaticMaxTiles = 16384;     // 64x64 tiles (2D) or 256-point tiles (1D)
constexpr int64_t kStaticMaxPairs = 1 << 21;   // (Gaussian, tile) list entries per chunk
constexpr size_t align256(size_t b) { return (b + 255) / 256 * 256; }
constexpr size_t kStOffShot = 0;
constexpr size_t kStOffStatus = align256(sizeof(ShotDev));
constexpr size_t kStOffTiles = kStOffStatus + 256;
constexpr size_t kStOffList = kStOffTiles + align256(sizeof(int64_t) * (kStaticMaxTiles + 1));
constexpr size_t kStaticBytes = kStOffList + align256(sizeof(int32_t) * kStaticMaxPairs);

// Gather of one tile over its whole list, added to the output (chunks of Gaussians
// are summed one after the other, so the order of summation is fixed).
__global__ void __launch_bounds__(NT) k_gather2_tile_add(GridDev gd, const ShotDev* __restrict__ shots,
                                                         double kappa,
                                                         const double* __restrict__ state, int64_t ld,
                                                         const double2* __restrict__ coef,
                                                         const int64_t* __restrict__ off,
                                                         const int32_t* __restrict__ list,
                                                         int64_t list_cap, double* __restrict__ out) {
  const int64_t t = blockIdx.x;
  const ShotDev& sh = shots[0];
  const double cut = kappa * sh.sqrt_eps, inv_eps = sh.inv_eps;
  int64_t a[2], b[2];
  tile_box<2>(gd, sh, t, a, b);
  __shared__ double2 Xs[CH][T2];
  __shared__ double2 Zs[CH][T2];
  __shared__ int win[CH][4];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int wx = warp >> 1, wz = warp & 1;
  const int lx = lane >> 3, lz = lane & 7;
  const int x0 = wx * 16 + lx * 4, z0 = wz * 32 + lz * 4;
  const int px0 = wx * 16, px1 = wx * 16 + 15, pz0 = wz * 32, pz1 = wz * 32 + 31;
  double accr[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) accr[i][j] = 0.0;
  const int64_t l0 = min(off[t], list_cap), l1 = min(off[t + 1], list_cap);
  for (int64_t c0 = l0; c0 < l1; c0 += CH) {
    const int nc = (int)((l1 - c0) < CH ? (l1 - c0) : CH);
    {
      const int gi = threadIdx.x >> 4, axis = (threadIdx.x >> 3) & 1, part = threadIdx.x & 7;
      if (gi < nc) {
        int32_t g = list[c0 + gi];
        double Q = state[axis * ld + g], P = state[(2 + axis) * ld + g];
        double2 cf = axis == 0 ? coef[g] : make_double2(1.0, 0.0);
        double2* dst = (axis == 0 ? Xs[gi] : Zs[gi]) + part * 8;
        const Axis ax = grid_axis(gd, axis);
        const int64_t a_ax = axis == 0 ? a[0] : a[1];
        if (ax.periodic) {
          for (int r = 0; r < 8; ++r) {
            double2 f = axis_factor(ax, a_ax + part * 8 + r, Q, P, cut, inv_eps);
            dst[r] = make_double2(cf.x * f.x - cf.y * f.y, cf.x * f.y + cf.y * f.x);
          }
        } else {
          double xi0 = ax.o + (double)(a_ax + part * 8) * ax.h;
          axis_factors<8>(xi0, ax.h, Q, P, cut, inv_eps, cf, dst);
        }
        if (part == 0) {
          if (ax.periodic) {
            win[gi][2 * axis] = 0;
            win[gi][2 * axis + 1] = T2 - 1;
          } else {
            int64_t lo, hi;
            window_range_ax(ax, Q, cut, lo, hi);
            win[gi][2 * axis] = (int)((lo - a_ax) > -1 ? (lo - a_ax) : -1);
            win[gi][2 * axis + 1] = (int)((hi - a_ax) < T2 ? (hi - a_ax) : T2);
          }
        }
      }
    }
    __syncthreads();
    for (int gi = 0; gi < nc; ++gi) {
      if (win[gi][0] > px1 || win[gi][1] < px0 || win[gi][2] > pz1 || win[gi][3] < pz0) continue;
      double2 xv[4], zv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        xv[i] = Xs[gi][x0 + i];
        zv[i] = Zs[gi][z0 + i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
          accr[i][j] = fma(xv[i].x, zv[j].x, fma(-xv[i].y, zv[j].y, accr[i][j]));
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int64_t ix = a[0] + x0 + i;
    if (ix > b[0]) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int64_t iz = a[1] + z0 + j;
      if (iz > b[1]) continue;
      out[ix * gd.n[1] + iz] += accr[i][j];
    }
  }
}

__global__ void __launch_bounds__(NT) k_gather1_tile_add(GridDev gd, const ShotDev* __restrict__ shots,
                                                         double kappa,
                                                         const double* __restrict__ state, int64_t ld,
                                                         const double2* __restrict__ coef,
                                                         const int64_t* __restrict__ off,
                                                         const int32_t* __restrict__ list,
                                                         int64_t list_cap, double* __restrict__ out) {
  const int64_t t = blockIdx.x;
  const ShotDev& sh = shots[0];
  const double cut = kappa * sh.sqrt_eps, inv_eps = sh.inv_eps;
  const int64_t i = t * T1 + threadIdx.x;
  __shared__ double sQ[CH1], sP[CH1];
  __shared__ double2 sC[CH1];
  double re = 0.0;
  const int64_t l0 = min(off[t], list_cap), l1 = min(off[t + 1], list_cap);
  for (int64_t c0 = l0; c0 < l1; c0 += CH1) {
    int nc = (int)((l1 - c0) < CH1 ? (l1 - c0) : CH1);
    if (threadIdx.x < nc) {
      int32_t g = list[c0 + threadIdx.x];
      sQ[threadIdx.x] = state[0 * ld + g];
      sP[threadIdx.x] = state[1 * ld + g];
      sC[threadIdx.x] = coef[g];
    }
    __syncthreads();
    for (int j = 0; j < nc; ++j) {
      double2 x = axis_factor(grid_axis(gd, 0), i, sQ[j], sP[j], cut, inv_eps);
      re = fma(sC[j].x, x.x, fma(-sC[j].y, x.y, re));
    }
    __syncthreads();
  }
  if (i < gd.n[0]) out[i] += re;
}

}  // namespace
}  // namespace fga

// The scratch of fga_reconstruct_static: [shot record | status | tile offsets | lists].
static __device__ __align__(256) unsigned char fga_static_scratch[fga::kStaticBytes];

namespace {

constexpr int kStaticMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_addr[kStaticMaxDevices] = {};

// Device address of the scratch on the current device, looked up once per device.
cudaError_t static_scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kStaticMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_addr[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, fga_static_scratch);
    if (e != cudaSuccess) return e;
    g_static_addr[dev] = ptr;
  }
  *out = g_static_addr[dev];
  return cudaSuccess;
}

fga_status static_fail(fga_status st, const std::string& msg) {
  fga::set_unbound_error(msg);
  return st;
}

// True for managed memory and for device memory of the current device (memory of
// another GPU would be reached without peer access by the kernels launched here).
bool device_pointer(const void* ptr) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace

extern "C" fga_status fga_reconstruct_static(int dim, const int64_t* n, const double* h,
                                             const double* origin, const int* periodic, double eps,
                                             double kappa, int64_t nG, const double* qp,
                                             const double* coef, double* u, void* stream) {
  using namespace fga;
  if (dim < 1 || dim > 2) return static_fail(FGA_ERR_INVALID, "dim must be 1 or 2");
  if (!n || !h || !origin || !periodic || !u)
    return static_fail(FGA_ERR_INVALID, "grid description and u must not be NULL");
  if (!(eps > 0.0) || !std::isfinite(eps) || !(kappa > 0.0) || !std::isfinite(kappa))
    return static_fail(FGA_ERR_INVALID, "eps and kappa must be finite and > 0");
  if (nG < 0 || nG > (((int64_t)1 << 31) - 1))
    return static_fail(FGA_ERR_INVALID, "nG must be in [0, 2^31 - 1]");
  if (nG > 0 && (!qp || !coef)) return static_fail(FGA_ERR_INVALID, "qp and coef must not be NULL");
  if (!device_pointer(u) || (nG > 0 && (!device_pointer(qp) || !device_pointer(coef))))
    return static_fail(FGA_ERR_INVALID, "qp, coef and u must be device pointers of the current device");
  cudaStream_t st = (cudaStream_t)stream;
  GridDev gd;
  std::memset(&gd, 0, sizeof(gd));
  gd.dim = dim;
  gd.npts = 1;
  ShotDev sh;
  std::memset(&sh, 0, sizeof(sh));
  sh.eps = eps;
  sh.sqrt_eps = std::sqrt(eps);
  sh.inv_eps = 1.0 / eps;
  const int TS = tile_edge(dim);
  int64_t ntiles = 1;
  size_t per = 1;  // tiles one Gaussian can meet at most
  for (int k = 0; k < kMaxDim; ++k) gd.tile[k] = TS;
  for (int k = 0; k < dim; ++k) {
    if (n[k] < 4 || n[k] > ((int64_t)1 << 30) || !(h[k] > 0.0) || !std::isfinite(h[k]) ||
        !std::isfinite(origin[k]))
      return static_fail(FGA_ERR_INVALID, "bad grid axis");
    gd.n[k] = n[k];
    gd.h[k] = h[k];
    gd.o[k] = origin[k];
    gd.inv_h[k] = 1.0 / h[k];
    gd.periodic[k] = periodic[k] ? 1 : 0;
    gd.L[k] = gd.periodic[k] ? (double)n[k] * h[k] : 0.0;
    gd.npts *= n[k];
    sh.ntile[k] = (int)((n[k] + TS - 1) / TS);
    ntiles *= sh.ntile[k];
    if (gd.periodic[k] && kappa * sh.sqrt_eps > 2.0 * gd.L[k])
      return static_fail(FGA_ERR_INVALID, "kappa sqrt(eps) must not exceed two periods");
    double wpts = 2.0 * kappa * sh.sqrt_eps * gd.inv_h[k] + 6.0;
    size_t mk = (size_t)(wpts / TS) + 2;
    if (gd.periodic[k]) mk *= 5;
    per *= std::min<size_t>(mk, (size_t)sh.ntile[k]);
  }
  for (int k = dim; k < kMaxDim; ++k) {
    gd.n[k] = 1;
    gd.h[k] = gd.inv_h[k] = 1.0;
  }
  if (ntiles > kStaticMaxTiles)
    return static_fail(FGA_ERR_CAPACITY,
                       "the grid needs " + std::to_string(ntiles) + " tiles; the static scratch holds " +
                           std::to_string(kStaticMaxTiles));
  void* base = nullptr;
  cudaError_t e = static_scratch_address(&base);
  if (e != cudaSuccess)
    return static_fail(FGA_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  unsigned char* b8 = (unsigned char*)base;
  ShotDev* d_shot = (ShotDev*)(b8 + kStOffShot);
  int* d_status = (int*)(b8 + kStOffStatus);
  int64_t* d_off = (int64_t*)(b8 + kStOffTiles);
  int32_t* d_list = (int32_t*)(b8 + kStOffList);
#define ST_CUDA(call)                                                                     \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return static_fail(FGA_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)
  ST_CUDA(cudaMemsetAsync(u, 0, sizeof(double) * gd.npts, st));
  ST_CUDA(cudaMemsetAsync(d_status, 0, sizeof(int), st));
  const int64_t chunk = std::max<int64_t>(1, kStaticMaxPairs / (int64_t)per);
  const double2* cf = reinterpret_cast<const double2*>(coef);
  for (int64_t g0 = 0; g0 < nG; g0 += chunk) {
    sh.g_off = g0;
    sh.g_cnt = std::min<int64_t>(chunk, nG - g0);
    // pageable source: the copy is staged before cudaMemcpyAsync returns
    ST_CUDA(cudaMemcpyAsync(d_shot, &sh, sizeof(ShotDev), cudaMemcpyHostToDevice, st));
    if (dim == 1) {
      k_bin<1, false><<<(unsigned)ntiles, NT, 0, st>>>(gd, d_shot, 1, kappa, qp, nG, d_off, nullptr,
                                                       nullptr, 0, 1, sh.g_cnt, d_status);
    } else {
      k_bin<2, false><<<(unsigned)ntiles, NT, 0, st>>>(gd, d_shot, 1, kappa, qp, nG, d_off, nullptr,
                                                       nullptr, 0, 1, sh.g_cnt, d_status);
    }
    ST_CUDA(cudaGetLastError());
    ST_CUDA(launch_scan_on(st, d_off, ntiles));
    if (dim == 1) {
      k_bin<1, true><<<(unsigned)ntiles, NT, 0, st>>>(gd, d_shot, 1, kappa, qp, nG, nullptr, d_off,
                                                      d_list, kStaticMaxPairs, 1, sh.g_cnt, d_status);
      k_gather1_tile_add<<<(unsigned)ntiles, NT, 0, st>>>(gd, d_shot, kappa, qp, nG, cf, d_off,
                                                          d_list, kStaticMaxPairs, u);
    } else {
      k_bin<2, true><<<(unsigned)ntiles, NT, 0, st>>>(gd, d_shot, 1, kappa, qp, nG, nullptr, d_off,
                                                      d_list, kStaticMaxPairs, 1, sh.g_cnt, d_status);
      k_gather2_tile_add<<<(unsigned)ntiles, NT, 0, st>>>(gd, d_shot, kappa, qp, nG, cf, d_off,
                                                          d_list, kStaticMaxPairs, u);
    }
    ST_CUDA(cudaGetLastError());
  }
  int status = 0;
  ST_CUDA(cudaMemcpyAsync(&status, d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
  ST_CUDA(cudaStreamSynchronize(st));
#undef ST_CUDA
  if (status & kStatusCapacity)
    return static_fail(FGA_ERR_CAPACITY, "a chunk overflowed the static tile lists");
  return FGA_OK;
}
