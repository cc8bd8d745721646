// Output tiles shared by the binning and the gather kernels: tile k of a shot covers
// grid indices [k * tile, min((k + 1) * tile, n) - 1] per axis (tile edges are a plan
// parameter); a Gaussian belongs to a tile when its kappa sqrt(eps) window meets it.
#pragma once

#include "fga_internal.cuh"

namespace fga {

__device__ __forceinline__ int shot_of_tile(const ShotDev* shots, int nshots, int64_t t) {
  int lo = 0, hi = nshots - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (shots[mid].tile_off <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// One axis of the grid picked by a runtime index with conditionals (indexing the grid's
// arrays with a runtime value would put the kernel parameter block in local memory).
struct Axis {
  double o, h, inv_h, L;
  int64_t n;
  int periodic;
};

__device__ __forceinline__ Axis grid_axis(const GridDev& gd, int k) {
  Axis ax;
  ax.o = k == 0 ? gd.o[0] : (k == 1 ? gd.o[1] : gd.o[2]);
  ax.h = k == 0 ? gd.h[0] : (k == 1 ? gd.h[1] : gd.h[2]);
  ax.inv_h = k == 0 ? gd.inv_h[0] : (k == 1 ? gd.inv_h[1] : gd.inv_h[2]);
  ax.L = k == 0 ? gd.L[0] : (k == 1 ? gd.L[1] : gd.L[2]);
  ax.n = k == 0 ? gd.n[0] : (k == 1 ? gd.n[1] : gd.n[2]);
  ax.periodic = k == 0 ? gd.periodic[0] : (k == 1 ? gd.periodic[1] : gd.periodic[2]);
  return ax;
}

__device__ __forceinline__ void window_range_ax(const Axis& ax, double Q, double cut, int64_t& lo,
                                                int64_t& hi) {
  lo = (int64_t)floor((Q - cut - ax.o) * ax.inv_h) - 1;
  hi = (int64_t)ceil((Q + cut - ax.o) * ax.inv_h) + 1;
}

// Window of Gaussian (Q, cut) along one axis as a conservative grid-index range.
__device__ __forceinline__ void window_range(const GridDev& gd, int k, double Q, double cut,
                                             int64_t& lo, int64_t& hi) {
  lo = (int64_t)floor((Q - cut - gd.o[k]) * gd.inv_h[k]) - 1;
  hi = (int64_t)ceil((Q + cut - gd.o[k]) * gd.inv_h[k]) + 1;
}

// Does the window of the Gaussian with centre Q meet the index box [a, b] on all axes?
template <int D>
__device__ __forceinline__ bool overlaps(const GridDev& gd, const double* Q, double cut,
                                         const int64_t* a, const int64_t* b) {
#pragma unroll
  for (int k = 0; k < D; ++k) {
    bool any = false;
    int lmax = gd.periodic[k] ? 2 : 0;
    for (int l = -lmax; l <= lmax; ++l) {
      int64_t lo, hi;
      window_range(gd, k, Q[k] + l * gd.L[k], cut, lo, hi);
      any = any || (lo <= b[k] && hi >= a[k]);
    }
    if (!any) return false;
  }
  return true;
}

template <int D>
__device__ __forceinline__ void tile_box(const GridDev& gd, const ShotDev& sh, int64_t tloc,
                                         int64_t* a, int64_t* b) {
  int64_t t[D];
  if constexpr (D == 1) {
    t[0] = tloc;
  } else if constexpr (D == 2) {
    t[0] = tloc / sh.ntile[1];
    t[1] = tloc - t[0] * sh.ntile[1];
  } else {
    const int64_t yz = (int64_t)sh.ntile[1] * sh.ntile[2];
    t[0] = tloc / yz;
    const int64_t r = tloc - t[0] * yz;
    t[1] = r / sh.ntile[2];
    t[2] = r - t[1] * sh.ntile[2];
  }
#pragma unroll
  for (int k = 0; k < D; ++k) {
    a[k] = t[k] * gd.tile[k];
    b[k] = min(a[k] + gd.tile[k] - 1, gd.n[k] - 1);
  }
}

__device__ __forceinline__ int64_t tile_of_item(const int64_t* seg_off, int64_t ntiles, int64_t w) {
  int64_t lo = 0, hi = ntiles - 1;
  while (lo < hi) {
    int64_t mid = (lo + hi + 1) >> 1;
    if (seg_off[mid] <= w) lo = mid; else hi = mid - 1;
  }
  return lo;
}

}  // namespace fga
