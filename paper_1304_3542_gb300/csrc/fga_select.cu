// Choice of the set G+ (thresholding paragraph of the Initial wavefield
// decomposition section): every valid (q,p) with |psi+| >= tau * max|psi+| is
// kept. Because the p-grid is symmetric and the data real, max|psi+| over the
// + branch equals the maximum over both branches.
//
// Deterministic stream compaction in three passes over the psi+ segments
// (each shot's segment is padded to whole blocks of kScanBlock entries):
// count per block, one exclusive scan over the blocks, and an ordered scatter
// that keeps the (q, p) order of the segment. The Gaussian list therefore comes
// out shot-major, q-major, p-minor, whatever the launch order.
#include "fga_internal.cuh"

namespace fga {

namespace {

constexpr int NT = 256;
constexpr int PER = kScanBlock / NT;  // entries per thread

__device__ __forceinline__ int shot_of_block(const ShotDev* shots, int nshots, int64_t e) {
  int lo = 0, hi = nshots - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (shots[mid].psi_off <= e) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <int D>
__device__ __forceinline__ bool p_valid(const ShotDev& sh, int64_t jp) {
  if constexpr (D == 1) {
    return jp != 0 && jp != sh.nb[0] / 2;
  } else if constexpr (D == 3) {
    const int64_t nb12 = (int64_t)sh.nb[1] * sh.nb[2];
    const int64_t j0 = jp / nb12, j1 = (jp - j0 * nb12) / sh.nb[2], j2 = jp - j0 * nb12 - j1 * sh.nb[2];
    return j0 != 0 && j1 != 0 && j2 != 0 &&
           !(j0 == sh.nb[0] / 2 && j1 == sh.nb[1] / 2 && j2 == sh.nb[2] / 2);
  } else {
    int64_t j0 = jp / sh.nb[1], j1 = jp - j0 * sh.nb[1];
    return j0 != 0 && j1 != 0 && !(j0 == sh.nb[0] / 2 && j1 == sh.nb[1] / 2);
  }
}

// Flat index on the full q-grid of the local index ql of the shot's active q rectangle.
template <int D>
__device__ __forceinline__ int64_t q_flat(const ShotDev& sh, int64_t ql) {
  if constexpr (D == 1) {
    return sh.qlo[0] + ql;
  } else if constexpr (D == 3) {
    const int64_t qn12 = sh.qn[1] * sh.qn[2];
    const int64_t m0 = ql / qn12, m1 = (ql - m0 * qn12) / sh.qn[2], m2 = ql - m0 * qn12 - m1 * sh.qn[2];
    return ((sh.qlo[0] + m0) * sh.nq[1] + (sh.qlo[1] + m1)) * sh.nq[2] + (sh.qlo[2] + m2);
  } else {
    const int64_t mxl = ql / sh.qn[1], mzl = ql - mxl * sh.qn[1];
    return (sh.qlo[0] + mxl) * sh.nq[1] + (sh.qlo[1] + mzl);
  }
}

template <int D>
__device__ __forceinline__ bool keep(const ShotDev& sh, const double2* psi, int64_t e, double thr2) {
  int64_t loc = e - sh.psi_off;
  if (loc < 0 || loc >= sh.psi_len) return false;
  int64_t jp = loc % sh.np;
  if (!p_valid<D>(sh, jp)) return false;
  double2 v = psi[e];
  return abs2_rn(v) >= thr2;
}

template <int D>
__global__ void __launch_bounds__(NT) k_select_count(const ShotDev* __restrict__ shots, int nshots,
                                                     const double2* __restrict__ psi,
                                                     const unsigned long long* __restrict__ max2,
                                                     double tau2, int64_t* blk) {
  int64_t base = (int64_t)blockIdx.x * kScanBlock;
  int s = shot_of_block(shots, nshots, base);
  const ShotDev& sh = shots[s];
  double thr2 = tau2 * __longlong_as_double((long long)max2[s]);
  int c = 0;
  for (int i = 0; i < PER; ++i) c += keep<D>(sh, psi, base + threadIdx.x + NT * i, thr2) ? 1 : 0;
  __shared__ int red[NT / 32];
  for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int sum = 0;
    for (int w = 0; w < NT / 32; ++w) sum += red[w];
    blk[blockIdx.x] = sum;
  }
}

// Exclusive scan of n int64 values in place; a[n] receives the total. One block.
__global__ void __launch_bounds__(1024) k_scan_exclusive(int64_t* a, int64_t n) {
  __shared__ int64_t warp_sums[32];
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t base = 0; base < n; base += 1024) {
    int64_t i = base + threadIdx.x;
    int64_t v = (i < n) ? a[i] : 0;
    int64_t x = v;
    for (int off = 1; off < 32; off <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, x, off);
      if (lane >= off) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
      int64_t w = warp_sums[lane];
      for (int off = 1; off < 32; off <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, w, off);
        if (lane >= off) w += y;
      }
      warp_sums[lane] = w;
    }
    __syncthreads();
    int64_t excl = x - v + (warp > 0 ? warp_sums[warp - 1] : 0) + carry;
    if (i < n) a[i] = excl;
    __syncthreads();
    if (threadIdx.x == 1023) carry = excl + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) a[n] = carry;
}

template <int D>
__global__ void __launch_bounds__(NT) k_select_scatter(const ShotDev* __restrict__ shots, int nshots,
                                                       const double2* __restrict__ psi,
                                                       const unsigned long long* __restrict__ max2,
                                                       double tau2, const int64_t* __restrict__ blk,
                                                       int32_t* gshot, int64_t* gq, int32_t* gp,
                                                       double2* gpsi, const double2* __restrict__ psi_f1,
                                                       double2* gpsi_f1, int64_t cap) {
  int64_t base = (int64_t)blockIdx.x * kScanBlock;
  int s = shot_of_block(shots, nshots, base);
  const ShotDev& sh = shots[s];
  double thr2 = tau2 * __longlong_as_double((long long)max2[s]);
  // thread t owns PER consecutive entries, so the block order is the entry order
  int64_t e0 = base + (int64_t)threadIdx.x * PER;
  bool f[PER];
  int c = 0;
  for (int i = 0; i < PER; ++i) {
    f[i] = keep<D>(sh, psi, e0 + i, thr2);
    c += f[i] ? 1 : 0;
  }
  __shared__ int warp_tot[NT / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = c;
  for (int off = 1; off < 32; off <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, off);
    if (lane >= off) x += y;
  }
  if (lane == 31) warp_tot[warp] = x;
  __syncthreads();
  int wbase = 0;
  for (int w = 0; w < warp; ++w) wbase += warp_tot[w];
  int64_t pos = blk[blockIdx.x] + wbase + (x - c);
  for (int i = 0; i < PER; ++i) {
    if (!f[i] || pos >= cap) continue;  // beyond the capacity: k_counts_finish flags it
    int64_t loc = e0 + i - sh.psi_off;
    int64_t ql = loc / sh.np, jp = loc - ql * sh.np;
    const int64_t qflat = q_flat<D>(sh, ql);
    gshot[pos] = s;
    gq[pos] = qflat;
    gp[pos] = (int32_t)jp;
    gpsi[pos] = psi[e0 + i];
    gpsi_f1[pos] = psi_f1[e0 + i];
    ++pos;
  }
}

// ---------------------------------------------------------------------------
// N-largest selection (keep_n > 0): per shot, the keep_n largest |psi+| over the valid
// (q, p), ties by segment order (q index, then p index). The key of an entry is the bit
// pattern of |psi+|^2 plus 1 (monotone for non-negative doubles; invalid p and padding
// get 0). A radix select over 8 passes of 8 bits (from the top) finds the cut key K and
// how many entries equal to K are still to take; the entries are then compacted in order:
// every key > K, and the first `take` keys == K.
template <int D>
__device__ __forceinline__ unsigned long long topk_key(const ShotDev& sh, const double2* psi, int64_t e) {
  const int64_t loc = e - sh.psi_off;
  if (loc < 0 || loc >= sh.psi_len) return 0ull;
  if (!p_valid<D>(sh, loc % sh.np)) return 0ull;
  const double2 v = psi[e];
  return (unsigned long long)__double_as_longlong(abs2_rn(v)) + 1ull;
}

// topk[s] = {prefix, mask, to_take, take_all}
__global__ void k_topk_init(unsigned long long* topk, int nshots, long long keep_n) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nshots) return;
  topk[4 * s + 0] = 0ull;
  topk[4 * s + 1] = 0ull;
  topk[4 * s + 2] = (unsigned long long)keep_n;
  topk[4 * s + 3] = 0ull;
}

template <int D>
__global__ void __launch_bounds__(NT) k_topk_hist(const ShotDev* __restrict__ shots, int nshots,
                                                  const double2* __restrict__ psi,
                                                  const unsigned long long* __restrict__ topk,
                                                  int shift, unsigned long long* hist) {
  __shared__ unsigned int h[256];
  for (int i = threadIdx.x; i < 256; i += NT) h[i] = 0u;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kScanBlock;
  const int s = shot_of_block(shots, nshots, base);
  const ShotDev& sh = shots[s];
  const unsigned long long prefix = topk[4 * s], mask = topk[4 * s + 1];
  for (int i = 0; i < PER; ++i) {
    const unsigned long long k = topk_key<D>(sh, psi, base + threadIdx.x + NT * i);
    if (k != 0ull && (k & mask) == prefix) atomicAdd(&h[(k >> shift) & 255ull], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 256; i += NT)
    if (h[i]) atomicAdd(hist + 256 * s + i, (unsigned long long)h[i]);
}

// One thread per shot: the digit at this pass where the count from the top reaches
// to_take; clears the histogram for the next pass.
__global__ void k_topk_pick(unsigned long long* topk, unsigned long long* hist, int nshots, int shift) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nshots) return;
  unsigned long long* h = hist + 256 * s;
  unsigned long long need = topk[4 * s + 2];
  if (topk[4 * s + 3] == 0ull && need > 0ull) {
    unsigned long long total = 0ull;
    for (int d = 0; d < 256; ++d) total += h[d];
    if (total < need) {
      // fewer candidates than asked for (only possible at the first pass): take them all
      topk[4 * s + 3] = 1ull;
    } else {
      unsigned long long cum = 0ull;
      for (int d = 255; d >= 0; --d) {
        if (cum + h[d] >= need) {
          topk[4 * s + 0] |= (unsigned long long)d << shift;
          topk[4 * s + 1] |= 255ull << shift;
          topk[4 * s + 2] = need - cum;
          break;
        }
        cum += h[d];
      }
    }
  }
  for (int d = 0; d < 256; ++d) h[d] = 0ull;
}

template <int D>
__device__ __forceinline__ void topk_class(unsigned long long k, const unsigned long long* t, bool& gt,
                                           bool& eq) {
  if (t[3] != 0ull) {  // take all
    gt = k != 0ull;
    eq = false;
  } else {
    gt = k > t[0];
    eq = k == t[0] && k != 0ull && t[2] > 0ull;
  }
}

template <int D>
__global__ void __launch_bounds__(NT) k_topk_count(const ShotDev* __restrict__ shots, int nshots,
                                                   const double2* __restrict__ psi,
                                                   const unsigned long long* __restrict__ topk,
                                                   int64_t* blk_gt, int64_t* blk_eq) {
  const int64_t base = (int64_t)blockIdx.x * kScanBlock;
  const int s = shot_of_block(shots, nshots, base);
  const ShotDev& sh = shots[s];
  int cg = 0, ce = 0;
  for (int i = 0; i < PER; ++i) {
    bool gt, eq;
    topk_class<D>(topk_key<D>(sh, psi, base + threadIdx.x + NT * i), topk + 4 * s, gt, eq);
    cg += gt ? 1 : 0;
    ce += eq ? 1 : 0;
  }
  __shared__ int red[2][NT / 32];
  for (int off = 16; off > 0; off >>= 1) {
    cg += __shfl_xor_sync(0xffffffffu, cg, off);
    ce += __shfl_xor_sync(0xffffffffu, ce, off);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = cg;
    red[1][threadIdx.x >> 5] = ce;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int a = 0, b = 0;
    for (int w = 0; w < NT / 32; ++w) {
      a += red[0][w];
      b += red[1][w];
    }
    blk_gt[blockIdx.x] = a;
    blk_eq[blockIdx.x] = b;
  }
}

// Per shot (one thread for all shots, in order): count = #(key > K) + min(#(key == K),
// to_take), the Gaussian segment offsets and counts.
__global__ void k_topk_counts(ShotDev* shots, int nshots, const int64_t* blk_gt, const int64_t* blk_eq,
                              const int64_t* blk_first, const unsigned long long* topk, int64_t* counts) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  int64_t off = 0;
  for (int s = 0; s < nshots; ++s) {
    const int64_t gt = blk_gt[blk_first[s + 1]] - blk_gt[blk_first[s]];
    const int64_t eq = blk_eq[blk_first[s + 1]] - blk_eq[blk_first[s]];
    const int64_t take = topk[4 * s + 3] ? 0 : (int64_t)topk[4 * s + 2];
    const int64_t c = gt + (eq < take ? eq : take);
    shots[s].g_off = off;
    shots[s].g_cnt = c;
    counts[s] = c;
    off += c;
  }
}

template <int D>
__global__ void __launch_bounds__(NT) k_topk_scatter(const ShotDev* __restrict__ shots, int nshots,
                                                     const double2* __restrict__ psi,
                                                     const unsigned long long* __restrict__ topk,
                                                     const int64_t* __restrict__ blk_gt,
                                                     const int64_t* __restrict__ blk_eq,
                                                     const int64_t* __restrict__ blk_first,
                                                     int32_t* gshot, int64_t* gq, int32_t* gp,
                                                     double2* gpsi, const double2* __restrict__ psi_f1,
                                                     double2* gpsi_f1, int64_t cap) {
  const int64_t base = (int64_t)blockIdx.x * kScanBlock;
  const int s = shot_of_block(shots, nshots, base);
  const ShotDev& sh = shots[s];
  const unsigned long long* t = topk + 4 * s;
  const int64_t take = t[3] ? 0 : (int64_t)t[2];
  const int64_t e0 = base + (int64_t)threadIdx.x * PER;
  bool g[PER], q[PER];
  int cg = 0, ce = 0;
  for (int i = 0; i < PER; ++i) {
    topk_class<D>(topk_key<D>(sh, psi, e0 + i), t, g[i], q[i]);
    cg += g[i] ? 1 : 0;
    ce += q[i] ? 1 : 0;
  }
  // exclusive ranks of this thread's entries within the block (thread order = entry order)
  __shared__ int wt[2][NT / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int xg = cg, xe = ce;
  for (int off = 1; off < 32; off <<= 1) {
    const int yg = __shfl_up_sync(0xffffffffu, xg, off), ye = __shfl_up_sync(0xffffffffu, xe, off);
    if (lane >= off) {
      xg += yg;
      xe += ye;
    }
  }
  if (lane == 31) {
    wt[0][warp] = xg;
    wt[1][warp] = xe;
  }
  __syncthreads();
  int bg = 0, be = 0;
  for (int w = 0; w < warp; ++w) {
    bg += wt[0][w];
    be += wt[1][w];
  }
  int64_t gt_before = blk_gt[blockIdx.x] - blk_gt[blk_first[s]] + bg + (xg - cg);
  int64_t eq_before = blk_eq[blockIdx.x] - blk_eq[blk_first[s]] + be + (xe - ce);
  for (int i = 0; i < PER; ++i) {
    bool keep = g[i];
    if (q[i]) keep = eq_before < take;
    const int64_t pos = sh.g_off + gt_before + (eq_before < take ? eq_before : take);
    if (keep && pos < cap) {
      const int64_t loc = e0 + i - sh.psi_off;
      const int64_t ql = loc / sh.np, jp = loc - ql * sh.np;
      gshot[pos] = s;
      gq[pos] = q_flat<D>(sh, ql);
      gp[pos] = (int32_t)jp;
      gpsi[pos] = psi[e0 + i];
      gpsi_f1[pos] = psi_f1[e0 + i];
    }
    if (g[i]) ++gt_before;
    if (q[i]) ++eq_before;
  }
}

// Pipeline graph (one thread): clamp every shot's segment to the Gaussian capacity
// (flagging kStatusCapacity if it had to), and write the total G and the work-order
// multiplier for the ray kernel.
__global__ void k_counts_finish(ShotDev* shots, int nshots, int64_t cap, int64_t* gm, int* status) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  int64_t G = 0;
  bool clamped = false;
  for (int s = 0; s < nshots; ++s) {
    const int64_t off = shots[s].g_off, cnt = shots[s].g_cnt;
    const int64_t room = cap - off > 0 ? cap - off : 0;
    const int64_t c = cnt < room ? cnt : room;
    clamped = clamped || c != cnt;
    shots[s].g_cnt = c;
    G = off + c > G ? off + c : G;
  }
  if (clamped) atomicOr(status, kStatusCapacity);
  gm[0] = G;
  gm[1] = (int64_t)work_order_mult_of(G);
}

// Per-shot Gaussian segment [g_off, g_off + g_cnt) from the scanned block offsets.
__global__ void k_select_counts(ShotDev* shots, int nshots, const int64_t* blk,
                                const int64_t* blk_first, int64_t* counts) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nshots) return;
  int64_t a = blk[blk_first[s]], b = blk[blk_first[s + 1]];
  shots[s].g_off = a;
  shots[s].g_cnt = b - a;
  counts[s] = b - a;
}

}  // namespace

// N-largest: radix select of the cut key, then the two block counts, their scans and
// the per-shot counts and offsets.
static cudaError_t launch_topk_count(fga_plan_s* p) {
  const int D = p->grid.dim;
  const unsigned sb = (unsigned)((p->nshots + 127) / 128);
  k_topk_init<<<sb, 128, 0, p->stream>>>(p->d_topk, p->nshots, (long long)p->keep_n);
  cudaError_t e = cudaMemsetAsync(p->d_topk_hist, 0, sizeof(unsigned long long) * 256 * p->nshots,
                                  p->stream);
  if (e != cudaSuccess) return e;
  auto hist = D == 1 ? k_topk_hist<1> : (D == 2 ? k_topk_hist<2> : k_topk_hist<3>);
  for (int pass = 0; pass < 8; ++pass) {
    const int shift = 56 - 8 * pass;
    hist<<<(unsigned)p->nblocks, NT, 0, p->stream>>>(p->d_shots, p->nshots, p->d_psi, p->d_topk, shift,
                                                     p->d_topk_hist);
    k_topk_pick<<<sb, 128, 0, p->stream>>>(p->d_topk, p->d_topk_hist, p->nshots, shift);
  }
  auto count = D == 1 ? k_topk_count<1> : (D == 2 ? k_topk_count<2> : k_topk_count<3>);
  count<<<(unsigned)p->nblocks, NT, 0, p->stream>>>(p->d_shots, p->nshots, p->d_psi, p->d_topk, p->d_blk,
                                                    p->d_blk_eq);
  k_scan_exclusive<<<1, 1024, 0, p->stream>>>(p->d_blk, p->nblocks);
  k_scan_exclusive<<<1, 1024, 0, p->stream>>>(p->d_blk_eq, p->nblocks);
  k_topk_counts<<<1, 1, 0, p->stream>>>(p->d_shots, p->nshots, p->d_blk, p->d_blk_eq, p->d_blk_first,
                                        p->d_topk, p->d_counts);
  p->launches += 2 + 16 + 4;
  return cudaGetLastError();
}

// Pass 1 + scan: block counts and offsets; per-shot counts to p->d_counts.
cudaError_t launch_select_count(fga_plan_s* p) {
  if (p->nblocks == 0) return cudaSuccess;
  if (p->keep_n > 0) return launch_topk_count(p);
  const int64_t* d_blk_first = p->d_blk_first;
  double tau2 = p->tau * p->tau;
  auto count = p->grid.dim == 1 ? k_select_count<1> : (p->grid.dim == 2 ? k_select_count<2>
                                                                         : k_select_count<3>);
  count<<<(unsigned)p->nblocks, NT, 0, p->stream>>>(p->d_shots, p->nshots, p->d_psi, p->d_max2, tau2,
                                                    p->d_blk);
  k_scan_exclusive<<<1, 1024, 0, p->stream>>>(p->d_blk, p->nblocks);
  k_select_counts<<<(p->nshots + 127) / 128, 128, 0, p->stream>>>(p->d_shots, p->nshots, p->d_blk,
                                                                  d_blk_first, p->d_counts);
  p->launches += 3;
  return cudaGetLastError();
}

cudaError_t launch_select(fga_plan_s* p) {
  double tau2 = p->tau * p->tau;
  if (p->nblocks == 0) return cudaSuccess;
  if (p->keep_n > 0) {
    const int D = p->grid.dim;
    auto scatter = D == 1 ? k_topk_scatter<1> : (D == 2 ? k_topk_scatter<2> : k_topk_scatter<3>);
    scatter<<<(unsigned)p->nblocks, NT, 0, p->stream>>>(p->d_shots, p->nshots, p->d_psi, p->d_topk,
                                                        p->d_blk, p->d_blk_eq, p->d_blk_first,
                                                        p->d_gshot, p->d_gq, p->d_gp, p->d_gpsi,
                                                        p->d_psi_f1, p->d_gpsi_f1, (int64_t)p->g_cap);
    p->launches += 1;
    return cudaGetLastError();
  }
  auto scatter = p->grid.dim == 1 ? k_select_scatter<1>
                                   : (p->grid.dim == 2 ? k_select_scatter<2> : k_select_scatter<3>);
  scatter<<<(unsigned)p->nblocks, NT, 0, p->stream>>>(p->d_shots, p->nshots, p->d_psi, p->d_max2,
                                                      tau2, p->d_blk, p->d_gshot, p->d_gq, p->d_gp,
                                                      p->d_gpsi, p->d_psi_f1, p->d_gpsi_f1,
                                                      (int64_t)p->g_cap);
  p->launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_counts_finish(fga_plan_s* p) {
  k_counts_finish<<<1, 1, 0, p->stream>>>(p->d_shots, p->nshots, (int64_t)p->g_cap, p->d_gm,
                                          p->d_status);
  p->launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_scan_on(cudaStream_t stream, int64_t* a, int64_t n) {
  k_scan_exclusive<<<1, 1024, 0, stream>>>(a, n);
  return cudaGetLastError();
}

cudaError_t launch_scan(fga_plan_s* p, int64_t* a, int64_t n) {
  k_scan_exclusive<<<1, 1024, 0, p->stream>>>(a, n);
  p->launches += 1;
  return cudaGetLastError();
}

}  // namespace fga
