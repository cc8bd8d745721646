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

// Position of a compaction block's first entry in its shot's segment: q row ql0 and p
// index r0 (one 64-bit division per block, by thread 0); entry k of the block is then
// q row ql0 + (r0 + k) / np and p index (r0 + k) mod np, found with fast_div. Thread 0
// also forms the block's threshold thr2 = tau2 max2 and its integer screen: a pair with
// |Re| < T and |Im| < T, T = sqrt(thr2 / 2) (1 - 2^-40), has |psi|^2 < thr2 even after
// the rounding of its FP64 square, and the comparisons of non-negative floating-point
// numbers are those of their bit patterns (Td, Tf: T as FP64 and, rounded down, FP32;
// 0 where thr2 is NaN or infinite, so that nothing is screened out). FP64 instructions
// are scarce on this part (two per clock per SM), so none is spent per thread or per
// rejected entry.
struct BlockPos {
  int64_t loc0, ql0;
  uint32_t r0;
  double thr2;
  unsigned long long Td;
  uint32_t Tf;
};
__device__ __forceinline__ BlockPos block_pos(const ShotDev& sh, int64_t base, double tau2,
                                              const unsigned long long* max2, int s) {
  __shared__ int64_t s_ql0;
  __shared__ uint32_t s_r0, s_Tf;
  __shared__ double s_thr2;
  __shared__ unsigned long long s_Td;
  const int64_t loc0 = base - sh.psi_off;
  if (threadIdx.x == 0) {
    s_ql0 = loc0 / sh.np;
    s_r0 = (uint32_t)(loc0 - s_ql0 * sh.np);
    const double thr2 = max2 ? tau2 * __longlong_as_double((long long)max2[s]) : 0.0;
    const double T = thr2 >= 0.0 && thr2 < INFINITY ? sqrt(0.5 * thr2) * (1.0 - 0x1p-40) : 0.0;
    s_thr2 = thr2;
    s_Td = (unsigned long long)__double_as_longlong(T);
    s_Tf = __float_as_uint(__double2float_rd(T));
  }
  __syncthreads();
  return BlockPos{loc0, s_ql0, s_r0, s_thr2, s_Td, s_Tf};
}
__device__ __forceinline__ bool below(const BlockPos& b, double2 v) {
  const unsigned long long ax = (unsigned long long)__double_as_longlong(v.x) & 0x7fffffffffffffffull;
  const unsigned long long ay = (unsigned long long)__double_as_longlong(v.y) & 0x7fffffffffffffffull;
  return ax < b.Td && ay < b.Td;
}
__device__ __forceinline__ bool below(const BlockPos& b, float2 v) {
  return (__float_as_uint(v.x) & 0x7fffffffu) < b.Tf && (__float_as_uint(v.y) & 0x7fffffffu) < b.Tf;
}

// The q row and p index (flat and per axis) of one entry, stepped along the segment.
struct PCur {
  int64_t ql;
  uint32_t jp, j0, j1, j2;
};
// Entry k of the block (the p index split with fast_div: once per thread, not per entry).
template <int D>
__device__ __forceinline__ PCur pcur_at(const ShotDev& sh, const BlockPos& b, int k) {
  PCur c;
  const uint32_t x = b.r0 + (uint32_t)k;
  const uint32_t qd = fast_div(sh.fd_np, x);
  c.jp = x - qd * (uint32_t)sh.np;
  c.ql = b.ql0 + qd;
  c.j1 = c.j2 = 0u;
  if constexpr (D == 1) {
    c.j0 = c.jp;
  } else if constexpr (D == 2) {
    c.j0 = fast_div(sh.fd_nbl, c.jp);
    c.j1 = c.jp - c.j0 * (uint32_t)sh.nb[1];
  } else {
    c.j0 = fast_div(sh.fd_nb12, c.jp);
    const uint32_t r = c.jp - c.j0 * ((uint32_t)sh.nb[1] * (uint32_t)sh.nb[2]);
    c.j1 = fast_div(sh.fd_nbl, r);
    c.j2 = r - c.j1 * (uint32_t)sh.nb[2];
  }
  return c;
}
// The next entry (p index + 1, carried into the axes and the q row).
template <int D>
__device__ __forceinline__ void pcur_next(const ShotDev& sh, PCur& c) {
  ++c.jp;
  bool wrap;
  if constexpr (D == 1) {
    wrap = ++c.j0 == (uint32_t)sh.nb[0];
  } else if constexpr (D == 2) {
    wrap = false;
    if (++c.j1 == (uint32_t)sh.nb[1]) {
      c.j1 = 0u;
      wrap = ++c.j0 == (uint32_t)sh.nb[0];
    }
  } else {
    wrap = false;
    if (++c.j2 == (uint32_t)sh.nb[2]) {
      c.j2 = 0u;
      if (++c.j1 == (uint32_t)sh.nb[1]) {
        c.j1 = 0u;
        wrap = ++c.j0 == (uint32_t)sh.nb[0];
      }
    }
  }
  if (wrap) {
    c.j0 = 0u;
    c.jp = 0u;
    ++c.ql;
  }
}
// Valid p: the Nyquist index of an axis and p = 0 are left out (as in the FBI).
template <int D>
__device__ __forceinline__ bool pcur_valid(const ShotDev& sh, const PCur& c) {
  if constexpr (D == 1) {
    return c.j0 != 0u && c.j0 != (uint32_t)(sh.nb[0] / 2);
  } else if constexpr (D == 2) {
    return c.j0 != 0u && c.j1 != 0u &&
           !(c.j0 == (uint32_t)(sh.nb[0] / 2) && c.j1 == (uint32_t)(sh.nb[1] / 2));
  } else {
    return c.j0 != 0u && c.j1 != 0u && c.j2 != 0u &&
           !(c.j0 == (uint32_t)(sh.nb[0] / 2) && c.j1 == (uint32_t)(sh.nb[1] / 2) &&
             c.j2 == (uint32_t)(sh.nb[2] / 2));
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

// psi is stored as FP64 pairs, or (mixed precision) as FP32 pairs that are widened
// exactly: every decision below is taken on the FP64 values either way.
__device__ __forceinline__ double2 widen2(double2 v) { return v; }
__device__ __forceinline__ double2 widen2(float2 v) { return make_double2((double)v.x, (double)v.y); }

// The exact test |psi|^2 >= thr2 in FP64, out of line: inlined, the compiler evaluates
// it (widening and all) for every entry instead of branching around it for the entries
// the screen rejects.
template <typename V>
__device__ __noinline__ bool above_exact(V v, double thr2) {
  return abs2_rn(widen2(v)) >= thr2;
}

// Entry k of the block (at cursor c): kept?
template <int D, typename V>
__device__ __forceinline__ bool keep(const ShotDev& sh, const BlockPos& b, const PCur& c, const V* psi,
                                     int64_t base, int k) {
  if (b.loc0 + k >= sh.psi_len || !pcur_valid<D>(sh, c)) return false;
  const V v = psi[base + k];
  if (below(b, v)) return false;  // |psi|^2 < thr2, decided without an FP64 instruction
  return above_exact(v, b.thr2);
}

template <int D, typename V>
__global__ void __launch_bounds__(NT) k_select_count(const ShotDev* __restrict__ shots, int nshots,
                                                     const V* __restrict__ psi,
                                                     const unsigned long long* __restrict__ max2,
                                                     double tau2, int64_t* blk) {
  int64_t base = (int64_t)blockIdx.x * kScanBlock;
  int s = shot_of_block(shots, nshots, base);
  const ShotDev& sh = shots[s];
  const BlockPos b = block_pos(sh, base, tau2, max2, s);
  // thread t counts the PER consecutive entries from PER t
  const int k0 = threadIdx.x * PER;
  PCur pc = pcur_at<D>(sh, b, k0);
  int c = 0;
  for (int i = 0; i < PER; ++i) {
    c += keep<D>(sh, b, pc, psi, base, k0 + i) ? 1 : 0;
    pcur_next<D>(sh, pc);
  }
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

template <int D, typename V>
__global__ void __launch_bounds__(NT) k_select_scatter(const ShotDev* __restrict__ shots, int nshots,
                                                       const V* __restrict__ psi,
                                                       const unsigned long long* __restrict__ max2,
                                                       double tau2, const int64_t* __restrict__ blk,
                                                       int32_t* gshot, int64_t* gq, int32_t* gp,
                                                       double2* gpsi, const V* __restrict__ psi_f1,
                                                       double2* gpsi_f1, int64_t cap) {
  int64_t base = (int64_t)blockIdx.x * kScanBlock;
  int s = shot_of_block(shots, nshots, base);
  const ShotDev& sh = shots[s];
  const BlockPos b = block_pos(sh, base, tau2, max2, s);
  // thread t owns PER consecutive entries, so the block order is the entry order
  const int k0 = threadIdx.x * PER;
  int64_t e0 = base + k0;
  const PCur pc0 = pcur_at<D>(sh, b, k0);
  PCur pc = pc0;
  bool f[PER];
  int c = 0;
  for (int i = 0; i < PER; ++i) {
    f[i] = keep<D>(sh, b, pc, psi, base, k0 + i);
    c += f[i] ? 1 : 0;
    pcur_next<D>(sh, pc);
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
  pc = pc0;
  for (int i = 0; i < PER; ++i, pcur_next<D>(sh, pc)) {
    if (!f[i] || pos >= cap) continue;  // beyond the capacity: k_counts_finish flags it
    const int64_t qflat = q_flat<D>(sh, pc.ql);
    gshot[pos] = s;
    gq[pos] = qflat;
    gp[pos] = (int32_t)pc.jp;
    gpsi[pos] = widen2(psi[e0 + i]);
    gpsi_f1[pos] = widen2(psi_f1[e0 + i]);
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
template <int D, typename V>
__device__ __forceinline__ unsigned long long topk_key(const ShotDev& sh, const BlockPos& b, const PCur& c,
                                                       const V* psi, int64_t base, int k) {
  if (b.loc0 + k >= sh.psi_len || !pcur_valid<D>(sh, c)) return 0ull;
  const double2 v = widen2(psi[base + k]);
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

template <int D, typename V>
__global__ void __launch_bounds__(NT) k_topk_hist(const ShotDev* __restrict__ shots, int nshots,
                                                  const V* __restrict__ psi,
                                                  const unsigned long long* __restrict__ topk,
                                                  int shift, unsigned long long* hist) {
  __shared__ unsigned int h[256];
  for (int i = threadIdx.x; i < 256; i += NT) h[i] = 0u;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kScanBlock;
  const int s = shot_of_block(shots, nshots, base);
  const ShotDev& sh = shots[s];
  const unsigned long long prefix = topk[4 * s], mask = topk[4 * s + 1];
  const BlockPos b = block_pos(sh, base, 0.0, nullptr, s);
  const int k0 = threadIdx.x * PER;
  PCur pc = pcur_at<D>(sh, b, k0);
  for (int i = 0; i < PER; ++i, pcur_next<D>(sh, pc)) {
    const unsigned long long k = topk_key<D>(sh, b, pc, psi, base, k0 + i);
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

template <int D, typename V>
__global__ void __launch_bounds__(NT) k_topk_count(const ShotDev* __restrict__ shots, int nshots,
                                                   const V* __restrict__ psi,
                                                   const unsigned long long* __restrict__ topk,
                                                   int64_t* blk_gt, int64_t* blk_eq) {
  const int64_t base = (int64_t)blockIdx.x * kScanBlock;
  const int s = shot_of_block(shots, nshots, base);
  const ShotDev& sh = shots[s];
  const BlockPos b = block_pos(sh, base, 0.0, nullptr, s);
  const int k0 = threadIdx.x * PER;
  PCur pc = pcur_at<D>(sh, b, k0);
  int cg = 0, ce = 0;
  for (int i = 0; i < PER; ++i, pcur_next<D>(sh, pc)) {
    bool gt, eq;
    topk_class<D>(topk_key<D>(sh, b, pc, psi, base, k0 + i), topk + 4 * s, gt, eq);
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

template <int D, typename V>
__global__ void __launch_bounds__(NT) k_topk_scatter(const ShotDev* __restrict__ shots, int nshots,
                                                     const V* __restrict__ psi,
                                                     const unsigned long long* __restrict__ topk,
                                                     const int64_t* __restrict__ blk_gt,
                                                     const int64_t* __restrict__ blk_eq,
                                                     const int64_t* __restrict__ blk_first,
                                                     int32_t* gshot, int64_t* gq, int32_t* gp,
                                                     double2* gpsi, const V* __restrict__ psi_f1,
                                                     double2* gpsi_f1, int64_t cap) {
  const int64_t base = (int64_t)blockIdx.x * kScanBlock;
  const int s = shot_of_block(shots, nshots, base);
  const ShotDev& sh = shots[s];
  const unsigned long long* t = topk + 4 * s;
  const int64_t take = t[3] ? 0 : (int64_t)t[2];
  const BlockPos b = block_pos(sh, base, 0.0, nullptr, s);
  const int k0 = threadIdx.x * PER;
  const int64_t e0 = base + k0;
  const PCur pc0 = pcur_at<D>(sh, b, k0);
  PCur pc = pc0;
  bool g[PER], q[PER];
  int cg = 0, ce = 0;
  for (int i = 0; i < PER; ++i, pcur_next<D>(sh, pc)) {
    topk_class<D>(topk_key<D>(sh, b, pc, psi, base, k0 + i), t, g[i], q[i]);
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
  pc = pc0;
  for (int i = 0; i < PER; ++i, pcur_next<D>(sh, pc)) {
    bool keep = g[i];
    if (q[i]) keep = eq_before < take;
    const int64_t pos = sh.g_off + gt_before + (eq_before < take ? eq_before : take);
    if (keep && pos < cap) {
      gshot[pos] = s;
      gq[pos] = q_flat<D>(sh, pc.ql);
      gp[pos] = (int32_t)pc.jp;
      gpsi[pos] = widen2(psi[e0 + i]);
      gpsi_f1[pos] = widen2(psi_f1[e0 + i]);
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
// the per-shot counts and offsets. V: the element type psi is stored in.
template <typename V>
static cudaError_t launch_topk_count(fga_plan_s* p, const V* psi) {
  const int D = p->grid.dim;
  const unsigned sb = (unsigned)((p->nshots + 127) / 128);
  k_topk_init<<<sb, 128, 0, p->stream>>>(p->d_topk, p->nshots, (long long)p->keep_n);
  cudaError_t e = cudaMemsetAsync(p->d_topk_hist, 0, sizeof(unsigned long long) * 256 * p->nshots,
                                  p->stream);
  if (e != cudaSuccess) return e;
  auto hist = D == 1 ? k_topk_hist<1, V> : (D == 2 ? k_topk_hist<2, V> : k_topk_hist<3, V>);
  for (int pass = 0; pass < 8; ++pass) {
    const int shift = 56 - 8 * pass;
    hist<<<(unsigned)p->nblocks, NT, 0, p->stream>>>(p->d_shots, p->nshots, psi, p->d_topk, shift,
                                                     p->d_topk_hist);
    k_topk_pick<<<sb, 128, 0, p->stream>>>(p->d_topk, p->d_topk_hist, p->nshots, shift);
  }
  auto count = D == 1 ? k_topk_count<1, V> : (D == 2 ? k_topk_count<2, V> : k_topk_count<3, V>);
  count<<<(unsigned)p->nblocks, NT, 0, p->stream>>>(p->d_shots, p->nshots, psi, p->d_topk, p->d_blk,
                                                    p->d_blk_eq);
  k_scan_exclusive<<<1, 1024, 0, p->stream>>>(p->d_blk, p->nblocks);
  k_scan_exclusive<<<1, 1024, 0, p->stream>>>(p->d_blk_eq, p->nblocks);
  k_topk_counts<<<1, 1, 0, p->stream>>>(p->d_shots, p->nshots, p->d_blk, p->d_blk_eq, p->d_blk_first,
                                        p->d_topk, p->d_counts);
  p->launches += 2 + 16 + 4;
  return cudaGetLastError();
}

template <typename V>
static cudaError_t select_count(fga_plan_s* p, const V* psi) {
  if (p->keep_n > 0) return launch_topk_count(p, psi);
  const int64_t* d_blk_first = p->d_blk_first;
  double tau2 = p->tau * p->tau;
  auto count = p->grid.dim == 1 ? k_select_count<1, V>
                                : (p->grid.dim == 2 ? k_select_count<2, V> : k_select_count<3, V>);
  count<<<(unsigned)p->nblocks, NT, 0, p->stream>>>(p->d_shots, p->nshots, psi, p->d_max2, tau2,
                                                    p->d_blk);
  k_scan_exclusive<<<1, 1024, 0, p->stream>>>(p->d_blk, p->nblocks);
  k_select_counts<<<(p->nshots + 127) / 128, 128, 0, p->stream>>>(p->d_shots, p->nshots, p->d_blk,
                                                                  d_blk_first, p->d_counts);
  p->launches += 3;
  return cudaGetLastError();
}

template <typename V>
static cudaError_t select_scatter(fga_plan_s* p, const V* psi, const V* psi_f1) {
  double tau2 = p->tau * p->tau;
  const int D = p->grid.dim;
  if (p->keep_n > 0) {
    auto scatter = D == 1 ? k_topk_scatter<1, V> : (D == 2 ? k_topk_scatter<2, V> : k_topk_scatter<3, V>);
    scatter<<<(unsigned)p->nblocks, NT, 0, p->stream>>>(p->d_shots, p->nshots, psi, p->d_topk,
                                                        p->d_blk, p->d_blk_eq, p->d_blk_first,
                                                        p->d_gshot, p->d_gq, p->d_gp, p->d_gpsi,
                                                        psi_f1, p->d_gpsi_f1, (int64_t)p->g_cap);
    p->launches += 1;
    return cudaGetLastError();
  }
  auto scatter = D == 1 ? k_select_scatter<1, V> : (D == 2 ? k_select_scatter<2, V> : k_select_scatter<3, V>);
  scatter<<<(unsigned)p->nblocks, NT, 0, p->stream>>>(p->d_shots, p->nshots, psi, p->d_max2, tau2,
                                                      p->d_blk, p->d_gshot, p->d_gq, p->d_gp,
                                                      p->d_gpsi, psi_f1, p->d_gpsi_f1,
                                                      (int64_t)p->g_cap);
  p->launches += 1;
  return cudaGetLastError();
}

// Pass 1 + scan: block counts and offsets; per-shot counts to p->d_counts.
cudaError_t launch_select_count(fga_plan_s* p) {
  if (p->nblocks == 0) return cudaSuccess;
  if (psi_is_f32(p)) return select_count(p, reinterpret_cast<const float2*>(p->d_psi));
  return select_count(p, static_cast<const double2*>(p->d_psi));
}

cudaError_t launch_select(fga_plan_s* p) {
  if (p->nblocks == 0) return cudaSuccess;
  if (psi_is_f32(p))
    return select_scatter(p, reinterpret_cast<const float2*>(p->d_psi),
                          reinterpret_cast<const float2*>(p->d_psi_f1));
  return select_scatter(p, static_cast<const double2*>(p->d_psi), static_cast<const double2*>(p->d_psi_f1));
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
