// Mixed-precision reconstruction on the tensor cores (2D, open axes).
//
// For one output tile of 128 x 128 points and one segment of its Gaussian list, the
// real part of the Gaussian sum (Eq. recons) is a real GEMM over the Gaussian index:
//   u[x][z] = sum_g Re(X_g(x) Z_g(z)) = sum_k A[x][k] B[z][k],
//   A[x][2g] = Re X_g(x), A[x][2g+1] = -Im X_g(x), B[z][2g] = Re Z_g(z), B[z][2g+1] = Im Z_g(z),
// where X_g carries the Gaussian's coefficient. Each factor is split into a TF32 head
// and an FP32 tail (v = hi + lo), and the three products hi*hi + hi*lo + lo*hi are
// accumulated in FP32 in tensor memory by tcgen05.mma (kind::tf32, M = N = 128,
// K = 8 per instruction), so each product carries about 21 significant bits.
//
// Precision policy: the phase P (x - Q)/eps is anchored in FP64 at the first point of
// each 16-point run and carried as a 32-bit fixed-point fraction of a turn (exact
// increments modulo 2 pi), so the FP32 sine/cosine see an argument in [-pi, pi) that is
// accurate to about 1e-7 rad; the Gaussian envelope exp(-d^2/(2 eps)) is FP32. The
// partial tile of each (tile, segment) work item is FP32 and the segments are summed in
// FP64 in a fixed order.
#include <algorithm>

#include "fga_internal.cuh"
#include "fga_tc.cuh"
#include "fga_tiles.cuh"

namespace fga {

namespace {

constexpr int TM = 128;       // tile edge (x = GEMM M, z = GEMM N)
constexpr int CHG = 16;       // Gaussians per chunk -> K = 32
constexpr int KC = 2 * CHG;   // GEMM K per chunk
constexpr int KB = KC / 4;    // 16-byte core matrices along K (tf32: 4 per core row)
constexpr int64_t SEGM = 2048;  // default Gaussians per work item
constexpr int NTC = 256;      // threads per CTA: 0..127 make A (x) rows, 128..255 B (z) rows
constexpr uint32_t kMaxTries = 1u << 22;
// core-matrix (8 rows x 16 bytes) strides of the K-major operand tiles
constexpr uint32_t kLBO = 128;       // next core matrix along K
constexpr uint32_t kSBO = KB * 128;  // next 8-row group along M / N
constexpr size_t kOperandBytes = (size_t)TM * KC * sizeof(float);  // 16 KiB
constexpr size_t kBufBytes = 4 * kOperandBytes;                     // A, B heads and tails
constexpr size_t kSmemBytes = kBufBytes + 64;                       // operands, barrier

__device__ __forceinline__ int core_offset(int row, int k) {
  return (((row >> 3) * KB + (k >> 2)) * 8 + (row & 7)) * 4 + (k & 3);
}

__device__ __forceinline__ float tf32_head(float v) {
  return __uint_as_float(__float_as_uint(v) & 0xFFFFE000u);
}

// What a Gaussian's factors on every tile need, per axis, made once per Gaussian in FP64
// (k_anchor_tc) so that the gather's chunk loop runs no FP64 instruction: with the grid
// index j of a point, x_j = o + j h,
//   phase  P (x_j - Q)/eps / (2 pi) = ub + j ud  (turns, 64-bit fixed point: exact
//          wrap-around sums; the rounding of ud times j stays below 2^-32 turns over the
//          grid),
//   offset (x_j - Q)/h = (j - iq) - fq  (rows; iq = floor((Q - o)/h), fq in [0, 1)),
//   window j in [glo, ghi] where |x_j - Q| <= kappa sqrt(eps).
struct GaussAnchor {
  unsigned long long ub[2], ud[2];
  int iq[2], glo[2], ghi[2];
  float fq[2];
  float2 cf;  // the Gaussian's coefficient (carried by the x factor)
};

// One Gaussian on one axis of one tile (first grid index a): the phase at the tile's first
// point and per point (32-bit turn fractions), the offset of the first point in rows,
// and the rows of the window.
struct Anchor {
  uint32_t u0, ud;
  float d0;   // (x_a - Q)/h
  int lo, hi; // rows inside the window (empty when lo > hi)
  float2 cf;  // coefficient (x axis) or 1 (z axis)
};

__device__ __forceinline__ Anchor tile_anchor(const GaussAnchor& ga, int axis, int64_t a) {
  Anchor an;
  const unsigned long long u = ga.ub[axis] + (unsigned long long)a * ga.ud[axis];
  an.u0 = (uint32_t)((u + 0x80000000ull) >> 32);
  an.ud = (uint32_t)((ga.ud[axis] + 0x80000000ull) >> 32);
  an.d0 = (float)(int)(a - ga.iq[axis]) - ga.fq[axis];
  const int64_t lo = ga.glo[axis] - a, hi = ga.ghi[axis] - a;
  an.lo = lo < 0 ? 0 : (lo > TM ? TM : (int)lo);
  an.hi = hi > TM - 1 ? TM - 1 : (hi < -1 ? -1 : (int)hi);
  an.cf = axis == 0 ? ga.cf : make_float2(1.f, 0.f);
  return an;
}

__device__ __forceinline__ Anchor make_empty_anchor() {
  Anchor an;
  an.u0 = an.ud = 0u;
  an.d0 = 0.f;
  an.lo = 1;
  an.hi = 0;
  an.cf = make_float2(0.f, 0.f);
  return an;
}

// Factor of a Gaussian at row r: cf * exp(i phase - d^2/(2 eps)) (0 outside the window);
// kq = h^2 log2(e) / (2 eps) of the axis, so the envelope is 2^(-kq (d/h)^2).
__device__ __forceinline__ float2 row_factor(const Anchor& an, int r, float kq) {
  if (r < an.lo || r > an.hi) return make_float2(0.f, 0.f);
  const float ang_scale = 1.4629180792671596e-09f;  // 2 pi / 2^32
  const float dr = an.d0 + (float)r;
  float gs;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(gs) : "f"(-kq * dr * dr));
  float sn, cs;
  __sincosf((float)(int32_t)(an.u0 + (uint32_t)r * an.ud) * ang_scale, &sn, &cs);
  const float fr = gs * cs, fi = gs * sn;
  return make_float2(an.cf.x * fr - an.cf.y * fi, an.cf.x * fi + an.cf.y * fr);
}

// floor(t 2^k) as a two's-complement integer for |t| < 2^(63-k), from the bits of t
// (no FP64 instruction: FP64 issues at two operations per clock per SM on this part).
// t = M 2^E with M the 53-bit significand; the result is floor(M 2^(E+k)) for t >= 0 and
// -ceil(M 2^(E+k)) for t < 0, reduced modulo 2^64 (so that k = 64 gives the fraction of
// t in units of 2^-64, modulo 1).
__device__ __forceinline__ unsigned long long fixed_floor(double t, int k) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(t);
  const int e = (int)((b >> 52) & 0x7ffull);
  if (e == 0 || e == 0x7ff) return 0ull;  // zero, subnormal (below any unit used here), inf/NaN
  const unsigned long long M = (b & 0xfffffffffffffull) | (1ull << 52);
  const int sh = e - 1075 + k;
  unsigned long long F, rem = 0ull;
  if (sh >= 64) {
    F = 0ull;
  } else if (sh >= 0) {
    F = M << sh;
  } else if (sh > -64) {
    F = M >> (-sh);
    rem = M & ((1ull << (-sh)) - 1ull);
  } else {
    F = 0ull;
    rem = M;
  }
  if (b >> 63) F = 0ull - F - (rem != 0ull ? 1ull : 0ull);  // floor of the negative value
  return F;
}

// One thread per Gaussian: its GaussAnchor (once per Gaussian instead of once per
// (Gaussian, tile) in the gather). G from the device when gm is given (pipeline graph).
__global__ void k_anchor_tc(GridDev gd, const ShotDev* __restrict__ shots,
                            const int32_t* __restrict__ gshot, const double* __restrict__ state,
                            int64_t ld, const double2* __restrict__ coef, int64_t G,
                            const int64_t* __restrict__ gm, double kappa, GaussAnchor* __restrict__ out) {
  if (gm) G = gm[0];
  const double inv_two_pi = 0.15915494309189535;
  const long long lim = 1ll << 30;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < G;
       g += (int64_t)gridDim.x * blockDim.x) {
    const ShotDev& sh = shots[gshot[g]];
    const double ce = sh.inv_eps * inv_two_pi;
    GaussAnchor ga;
#pragma unroll
    for (int axis = 0; axis < 2; ++axis) {
      const double Q = state[axis * ld + g], P = state[(2 + axis) * ld + g];
      // phase at grid index 0 and per index, as 64-bit fractions of a turn
      ga.ub[axis] = fixed_floor(P * (gd.o[axis] - Q) * ce, 64);
      ga.ud[axis] = fixed_floor(P * (gd.h[axis] * ce), 64);
      // centre (Q - o)/h and half-width kappa sqrt(eps)/h in 32.32 fixed point; the window
      // is [ceil(u - w), floor(u + w)] (an empty window where it leaves +-2^30)
      const long long u = (long long)fixed_floor((Q - gd.o[axis]) * gd.inv_h[axis], 32);
      const long long wd = (long long)fixed_floor(kappa * sh.sqrt_eps * gd.inv_h[axis], 32);
      const long long glo = (u - wd + 0xffffffffll) >> 32, ghi = (u + wd) >> 32;
      if (glo > -lim && ghi < lim && (u >> 32) > -lim && (u >> 32) < lim) {
        ga.iq[axis] = (int)(u >> 32);
        ga.fq[axis] = (float)(uint32_t)(u & 0xffffffffll) * 2.3283064365386963e-10f;  // 2^-32
        ga.glo[axis] = (int)glo;
        ga.ghi[axis] = (int)ghi;
      } else {
        ga.iq[axis] = 0;
        ga.fq[axis] = 0.f;
        ga.glo[axis] = (int)lim;
        ga.ghi[axis] = -(int)lim;
      }
    }
    const double2 c = coef[g];
    ga.cf = make_float2((float)c.x, (float)c.y);
    out[g] = ga;
  }
}

__global__ void __launch_bounds__(NTC) k_gather_tc(GridDev gd, const ShotDev* __restrict__ shots,
                                                   int nshots, const GaussAnchor* __restrict__ ganc,
                                                   const int64_t* __restrict__ off,
                                                   const int32_t* __restrict__ list, int64_t list_cap,
                                                   const int64_t* __restrict__ seg_off, int64_t ntiles,
                                                   int64_t seg, float* __restrict__ partial,
                                                   int* status, uint32_t tries) {
  const int64_t w = blockIdx.x;
  if (w >= seg_off[ntiles]) return;  // uniform over the CTA
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + kBufBytes);
  uint32_t* tbase = reinterpret_cast<uint32_t*>(smem + kBufBytes + 16);
  __shared__ float kq_s[2];
  const int tid = threadIdx.x, warp = tid >> 5;
  const int axis = tid >> 7, row = tid & (TM - 1);  // this thread's operand (A: x, B: z) and row
  const int64_t t = tile_of_item(seg_off, ntiles, w);
  const int s = shot_of_tile(shots, nshots, t);
  const ShotDev& sh = shots[s];
  int64_t a[2], b[2];
  tile_box<2>(gd, sh, t - sh.tile_off, a, b);
  if (tid == 0) {
    tc::mbar_init(bar, 1);
    tc::fence_mbar_init();
    const double log2e = 1.4426950408889634;
    kq_s[0] = (float)(0.5 * gd.h[0] * gd.h[0] * sh.inv_eps * log2e);
    kq_s[1] = (float)(0.5 * gd.h[1] * gd.h[1] * sh.inv_eps * log2e);
  }
  if (warp == 0) {
    tc::tmem_alloc(tbase, TM);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tbase;
  const uint32_t idesc = tc::idesc_f32acc(tc::kFmtTF32, TM, TM);
  const int64_t l0 = min(off[t], list_cap) + (w - seg_off[t]) * seg;
  const int64_t l1 = min(min(off[t + 1], list_cap), l0 + seg);
  __shared__ Anchor anc[2][CHG];  // [axis][Gaussian of the chunk]
  const float kq = kq_s[axis];
  // One operand buffer (three CTAs share an SM, so one CTA's factors are made while
  // another's MMAs run); before it is overwritten the previous chunk's MMAs must be done.
  float* Ahi = reinterpret_cast<float*>(smem);
  float* Alo = Ahi + TM * KC;
  float* Bhi = Alo + TM * KC;
  float* Blo = Bhi + TM * KC;
  float* Ohi = axis == 0 ? Ahi : Bhi;  // this thread's operand
  float* Olo = axis == 0 ? Alo : Blo;
  uint32_t chunks = 0;
  bool gave_up = false;
  for (int64_t c0 = l0; c0 < l1; c0 += CHG) {
    const int nc = (int)((l1 - c0) < CHG ? (l1 - c0) : CHG);
    // anchors: thread gi of each half; every thread has passed the barrier after the
    // previous chunk's factors, so the anchors can be overwritten before the wait, whose
    // barrier publishes them
    if (row < CHG) anc[axis][row] = row < nc ? tile_anchor(ganc[list[c0 + row]], axis, a[axis])
                                             : make_empty_anchor();
    // the CTA gives up as a whole, with at most the previous commit outstanding
    bool waited = true;
    if (chunks > 0) waited = tc::mbar_wait_bounded(bar, (chunks - 1) & 1u, tries);
    if (!__syncthreads_and(waited)) {
      gave_up = true;
      break;
    }
    // operands: A[x][2g] = Re X_g, A[x][2g+1] = -Im X_g; B[z][2g] = Re Z_g, B[z][2g+1] =
    // Im Z_g. Thread (g, t8) of the half makes Gaussian g's factors on the 16 rows
    // t8 + 8j by the recurrence f(r + 8) = f(r) R(r), R(r + 8) = R(r) C: the first row of
    // the window in that class is evaluated directly (coefficient included), so no factor
    // starts from an underflowed value; the other rows cost a complex product each
    {
      const float sg = axis == 0 ? -1.f : 1.f;
      const int g = row >> 3, t8 = row & 7;
      const Anchor an = anc[axis][g];
      const int r0 = an.lo + ((t8 - an.lo) & 7);  // first row >= lo with row = t8 (mod 8)
      float2 f = row_factor(an, r0 <= an.hi ? r0 : an.lo, kq);  // zero for an empty window
      // R(r0) = exp(-kq (2 (d0 + r0) 8 + 64)) e^{i 8 ud 2 pi / 2^32} (kq already in log2 units)
      const float ang8 = (float)(int32_t)(8u * an.ud) * 1.4629180792671596e-09f;
      float s8, c8;
      __sincosf(ang8, &s8, &c8);
      float g8;
      asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(g8) : "f"(-kq * (16.0f * (an.d0 + (float)r0) + 64.0f)));
      float Rr = g8 * c8, Ri = g8 * s8, cc;
      asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(cc) : "f"(-128.0f * kq));  // C = exp(-kq 2 8^2)
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int r = t8 + 8 * j;
        const bool in = r >= r0 && r <= an.hi;
        const float vr = in ? f.x : 0.f, vi = in ? sg * f.y : 0.f;
        const int o = core_offset(r, 2 * g);
        const float hr = tf32_head(vr), hi = tf32_head(vi);
        *reinterpret_cast<float2*>(Ohi + o) = make_float2(hr, hi);
        *reinterpret_cast<float2*>(Olo + o) = make_float2(vr - hr, vi - hi);
        if (r >= r0) {  // advance to row r + 8
          const float nr = f.x * Rr - f.y * Ri, ni = f.x * Ri + f.y * Rr;
          f = make_float2(nr, ni);
          Rr *= cc;
          Ri *= cc;
        }
      }
    }
    tc::fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      const uint32_t ah = tc::smem_u32(Ahi), al = tc::smem_u32(Alo);
      const uint32_t bh = tc::smem_u32(Bhi), bl = tc::smem_u32(Blo);
#pragma unroll
      for (int ks = 0; ks < KC / 8; ++ks) {
        const uint32_t step = ks * 256;  // 8 tf32 of K = two core matrices
        tc::mma_tf32(tmem, tc::smem_desc(ah + step, kLBO, kSBO), tc::smem_desc(bh + step, kLBO, kSBO),
                     idesc, (chunks > 0 || ks > 0) ? 1u : 0u);
        tc::mma_tf32(tmem, tc::smem_desc(ah + step, kLBO, kSBO), tc::smem_desc(bl + step, kLBO, kSBO),
                     idesc, 1u);
        tc::mma_tf32(tmem, tc::smem_desc(al + step, kLBO, kSBO), tc::smem_desc(bh + step, kLBO, kSBO),
                     idesc, 1u);
      }
      tc::mma_commit(bar);
    }
    ++chunks;
  }
  bool done = true;
  if (!gave_up && chunks > 0) done = tc::mbar_wait_bounded(bar, (chunks - 1) & 1u, tries);
  const bool ok = __syncthreads_and(done) && !gave_up;
  if (!ok) {
    if (tid == 0) atomicOr(status, kStatusTimeout);
    // every earlier phase was observed, so only the last commit can be outstanding: wait
    // for it with the full budget before the accumulator's columns are released
    tc::mbar_wait_bounded(bar, (chunks - 1) & 1u, kMaxTries);
  }
  tc::fence_after_sync();
  // epilogue: warp w holds rows (x) 32 (w % 4) .. + 31, one row per thread, and takes
  // the 64 columns (z) of half w / 4
  const int quarter = warp & 3, half = warp >> 2;
  float* dst = partial + (size_t)w * TM * TM + (size_t)(32 * quarter + (tid & 31)) * TM;
  float v[32];
#pragma unroll 1
  for (int col = 64 * half; col < 64 * half + 64; col += 32) {
    if (chunks > 0 && ok) {
      tc::tmem_ld_32x32b_x32(tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)col, v);
    } else {
#pragma unroll
      for (int i = 0; i < 32; ++i) v[i] = 0.f;
    }
#pragma unroll
    for (int i = 0; i < 32; i += 4)
      *reinterpret_cast<float4*>(dst + col + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, TM);
}

// Ordered FP64 sum of the FP32 partial tiles of every tile into the output grid.
__global__ void __launch_bounds__(256) k_reduce_tc(GridDev gd, const ShotDev* __restrict__ shots,
                                                   int nshots, const int64_t* __restrict__ seg_off,
                                                   const float* __restrict__ partial,
                                                   double* __restrict__ out) {
  const int64_t t = blockIdx.x;
  const int s = shot_of_tile(shots, nshots, t);
  const ShotDev& sh = shots[s];
  int64_t a[2], b[2];
  tile_box<2>(gd, sh, t - sh.tile_off, a, b);
  const int64_t w0 = seg_off[t], w1 = seg_off[t + 1];
  for (int idx = threadIdx.x; idx < TM * TM; idx += 256) {
    double v = 0.0;
    for (int64_t w = w0; w < w1; ++w) v += (double)partial[w * TM * TM + idx];
    int64_t ix = a[0] + idx / TM, iz = a[1] + idx % TM;
    if (ix <= b[0] && iz <= b[1]) out[(int64_t)s * gd.npts + ix * gd.n[1] + iz] = v;
  }
}

__global__ void k_segments_tc(const int64_t* __restrict__ off, int64_t ntiles, int64_t list_cap,
                              int64_t seg, int64_t* __restrict__ seg_cnt) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= ntiles) return;
  int64_t a = min(off[t], list_cap), b = min(off[t + 1], list_cap);
  seg_cnt[t] = (b - a + seg - 1) / seg;
}

}  // namespace

int tile_edge_tc() { return TM; }

// Gaussians per work item, raised when needed to keep the FP32 partial tiles within
// 4 GiB (see segment_len).
int64_t segment_len_tc(fga_plan_s* p) {
  const int64_t want = p->seg > 0 ? p->seg : SEGM;
  const int64_t tile_bytes = (int64_t)TM * TM * (int64_t)sizeof(float);
  const int64_t items = std::max<int64_t>((((int64_t)4 << 30) / tile_bytes) - p->ntiles, 1);
  const int64_t floor_len = ((int64_t)p->list_cap + items - 1) / items;
  return std::max<int64_t>(want, floor_len);
}

size_t partial_items_tc(fga_plan_s* p) {
  const int64_t seg = segment_len_tc(p);
  return (size_t)p->ntiles + (p->list_cap + seg - 1) / seg;
}

size_t partial_bytes_tc(fga_plan_s* p) { return partial_items_tc(p) * TM * TM * sizeof(float); }

size_t anchor_bytes_tc(fga_plan_s* p) { return std::max<size_t>(p->g_cap, 1) * sizeof(GaussAnchor); }

cudaError_t launch_reconstruct_tc(fga_plan_s* p, double* u_dev) {
  if (p->ntiles == 0) return cudaSuccess;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_gather_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kSmemBytes);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  k_segments_tc<<<(unsigned)((p->ntiles + 255) / 256), 256, 0, p->stream>>>(
      p->d_tile_off, p->ntiles, (int64_t)p->list_cap, segment_len_tc(p), p->d_seg_off);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = launch_scan(p, p->d_seg_off, p->ntiles);
  if (e != cudaSuccess) return e;
  if (p->ganc_cap < anchor_bytes_tc(p)) return cudaErrorInvalidValue;  // sized by reconstruct_capacity
  GaussAnchor* ganc = reinterpret_cast<GaussAnchor*>(p->d_ganc);
  const int64_t G = p->dev_counts ? (int64_t)p->g_cap : p->G;
  if (G > 0) {
    const unsigned gb = (unsigned)std::min<int64_t>((G + 255) / 256, 4096);
    k_anchor_tc<<<gb, 256, 0, p->stream>>>(p->grid, p->d_shots, p->d_gshot, p->d_state,
                                            (int64_t)p->g_cap, p->d_gcoef, G,
                                            p->dev_counts ? p->d_gm : nullptr, p->kappa, ganc);
    p->launches += 1;
  }
  const unsigned items = (unsigned)partial_items_tc(p);
  k_gather_tc<<<items, NTC, kSmemBytes, p->stream>>>(
      p->grid, p->d_shots, p->nshots, ganc, p->d_tile_off, p->d_tile_list, (int64_t)p->list_cap,
      p->d_seg_off, p->ntiles, segment_len_tc(p), reinterpret_cast<float*>(p->d_partial), p->d_status,
      p->wait_tries >= 0 ? (uint32_t)p->wait_tries : kMaxTries);
  k_reduce_tc<<<(unsigned)p->ntiles, 256, 0, p->stream>>>(p->grid, p->d_shots, p->nshots,
                                                          p->d_seg_off,
                                                          reinterpret_cast<float*>(p->d_partial),
                                                          u_dev);
  p->launches += 3;
  return cudaGetLastError();
}

}  // namespace fga
