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
constexpr int NTC = 128;      // threads per CTA
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

// Per (Gaussian, axis) of a chunk: what every thread needs to make that Gaussian's
// factor at its own row of the tile.
struct Anchor {
  uint32_t u0, ud;  // phase at the tile's first point and per point, as fractions of a turn
  float d0, h;      // offset of the first point from Q, and the spacing
  int lo, hi;       // rows inside the window |d| <= cut (empty when lo > hi)
  float2 cf;        // coefficient (x axis) or 1 (z axis)
};

// The anchor of one Gaussian on one axis of the tile starting at x0 (FP64: the phase
// P (x0 - Q)/eps and its per-point step P h/eps as 32-bit fractions of a turn, so that
// the phase at row r is the exact wrap-around sum u0 + r ud).
__device__ __forceinline__ Anchor make_anchor(double x0, double h, double inv_h, double Q, double P,
                                              double cut, double inv_eps, float2 cf) {
  const double inv_two_pi = 0.15915494309189535;
  const double d0 = x0 - Q;
  double t0 = P * d0 * inv_eps * inv_two_pi, td = P * h * inv_eps * inv_two_pi;
  t0 -= floor(t0);
  td -= floor(td);
  Anchor an;
  an.u0 = (uint32_t)(unsigned long long)floor(t0 * 4294967296.0 + 0.5);
  an.ud = (uint32_t)(unsigned long long)floor(td * 4294967296.0 + 0.5);
  an.d0 = (float)d0;
  an.h = (float)h;
  double lo = ceil((-cut - d0) * inv_h), hi = floor((cut - d0) * inv_h);
  lo = lo < 0.0 ? 0.0 : lo;
  hi = hi > (double)(TM - 1) ? (double)(TM - 1) : hi;
  an.lo = (int)lo;
  an.hi = (int)hi;
  an.cf = cf;
  return an;
}

__device__ __forceinline__ Anchor make_empty_anchor() {
  Anchor an;
  an.u0 = an.ud = 0u;
  an.d0 = an.h = 0.f;
  an.lo = 1;
  an.hi = 0;
  an.cf = make_float2(0.f, 0.f);
  return an;
}

// Factor of a Gaussian at row r: cf * exp(i phase - d^2/(2 eps)) (0 outside the window).
__device__ __forceinline__ float2 row_factor(const Anchor& an, int r, float inv_eps) {
  if (r < an.lo || r > an.hi) return make_float2(0.f, 0.f);
  const float ang_scale = 1.4629180792671596e-09f;  // 2 pi / 2^32
  const float d = fmaf((float)r, an.h, an.d0);
  const float gs = __expf(-0.5f * d * d * inv_eps);
  float sn, cs;
  __sincosf((float)(int32_t)(an.u0 + (uint32_t)r * an.ud) * ang_scale, &sn, &cs);
  const float fr = gs * cs, fi = gs * sn;
  return make_float2(an.cf.x * fr - an.cf.y * fi, an.cf.x * fi + an.cf.y * fr);
}

__device__ __forceinline__ void store_split4(float* hi, float* lo, int o, float4 v) {
  const float4 h = make_float4(tf32_head(v.x), tf32_head(v.y), tf32_head(v.z), tf32_head(v.w));
  *reinterpret_cast<float4*>(hi + o) = h;
  *reinterpret_cast<float4*>(lo + o) = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
}

__global__ void __launch_bounds__(NTC) k_gather_tc(GridDev gd, const ShotDev* __restrict__ shots,
                                                   int nshots, double kappa,
                                                   const double* __restrict__ state, int64_t ld,
                                                   const double2* __restrict__ coef,
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
  const int tid = threadIdx.x, warp = tid >> 5;
  const int64_t t = tile_of_item(seg_off, ntiles, w);
  const int s = shot_of_tile(shots, nshots, t);
  const ShotDev& sh = shots[s];
  const double cut = kappa * sh.sqrt_eps, inv_eps = sh.inv_eps;
  int64_t a[2], b[2];
  tile_box<2>(gd, sh, t - sh.tile_off, a, b);
  if (tid == 0) {
    tc::mbar_init(bar, 1);
    tc::fence_mbar_init();
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
  const float inv_eps_f = (float)inv_eps;
  // One operand buffer (three CTAs share an SM, so one CTA's factors are made while
  // another's MMAs run); before it is overwritten the previous chunk's MMAs must be done.
  float* Ahi = reinterpret_cast<float*>(smem);
  float* Alo = Ahi + TM * KC;
  float* Bhi = Alo + TM * KC;
  float* Blo = Bhi + TM * KC;
  uint32_t chunks = 0;
  bool gave_up = false;
  for (int64_t c0 = l0; c0 < l1; c0 += CHG) {
    const int nc = (int)((l1 - c0) < CHG ? (l1 - c0) : CHG);
    // anchors: thread 2 gi + axis (the factors of the previous chunk are already made)
    Anchor an = make_empty_anchor();
    const int gi = tid >> 1, axis = tid & 1;
    if (tid < 2 * CHG && gi < nc) {
      const int32_t g = list[c0 + gi];
      const double Q = state[axis * ld + g], P = state[(2 + axis) * ld + g];
      float2 cf = make_float2(1.f, 0.f);
      if (axis == 0) {
        const double2 c = coef[g];
        cf = make_float2((float)c.x, (float)c.y);
      }
      const double x0 = axis == 0 ? gd.o[0] + (double)a[0] * gd.h[0] : gd.o[1] + (double)a[1] * gd.h[1];
      an = make_anchor(x0, gd.h[axis], gd.inv_h[axis], Q, P, cut, inv_eps, cf);
    }
    // the CTA gives up as a whole, with at most the previous commit outstanding
    bool waited = true;
    if (chunks > 0) waited = tc::mbar_wait_bounded(bar, (chunks - 1) & 1u, tries);
    if (!__syncthreads_and(waited)) {
      gave_up = true;
      break;
    }
    if (tid < 2 * CHG) anc[axis][gi] = an;
    __syncthreads();
    // operands: thread = row of the tile (x for A, z for B), four K values per store
    // A[x][2g] = Re X_g, A[x][2g+1] = -Im X_g; B[z][2g] = Re Z_g, B[z][2g+1] = Im Z_g
#pragma unroll
    for (int gp = 0; gp < CHG / 2; ++gp) {
      const float2 x0 = row_factor(anc[0][2 * gp], tid, inv_eps_f);
      const float2 x1 = row_factor(anc[0][2 * gp + 1], tid, inv_eps_f);
      const float2 z0 = row_factor(anc[1][2 * gp], tid, inv_eps_f);
      const float2 z1 = row_factor(anc[1][2 * gp + 1], tid, inv_eps_f);
      const int o = core_offset(tid, 4 * gp);
      store_split4(Ahi, Alo, o, make_float4(x0.x, -x0.y, x1.x, -x1.y));
      store_split4(Bhi, Blo, o, make_float4(z0.x, z0.y, z1.x, z1.y));
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
  // epilogue: warp w holds rows (x) 32w .. 32w+31, one row per thread, 128 columns (z)
  float* dst = partial + (size_t)w * TM * TM + (size_t)(32 * warp + (tid & 31)) * TM;
  float v[32];
#pragma unroll 1
  for (int col = 0; col < TM; col += 32) {
    if (chunks > 0 && ok) {
      tc::tmem_ld_32x32b_x32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)col, v);
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
  const unsigned items = (unsigned)partial_items_tc(p);
  k_gather_tc<<<items, NTC, kSmemBytes, p->stream>>>(
      p->grid, p->d_shots, p->nshots, p->kappa, p->d_state, (int64_t)p->g_cap, p->d_gcoef,
      p->d_tile_off, p->d_tile_list, (int64_t)p->list_cap, p->d_seg_off, p->ntiles,
      segment_len_tc(p), reinterpret_cast<float*>(p->d_partial), p->d_status,
      p->wait_tries >= 0 ? (uint32_t)p->wait_tries : kMaxTries);
  k_reduce_tc<<<(unsigned)p->ntiles, 256, 0, p->stream>>>(p->grid, p->d_shots, p->nshots,
                                                          p->d_seg_off,
                                                          reinterpret_cast<float*>(p->d_partial),
                                                          u_dev);
  p->launches += 3;
  return cudaGetLastError();
}

}  // namespace fga
