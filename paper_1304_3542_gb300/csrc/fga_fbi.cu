// Step 1 of the method (Initial wavefield decomposition section): the FBI
// transform of f0 and f1 on a box of n_b points per axis around every q, and
// the branch split of Eq. psi.
//
// The paper evaluates each box with an FFT. Here the box transform is the
// separable contraction with the constant window-DFT matrix of each axis,
//   E_k[jp][j] = w_k(r_j) exp(-i p_jp r_j/eps),  r_j = (j - n_b/2) h_k,
// which is the same sum: psi(q, p) = h^d sum_j f(q + r_j) prod_k E_k[jp_k][j_k].
// In 2D the contraction along the last axis does not depend on the q-row, so it
// is done once per data row (stage 1, shared by every q of a column) and the
// contraction along the first axis is a dense complex GEMM per q (stage 2).
// Both stages are FP64 tiled GEMMs; the stage that yields psi fuses the branch
// split psi+ = 1/2 (psi_0 + i eps psi_1/(c(q)|p|)), the removal of the left-out
// p values and the running max of |psi+|^2 per shot. In the mixed precision the
// per-q GEMM of stage 2 (2D) runs on the tensor cores instead (k_fbi_stage2_tc).
#include <algorithm>
#include <climits>

#include <type_traits>

#include "fga_internal.cuh"
#include "fga_medium.cuh"
#include "fga_tc.cuh"

namespace fga {

namespace {

constexpr int BM = 32, BN = 32, BK = 16, NT = 256;

__device__ __forceinline__ int64_t wrap_or_invalid(int64_t i, int64_t n, int periodic) {
  if (periodic) {
    int64_t r = i % n;
    return r < 0 ? r + n : r;
  }
  return (i >= 0 && i < n) ? i : -1;
}

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* addr, double v) {
  atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}

__global__ void k_bbox_init(int* bbox, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) bbox[i] = (i & 1) ? -1 : INT_MAX;
}

// Bounding box of the nonzero samples of (u0, u1) per shot: bbox[s][k] = {lo, hi}.
__global__ void k_support_bbox(GridDev gd, const double* __restrict__ u0,
                               const double* __restrict__ u1, int* bbox) {
  int s = blockIdx.y;
  const double* a = u0 + (int64_t)s * gd.npts;
  const double* b = u1 + (int64_t)s * gd.npts;
  int lo[kMaxDim], hi[kMaxDim];
  for (int k = 0; k < kMaxDim; ++k) {
    lo[k] = INT_MAX;
    hi[k] = -1;
  }
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < gd.npts;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (a[i] != 0.0 || b[i] != 0.0) {
      int64_t rem = i;
      for (int k = gd.dim - 1; k >= 0; --k) {
        int c = (int)(rem % gd.n[k]);
        rem /= gd.n[k];
        lo[k] = min(lo[k], c);
        hi[k] = max(hi[k], c);
      }
    }
  }
  for (int k = 0; k < gd.dim; ++k) {
    for (int off = 16; off > 0; off >>= 1) {
      lo[k] = min(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], off));
      hi[k] = max(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], off));
    }
    if ((threadIdx.x & 31) == 0 && hi[k] >= 0) {
      atomicMin(bbox + (s * gd.dim + k) * 2 + 0, lo[k]);
      atomicMax(bbox + (s * gd.dim + k) * 2 + 1, hi[k]);
    }
  }
}

// Branch split, left-out p values and max |psi+|^2 for one output element.
// out = psi+ = psi_0/2 + t, t = i eps psi_1/(2 c(q)|p|) (t is kept for the adjoint).
template <int D>
__device__ __forceinline__ double psi_plus(const ShotDev& sh, int64_t jp, double2 p0, double2 p1,
                                           double cq, double2& out, double2& t) {
  bool valid;
  double pn;
  if constexpr (D == 1) {
    int64_t m = jp - sh.nb[0] / 2;
    valid = (jp != 0) && (m != 0);
    pn = fabs((double)m) * sh.pscale[0];
  } else {
    int64_t j0 = jp / sh.nb[1], j1 = jp - j0 * sh.nb[1];
    int64_t m0 = j0 - sh.nb[0] / 2, m1 = j1 - sh.nb[1] / 2;
    valid = (j0 != 0) && (j1 != 0) && !(m0 == 0 && m1 == 0);
    double a = (double)m0 * sh.pscale[0], b = (double)m1 * sh.pscale[1];
    pn = sqrt(a * a + b * b);
  }
  if (!valid) {
    out = make_double2(0.0, 0.0);
    t = out;
    return 0.0;
  }
  double r = sh.eps / (cq * pn);
  t = make_double2(-0.5 * r * p1.y, 0.5 * r * p1.x);
  out = make_double2(0.5 * p0.x + t.x, 0.5 * p0.y + t.y);
  return abs2_rn(out);
}

// Scalar and complex types of stage 1: FP64 (the FP64 path) or FP32 (the mixed path).
template <typename T> struct Cplx;
template <> struct Cplx<double> {
  using type = double2;
  static __device__ __forceinline__ double2 make(double x, double y) { return make_double2(x, y); }
};
template <> struct Cplx<float> {
  using type = float2;
  static __device__ __forceinline__ float2 make(float x, float y) { return make_float2(x, y); }
};

// TF32 head and FP32 tail of a complex value: (Re head, Re tail, Im head, Im tail); for
// an FP32 value head + tail is the value itself.
__device__ __forceinline__ float4 split4(float2 v) {
  const float hr = __uint_as_float(__float_as_uint(v.x) & 0xFFFFE000u);
  const float hi = __uint_as_float(__float_as_uint(v.y) & 0xFFFFE000u);
  return make_float4(hr, v.x - hr, hi, v.y - hi);
}
__device__ __forceinline__ float4 split4(double2 v) {
  const float xr = (float)v.x, xi = (float)v.y;
  const float hr = __uint_as_float(__float_as_uint(xr) & 0xFFFFE000u);
  const float hi = __uint_as_float(__float_as_uint(xi) & 0xFFFFE000u);
  return make_float4(hr, (float)(v.x - (double)hr), hi, (float)(v.y - (double)hi));
}

// Stage 1: C_f[m][n] = sum_k data_f(m, k) * E_last[n][k], f = 0, 1.
// D == 2: m = (row r, q_z local), k runs along the last axis of the box; the
//         result goes to the stage-1 buffer.
// D == 1: m = q local, and the epilogue forms psi+.
// T: the arithmetic (double; float in the mixed path, 2D, where the result becomes the
// split-TF32 B operand of the tensor-core stage 2: FP32 products, each an exact FP32
// rounding and so finer than the TF32 split products that consume them, accumulated in
// FP32 on the CUDA cores, which run FP32 at 62 times the FP64 rate).
template <int D, typename T = double>
__global__ void __launch_bounds__(NT) k_fbi_stage1(GridDev gd, const ShotDev* __restrict__ shots,
                                                   const double* __restrict__ u0,
                                                   const double* __restrict__ u1,
                                                   const double* __restrict__ C,
                                                   double2* __restrict__ g1,
                                                   double2* __restrict__ psi,
                                                   double2* __restrict__ psi_f1,
                                                   unsigned long long* __restrict__ max2,
                                                   int split_out) {
  const int s = blockIdx.z;
  const ShotDev sh = shots[s];
  constexpr int L = D - 1;  // last axis
  const int64_t nbl = sh.nb[L];
  const int64_t M = (D == 2) ? sh.nrows * sh.qn[1] : sh.qn[0];
  const int64_t N = nbl, K = nbl;
  const int64_t m0 = (int64_t)blockIdx.y * BM, n0 = (int64_t)blockIdx.x * BN;
  if (m0 >= M || n0 >= N) return;
  using T2 = typename Cplx<T>::type;
  __shared__ T As[2][BK][BM];
  __shared__ T2 Bs[BK][BN];
  __shared__ double cq_s[BM];
  const int t = threadIdx.x, tx = t % 16, ty = t / 16;
  const double* f0 = u0 + (int64_t)s * gd.npts;
  const double* f1 = u1 + (int64_t)s * gd.npts;
  T2 acc0[2][2], acc1[2][2];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      acc0[i][j] = Cplx<T>::make(0, 0);
      acc1[i][j] = Cplx<T>::make(0, 0);
    }
  const double2* ELAST = sh.E[L];  // last-axis window-DFT matrix [n_b][n_b]
  for (int64_t k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      int e = t + NT * i;
      int mm = e / BK, kk = e % BK;
      int64_t m = m0 + mm, k = k0 + kk;
      double v0 = 0.0, v1 = 0.0;
      if (m < M && k < K) {
        int64_t idx;
        if constexpr (D == 2) {
          int64_t r = m / sh.qn[1], mzl = m - r * sh.qn[1];
          int64_t ix = wrap_or_invalid(sh.row_lo + r, gd.n[0], gd.periodic[0]);
          int64_t iz = wrap_or_invalid(sh.s[1] * (sh.qlo[1] + mzl) + k - nbl / 2, gd.n[1],
                                       gd.periodic[1]);
          idx = (ix < 0 || iz < 0) ? -1 : ix * gd.n[1] + iz;
        } else {
          idx = wrap_or_invalid(sh.s[0] * (sh.qlo[0] + m) + k - nbl / 2, gd.n[0],
                                gd.periodic[0]);
        }
        if (idx >= 0) {
          v0 = __ldg(f0 + idx);
          v1 = __ldg(f1 + idx);
        }
      }
      As[0][kk][mm] = (T)v0;
      As[1][kk][mm] = (T)v1;
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      int e = t + NT * i;
      int nn = e / BK, kk = e % BK;
      int64_t n = n0 + nn, k = k0 + kk;
      double2 v = make_double2(0, 0);
      if (n < N && k < K) v = __ldg(ELAST + n * K + k);
      Bs[kk][nn] = Cplx<T>::make((T)v.x, (T)v.y);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a0[2], a1[2];
      T2 b[2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        a0[i] = As[0][kk][ty + 16 * i];
        a1[i] = As[1][kk][ty + 16 * i];
        b[i] = Bs[kk][tx + 16 * i];
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          acc0[i][j].x = fma(a0[i], b[j].x, acc0[i][j].x);
          acc0[i][j].y = fma(a0[i], b[j].y, acc0[i][j].y);
          acc1[i][j].x = fma(a1[i], b[j].x, acc1[i][j].x);
          acc1[i][j].y = fma(a1[i], b[j].y, acc1[i][j].y);
        }
    }
    __syncthreads();
  }
  if constexpr (D == 2) {
    const int64_t plane = M * N;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        int64_t m = m0 + ty + 16 * i, n = n0 + tx + 16 * j;
        if (m < M && n < N) {
          if (split_out) {
            // mixed precision: TF32 head/tail splits, written straight into the B operand
            // image of the tensor-core stage 2 (every row is the first row of a pair of
            // its own parity and the second of a pair of the other parity)
            const int64_t r = m / sh.qn[1], mzl = m - r * sh.qn[1];
            float* img = reinterpret_cast<float*>(g1 + sh.g1_off);
            const int64_t nt = n / 128, w = n % 128, npair = fbi_b_pairs(sh), ntile = fbi_b_ntile(sh);
#pragma unroll
            for (int f = 0; f < 2; ++f) {
              const float4 v = split4(f == 0 ? acc0[i][j] : acc1[i][j]);
#pragma unroll
              for (int slot = 0; slot < 2; ++slot) {
                const int64_t rr = r - slot;
                if (rr < 0) continue;
                const int64_t par = rr & 1, t = rr >> 1;
                const int64_t b = ((((((int64_t)f * sh.qn[1] + mzl) * 2 + par) * ntile + nt) * 2) * npair + t) * 512 +
                                  w * 4 + 2 * slot;
                *reinterpret_cast<float2*>(img + b) = make_float2(v.x, v.z);                 // head
                *reinterpret_cast<float2*>(img + b + npair * 512) = make_float2(v.y, v.w);   // tail
              }
            }
          } else if constexpr (std::is_same<T, double>::value) {
            g1[sh.g1_off + m * N + n] = acc0[i][j];
            g1[sh.g1_off + plane + m * N + n] = acc1[i][j];
          }
        }
      }
  } else if constexpr (std::is_same<T, double>::value) {
    // c(q) for the rows of this tile
    if (t < BM) {
      int64_t m = m0 + t;
      double q = gd.o[0] + (double)(sh.s[0] * (sh.qlo[0] + m)) * gd.h[0];
      cq_s[t] = (m < M) ? medium_value<1>(gd, C, &q) : 1.0;
    }
    __syncthreads();
    const double hv = gd.h[0];
    double mymax = 0.0;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        int64_t m = m0 + ty + 16 * i, n = n0 + tx + 16 * j;
        if (m < M && n < N) {
          double2 p0 = make_double2(hv * acc0[i][j].x, hv * acc0[i][j].y);
          double2 p1 = make_double2(hv * acc1[i][j].x, hv * acc1[i][j].y);
          double2 o, tt;
          double a2 = psi_plus<1>(sh, n, p0, p1, cq_s[ty + 16 * i], o, tt);
          psi[sh.psi_off + m * sh.np + n] = o;
          psi_f1[sh.psi_off + m * sh.np + n] = tt;
          mymax = fmax(mymax, a2);
        }
      }
    for (int off = 16; off > 0; off >>= 1) mymax = fmax(mymax, __shfl_xor_sync(0xffffffffu, mymax, off));
    if ((t & 31) == 0) atomic_max_nonneg(max2 + s, mymax);
  }
}

// Stage 2 (2D): for one q, psi_f[jpx][jpz] = h_x h_z sum_jx E_x[jpx][jx] G1_f[row(jx)][jpz],
// then the branch split.
__global__ void __launch_bounds__(NT) k_fbi_stage2(GridDev gd, const ShotDev* __restrict__ shots,
                                                   const double* __restrict__ C,
                                                   const double2* __restrict__ g1,
                                                   double2* __restrict__ psi,
                                                   double2* __restrict__ psi_f1,
                                                   unsigned long long* __restrict__ max2) {
  const int s = blockIdx.z;
  const ShotDev sh = shots[s];
  const int64_t qtot = sh.qn[0] * sh.qn[1];
  const int64_t ql = blockIdx.y;
  if (ql >= qtot) return;
  const int64_t nbx = sh.nb[0], nbz = sh.nb[1];
  const int64_t tiles_n = (nbz + BN - 1) / BN;
  const int64_t m0 = (blockIdx.x / tiles_n) * BM, n0 = (blockIdx.x % tiles_n) * BN;
  if (m0 >= nbx) return;
  const int64_t mxl = ql / sh.qn[1], mzl = ql - mxl * sh.qn[1];
  const int64_t M1 = sh.nrows * sh.qn[1];
  const int64_t plane = M1 * nbz;
  const double2* G0 = g1 + sh.g1_off;
  const double2* G1p = G0 + plane;
  const double2* Ex = sh.E[0];
  __shared__ double2 As[BK][BM];
  __shared__ double2 Bs[2][BK][BN];
  __shared__ double cq_s;
  const int t = threadIdx.x, tx = t % 16, ty = t / 16;
  if (t == 0) {
    double q[2] = {gd.o[0] + (double)(sh.s[0] * (sh.qlo[0] + mxl)) * gd.h[0],
                   gd.o[1] + (double)(sh.s[1] * (sh.qlo[1] + mzl)) * gd.h[1]};
    cq_s = medium_value<2>(gd, C, q);
  }
  double2 acc0[2][2], acc1[2][2];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      acc0[i][j] = make_double2(0, 0);
      acc1[i][j] = make_double2(0, 0);
    }
  const int64_t row0 = sh.s[0] * mxl;  // stage-1 row of box index jx = 0
  for (int64_t k0 = 0; k0 < nbx; k0 += BK) {
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      int e = t + NT * i;
      int mm = e / BK, kk = e % BK;
      int64_t m = m0 + mm, k = k0 + kk;
      As[kk][mm] = (m < nbx && k < nbx) ? __ldg(Ex + m * nbx + k) : make_double2(0, 0);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      int e = t + NT * i;
      int kk = e / BN, nn = e % BN;
      int64_t k = k0 + kk, n = n0 + nn;
      double2 v0 = make_double2(0, 0), v1 = make_double2(0, 0);
      if (k < nbx && n < nbz) {
        int64_t off = ((row0 + k) * sh.qn[1] + mzl) * nbz + n;
        v0 = __ldg(G0 + off);
        v1 = __ldg(G1p + off);
      }
      Bs[0][kk][nn] = v0;
      Bs[1][kk][nn] = v1;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double2 a[2], b0[2], b1[2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        a[i] = As[kk][ty + 16 * i];
        b0[i] = Bs[0][kk][tx + 16 * i];
        b1[i] = Bs[1][kk][tx + 16 * i];
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          acc0[i][j].x = fma(a[i].x, b0[j].x, fma(-a[i].y, b0[j].y, acc0[i][j].x));
          acc0[i][j].y = fma(a[i].x, b0[j].y, fma(a[i].y, b0[j].x, acc0[i][j].y));
          acc1[i][j].x = fma(a[i].x, b1[j].x, fma(-a[i].y, b1[j].y, acc1[i][j].x));
          acc1[i][j].y = fma(a[i].x, b1[j].y, fma(a[i].y, b1[j].x, acc1[i][j].y));
        }
    }
    __syncthreads();
  }
  const double hv = gd.h[0] * gd.h[1];
  double mymax = 0.0;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      int64_t m = m0 + ty + 16 * i, n = n0 + tx + 16 * j;
      if (m < nbx && n < nbz) {
        double2 p0 = make_double2(hv * acc0[i][j].x, hv * acc0[i][j].y);
        double2 p1 = make_double2(hv * acc1[i][j].x, hv * acc1[i][j].y);
        double2 o, tt;
        int64_t jp = m * nbz + n;
        double a2 = psi_plus<2>(sh, jp, p0, p1, cq_s, o, tt);
        psi[sh.psi_off + ql * sh.np + jp] = o;
        psi_f1[sh.psi_off + ql * sh.np + jp] = tt;
        mymax = fmax(mymax, a2);
      }
    }
  for (int off = 16; off > 0; off >>= 1) mymax = fmax(mymax, __shfl_xor_sync(0xffffffffu, mymax, off));
  if ((t & 31) == 0) atomic_max_nonneg(max2 + s, mymax);
}

// ---------------------------------------------------------------------------
// 3D: three separable stages over all active q of a shot, one thread per output
// entry (FP64; the stage outputs and psi are held for every active q):
//   stage 1 (z): G1_f[x][y][q_z][p_z]     = sum_jz f(x, y, z(q_z, jz)) E_z[p_z][jz]
//   stage 2 (y): G2_f[x][q_y][q_z][p_y][p_z] = sum_jy E_y[p_y][jy] G1_f[x][y(q_y, jy)][q_z][p_z]
//   stage 3 (x): psi_f[q][p_x][p_y][p_z]   = h^3 sum_jx E_x[p_x][jx] G2_f[x(q_x, jx)][q_y][q_z][p_y][p_z]
// with the branch split of Eq. psi in the last stage. x and y run over the data rows the
// active q's boxes touch (wrapped on periodic axes, zero outside an open axis).
__global__ void k_fbi3_stage1(GridDev gd, const ShotDev* __restrict__ shots,
                              const double* __restrict__ u0, const double* __restrict__ u1,
                              double2* __restrict__ g1) {
  const int s = blockIdx.y;
  const ShotDev& sh = shots[s];
  const int64_t nbz = sh.nb[2];
  const int64_t plane = sh.nrows * sh.nrows1 * sh.qn[2] * nbz;
  const double* f0 = u0 + (int64_t)s * gd.npts;
  const double* f1 = u1 + (int64_t)s * gd.npts;
  const double2* Ez = sh.E[2];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < plane;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pz = e % nbz;
    int64_t r = e / nbz;
    const int64_t qz = r % sh.qn[2];
    r /= sh.qn[2];
    const int64_t yr = r % sh.nrows1, xr = r / sh.nrows1;
    const int64_t ix = wrap_or_invalid(sh.row_lo + xr, gd.n[0], gd.periodic[0]);
    const int64_t iy = wrap_or_invalid(sh.row_lo1 + yr, gd.n[1], gd.periodic[1]);
    double2 a0 = make_double2(0.0, 0.0), a1 = a0;
    if (ix >= 0 && iy >= 0) {
      const int64_t base = (ix * gd.n[1] + iy) * gd.n[2];
      const int64_t z0 = (int64_t)sh.s[2] * (sh.qlo[2] + qz) - nbz / 2;
      for (int64_t jz = 0; jz < nbz; ++jz) {
        const int64_t iz = wrap_or_invalid(z0 + jz, gd.n[2], gd.periodic[2]);
        if (iz < 0) continue;
        const double v0 = __ldg(f0 + base + iz), v1 = __ldg(f1 + base + iz);
        const double2 E = __ldg(Ez + pz * nbz + jz);
        a0.x = fma(v0, E.x, a0.x);
        a0.y = fma(v0, E.y, a0.y);
        a1.x = fma(v1, E.x, a1.x);
        a1.y = fma(v1, E.y, a1.y);
      }
    }
    g1[sh.g1_off + e] = a0;
    g1[sh.g1_off + plane + e] = a1;
  }
}

__global__ void k_fbi3_stage2(const ShotDev* __restrict__ shots, const double2* __restrict__ g1,
                              double2* __restrict__ g2) {
  const int s = blockIdx.y;
  const ShotDev& sh = shots[s];
  const int64_t nby = sh.nb[1], nbz = sh.nb[2];
  const int64_t plane1 = sh.nrows * sh.nrows1 * sh.qn[2] * nbz;
  const int64_t plane2 = sh.nrows * sh.qn[1] * sh.qn[2] * nby * nbz;
  const double2* Ey = sh.E[1];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < plane2;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pz = e % nbz;
    int64_t r = e / nbz;
    const int64_t py = r % nby;
    r /= nby;
    const int64_t qz = r % sh.qn[2];
    r /= sh.qn[2];
    const int64_t qy = r % sh.qn[1], xr = r / sh.qn[1];
    const int64_t y0 = (int64_t)sh.s[1] * qy;  // y row of jy = 0 relative to row_lo1
    double2 a0 = make_double2(0.0, 0.0), a1 = a0;
    for (int64_t jy = 0; jy < nby; ++jy) {
      const int64_t off = ((xr * sh.nrows1 + y0 + jy) * sh.qn[2] + qz) * nbz + pz;
      const double2 b0 = g1[sh.g1_off + off], b1 = g1[sh.g1_off + plane1 + off];
      const double2 E = __ldg(Ey + py * nby + jy);
      a0.x = fma(E.x, b0.x, fma(-E.y, b0.y, a0.x));
      a0.y = fma(E.x, b0.y, fma(E.y, b0.x, a0.y));
      a1.x = fma(E.x, b1.x, fma(-E.y, b1.y, a1.x));
      a1.y = fma(E.x, b1.y, fma(E.y, b1.x, a1.y));
    }
    g2[sh.g2_off + e] = a0;
    g2[sh.g2_off + plane2 + e] = a1;
  }
}

// Stage 3 and the branch split: one block per (active q, shot), its threads over the p
// indices of the box. c(q) is evaluated once per block; a thread steps its p index
// (j0, j1, j2) by the block size with carries instead of dividing.
__global__ void __launch_bounds__(256) k_fbi3_stage3(GridDev gd, const ShotDev* __restrict__ shots,
                                                     const double* __restrict__ C,
                                                     const double2* __restrict__ g2,
                                                     double2* __restrict__ psi,
                                                     double2* __restrict__ psi_f1,
                                                     unsigned long long* __restrict__ max2) {
  const int s = blockIdx.y;
  const ShotDev& sh = shots[s];
  const int64_t qn12 = sh.qn[1] * sh.qn[2];
  const int64_t ql = blockIdx.x;
  if (ql >= sh.qn[0] * qn12) return;  // the whole block
  const int nbx = sh.nb[0], nby = sh.nb[1], nbz = sh.nb[2], nbyz = nby * nbz;
  const int64_t mx = ql / qn12, myz = ql - mx * qn12;
  __shared__ double epc_s;  // eps / c(q)
  if (threadIdx.x == 0) {
    const int64_t my = myz / sh.qn[2], mz = myz - my * sh.qn[2];
    const double q[3] = {gd.o[0] + (double)(sh.s[0] * (sh.qlo[0] + mx)) * gd.h[0],
                         gd.o[1] + (double)(sh.s[1] * (sh.qlo[1] + my)) * gd.h[1],
                         gd.o[2] + (double)(sh.s[2] * (sh.qlo[2] + mz)) * gd.h[2]};
    epc_s = sh.eps / medium_value<3>(gd, C, q);
  }
  __syncthreads();
  const double epc = epc_s;
  const double hv = gd.h[0] * gd.h[1] * gd.h[2];
  const int64_t plane2 = sh.nrows * qn12 * nbyz;
  const int64_t xstride = qn12 * nbyz;  // G2 entries between consecutive data rows x
  const double2* G0 = g2 + sh.g2_off + ((int64_t)sh.s[0] * mx * qn12 + myz) * nbyz;
  const double2* G1 = G0 + plane2;
  double2* out0 = psi + sh.psi_off + ql * sh.np;
  double2* out1 = psi_f1 + sh.psi_off + ql * sh.np;
  const int step = blockDim.x;
  int j0 = threadIdx.x / nbyz, j1 = (threadIdx.x - j0 * nbyz) / nbz;
  int j2 = threadIdx.x - j0 * nbyz - j1 * nbz;
  const int d0 = step / nbyz, d1 = (step - d0 * nbyz) / nbz, d2 = step - d0 * nbyz - d1 * nbz;
  double mymax = 0.0;
  for (int64_t jp = threadIdx.x; jp < sh.np; jp += step) {
    const int pyz = j1 * nbz + j2;
    const double2* b0p = G0 + pyz;
    const double2* b1p = G1 + pyz;
    const double2* Ep = sh.E[0] + (int64_t)j0 * nbx;
    double2 a0 = make_double2(0.0, 0.0), a1 = a0;
    for (int jx = 0; jx < nbx; ++jx, b0p += xstride, b1p += xstride) {
      const double2 b0 = *b0p, b1 = *b1p;
      const double2 E = __ldg(Ep + jx);
      a0.x = fma(E.x, b0.x, fma(-E.y, b0.y, a0.x));
      a0.y = fma(E.x, b0.y, fma(E.y, b0.x, a0.y));
      a1.x = fma(E.x, b1.x, fma(-E.y, b1.y, a1.x));
      a1.y = fma(E.x, b1.y, fma(E.y, b1.x, a1.y));
    }
    // Eq. psi: psi+ = psi_0/2 + t, t = i eps psi_1/(2 c(q)|p|); the Nyquist index of any
    // axis and p = 0 are left out
    const int m0 = j0 - nbx / 2, m1 = j1 - nby / 2, m2 = j2 - nbz / 2;
    double2 o = make_double2(0.0, 0.0), tt = o;
    if (j0 != 0 && j1 != 0 && j2 != 0 && !(m0 == 0 && m1 == 0 && m2 == 0)) {
      const double a = (double)m0 * sh.pscale[0], b = (double)m1 * sh.pscale[1],
                   c = (double)m2 * sh.pscale[2];
      const double r = epc * rsqrt_nr(fma(a, a, fma(b, b, c * c)));
      const double2 p0 = make_double2(hv * a0.x, hv * a0.y), p1 = make_double2(hv * a1.x, hv * a1.y);
      tt = make_double2(-0.5 * r * p1.y, 0.5 * r * p1.x);
      o = make_double2(0.5 * p0.x + tt.x, 0.5 * p0.y + tt.y);
      mymax = fmax(mymax, abs2_rn(o));
    }
    out0[jp] = o;
    out1[jp] = tt;
    j2 += d2;
    j1 += d1;
    j0 += d0;
    if (j2 >= nbz) {
      j2 -= nbz;
      ++j1;
    }
    if (j1 >= nby) {
      j1 -= nby;
      ++j0;
    }
  }
  for (int off = 16; off > 0; off >>= 1) mymax = fmax(mymax, __shfl_xor_sync(0xffffffffu, mymax, off));
  if ((threadIdx.x & 31) == 0) atomic_max_nonneg(max2 + s, mymax);
}

// ---------------------------------------------------------------------------
// Stage 2 on the tensor cores (mixed precision, 2D). For one q and one 128 x 128 tile
// of (p_x, p_z), the complex GEMM psi_f[px][pz] = sum_jx E_x[px][jx] G1_f[jx][pz] is
// written as real GEMMs over K = 2 jx:
//   Re psi_f = A_re B_f^T,  Im psi_f = A_im B_f^T,
//   A_re[px][2j] = Re E, A_re[px][2j+1] = -Im E,  A_im[px][2j] = Im E, A_im[px][2j+1] = Re E,
//   B_f[pz][2j] = Re G1_f, B_f[pz][2j+1] = Im G1_f,
// with every operand split into a TF32 head and an FP32 tail and the three products
// hi*hi + hi*lo + lo*hi accumulated in FP32 in tensor memory (four accumulators of 128
// columns: field 0 re/im, field 1 re/im).
//
// Operands: both live in global memory as the shared-memory image of a K chunk of 8
// complex jx (K = 16): the A image is built at plan time (E_x is the same for every q),
// the B image is what stage 1 writes (for each q column the pairs of stage-1 rows of
// either parity, so that every q's box, whatever the parity of its first row, reads its
// chunk as one contiguous block). K-major without swizzle: the core matrices (8 rows x
// 16 bytes) of one K quad lie for all 8-row groups in a row (SBO = 128 B), the four K
// quads of a chunk 2 KiB apart (LBO) in the B image; the A image stacks the Re-part and
// Im-part rows (32 groups, K quads 4 KiB apart), so that one MMA of N = 256 fills both
// accumulators of a field. The tensor cores read their operands from shared memory at
// about 128 B per clock; two MMAs of 128 x 128 x 8 (8 KiB each) per field would keep
// that bandwidth saturated, one of 128 x 256 x 8 (12 KiB) leaves room for the bulk
// copies. One thread runs a 3-stage pipeline: bulk
// copies (TMA, cp.async.bulk) of a chunk's A (32 KiB) and B (4 x 8 KiB) into a stage
// complete on the stage's "full" mbarrier; the chunk's 12 MMAs are committed to its
// "empty" mbarrier, after which the stage is refilled three chunks ahead; the last
// commit goes to "done", which the whole CTA waits on before the epilogue. Every wait
// is bounded; a thread that gives up issues nothing more and waits for what it has in
// flight (one phase per barrier at most) with the full budget before the tensor memory
// is released.
//
// The MMAs compute the transpose psi^T = B_f A^T (B_f as the M operand), so that the
// accumulator's TMEM lanes are p_z and its columns p_x. Epilogue (16 warps, four per
// TMEM lane quarter, each taking a quarter of the 128 columns, 16 at a time): a thread holds 16
// p_x values of its p_z column, and every store of a warp is one contiguous run of 32
// p_z columns of a p_x row, straight from registers. The branch split is FP32
// arithmetic on the FP32 accumulations (with 1/|p| from rsqrtf), stored as FP32 pairs:
// in this precision psi and its psi_1 part are FP32 values, and the selection widens
// them exactly. The maximum of |psi+|^2 is the selection's own FP64 |psi+|^2 of the
// stored values: a thread keeps its values in shared memory and afterwards evaluates
// the FP64 square only of those whose FP32 square (after an exact power-of-two scaling
// to the range of its largest component) is within 1e-6 of the largest such square,
// which any value whose FP64 square could be the largest is.
constexpr int FT = 128;        // tile edge in p_z (GEMM M) and p_x (GEMM N)
constexpr int FJ = 8;          // complex jx per chunk -> K = 16
constexpr int FNT = 512;       // 16 warps: warp w reads TMEM lanes 32 (w % 4) .., column quarter w / 4
constexpr int FCOLS = 32;      // p_x columns of the accumulators per epilogue warp
constexpr int FSTAGES = 3;
constexpr uint32_t kFbiOp = FT * 2 * FJ * sizeof(float);   // one operand part of a chunk: 8 KiB
constexpr uint32_t kFbiStage = 8 * kFbiOp;  // A: head and tail of 256 rows, B: 2 fields x 2 parts
constexpr uint32_t kFbiLBO = 2048, kFbiSBO = 128;  // B operand (128 rows): K quads 2 KiB apart
constexpr uint32_t kFbiALBO = 4096;                 // A operand (256 stacked rows): K quads 4 KiB apart
constexpr size_t kFbiBarOff = (size_t)FSTAGES * kFbiStage;
constexpr size_t kFbiSmem = kFbiBarOff + 128;
static_assert((size_t)FCOLS * FNT * sizeof(float2) <= kFbiBarOff,
              "the epilogue's values fit in the stage buffers");
constexpr uint32_t kFbiTries = 1u << 22;

// IEEE binary32 -> binary64 in integer arithmetic (exact, keeps the FP64 pipe free):
// re-bias the exponent and widen the significand; a subnormal m 2^-149 is normalised at
// its leading bit b (value 1.f 2^(b-149)); infinities and NaNs keep exponent 0x7ff.
__device__ __forceinline__ double widen_f32(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint64_t sign = (uint64_t)(u >> 31) << 63;
  const uint32_t e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
  uint64_t bits;
  if (e != 0u) {
    const uint64_t ed = e == 0xffu ? 0x7ffull : (uint64_t)(e + 896u);
    bits = sign | (ed << 52) | ((uint64_t)m << 29);
  } else if (m != 0u) {
    const int b = 31 - __clz(m);
    bits = sign | ((uint64_t)(b + 874) << 52) | (((uint64_t)m << (52 - b)) & 0xfffffffffffffull);
  } else {
    bits = sign;
  }
  return __longlong_as_double((long long)bits);
}

__global__ void __launch_bounds__(FNT) k_fbi_stage2_tc(GridDev gd, const ShotDev* __restrict__ shots,
                                                      const double* __restrict__ C,
                                                      const double2* __restrict__ g1,
                                                      float2* __restrict__ psi,
                                                      float2* __restrict__ psi_f1,
                                                      unsigned long long* __restrict__ max2,
                                                      int* status, uint32_t tries) {
  const int s = blockIdx.z;
  const ShotDev& sh = shots[s];
  const int64_t qtot = sh.qn[0] * sh.qn[1];
  const int64_t ql = blockIdx.y;
  const int64_t nbx = sh.nb[0], nbz = sh.nb[1];
  const int64_t tiles_z = (nbz + FT - 1) / FT;
  const int64_t mt = blockIdx.x / tiles_z, nt = blockIdx.x % tiles_z;
  const int64_t m0 = mt * FT, n0 = nt * FT;
  if (ql >= qtot || m0 >= nbx) return;  // uniform over the CTA
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kFbiBarOff);
  uint64_t* empty = full + FSTAGES;
  uint64_t* done = empty + FSTAGES;
  uint32_t* tbase = reinterpret_cast<uint32_t*>(done + 1);
  __shared__ float h2_s, c1_s, psx_s, psz_s;
  __shared__ int aborted_s;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int64_t mxl = ql / sh.qn[1], mzl = ql - mxl * sh.qn[1];
  if (tid == 0) {
    for (int i = 0; i < FSTAGES; ++i) {
      tc::mbar_init(&full[i], 1);
      tc::mbar_init(&empty[i], 1);
    }
    tc::mbar_init(done, 1);
    tc::fence_mbar_init();
    aborted_s = 0;
    psx_s = (float)sh.pscale[0];
    psz_s = (float)sh.pscale[1];
  }
  if (warp == 0) {
    tc::tmem_alloc(tbase, 4 * FT);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tbase;
  if (tid == 0) {
    const int nchunk = (int)(nbx / FJ);
    const float* Aimg = sh.Etc + (size_t)mt * nchunk * 4 * (kFbiOp / sizeof(float));
    const int64_t row0 = (int64_t)sh.s[0] * mxl;  // first stage-1 row of this q's box
    const int64_t par = row0 & 1, t0 = row0 >> 1;
    const float* Bimg = reinterpret_cast<const float*>(g1 + sh.g1_off);
    const int64_t npair = fbi_b_pairs(sh), ntile = fbi_b_ntile(sh);
    auto load = [&](int c) {
      const int st = c % FSTAGES;
      unsigned char* base = smem + (size_t)st * kFbiStage;
      tc::mbar_arrive_expect_tx(&full[st], kFbiStage);
      tc::bulk_g2s(base, Aimg + (size_t)c * 4 * (kFbiOp / sizeof(float)), 4 * kFbiOp, &full[st]);
#pragma unroll
      for (int f = 0; f < 2; ++f)
#pragma unroll
        for (int part = 0; part < 2; ++part) {
          const float* src =
              Bimg + (((((f * sh.qn[1] + mzl) * 2 + par) * ntile + nt) * 2 + part) * npair + t0 + 4 * c) * 512;
          tc::bulk_g2s(base + (4 + 2 * f + part) * kFbiOp, src, kFbiOp, &full[st]);
        }
    };
    // N = 256: the A image stacks the Re-part and Im-part rows, so one MMA fills both
    // accumulators of a field (half the instructions and a quarter less shared-memory
    // operand traffic than two 128-column MMAs)
    const uint32_t idesc = tc::idesc_f32acc(tc::kFmtTF32, FT, 2 * FT);
    int loaded = 0, fulled = 0, committed = 0, emptied = 0;  // chunks issued / observed
    bool ok = true;
    for (; loaded < FSTAGES && loaded < nchunk; ++loaded) load(loaded);
    for (int c = 0; c < nchunk && ok; ++c) {
      const int st = c % FSTAGES;
      if (!tc::mbar_wait_bounded(&full[st], (uint32_t)(c / FSTAGES) & 1u, tries)) {
        ok = false;
        break;
      }
      ++fulled;
      tc::fence_after_sync();
      const uint32_t base = tc::smem_u32(smem + (size_t)st * kFbiStage);
#pragma unroll
      for (int ks = 0; ks < 2; ++ks) {
#pragma unroll
        for (int f = 0; f < 2; ++f) {
          // transposed product psi^T = B_f A^T: the accumulator's lanes are p_z, its
          // columns p_x (Re part in the first 128, Im part in the next 128), so the
          // epilogue stores p_z-contiguous rows from registers
          const uint32_t d = tmem + (uint32_t)(2 * f * FT);
          const uint32_t ah = base + ks * 2 * kFbiALBO, al = ah + 2 * kFbiOp;
          const uint32_t bh = base + (4 + 2 * f) * kFbiOp + ks * 2 * kFbiLBO, bl = bh + kFbiOp;
          tc::mma_tf32(d, tc::smem_desc(bh, kFbiLBO, kFbiSBO), tc::smem_desc(ah, kFbiALBO, kFbiSBO), idesc,
                       (c > 0 || ks > 0) ? 1u : 0u);
          tc::mma_tf32(d, tc::smem_desc(bl, kFbiLBO, kFbiSBO), tc::smem_desc(ah, kFbiALBO, kFbiSBO), idesc, 1u);
          tc::mma_tf32(d, tc::smem_desc(bh, kFbiLBO, kFbiSBO), tc::smem_desc(al, kFbiALBO, kFbiSBO), idesc, 1u);
        }
      }
      tc::mma_commit(&empty[st]);
      ++committed;
      // refill the stage of the previous chunk once its MMAs are done
      if (c >= 1 && loaded < nchunk) {
        const int pc = c - 1;
        if (!tc::mbar_wait_bounded(&empty[pc % FSTAGES], (uint32_t)(pc / FSTAGES) & 1u, tries)) {
          ok = false;
          break;
        }
        emptied = pc + 1;
        load(loaded++);
      }
    }
    if (ok) {
      tc::mma_commit(done);  // arrives once every MMA of the CTA is complete
    } else {
      aborted_s = 1;
      atomicOr(status, kStatusTimeout);
      // nothing more is issued; wait, in order and with the full budget, for the copies and
      // the MMAs in flight (each barrier has at most one phase outstanding)
      for (int x = fulled; x < loaded; ++x)
        tc::mbar_wait_bounded(&full[x % FSTAGES], (uint32_t)(x / FSTAGES) & 1u, kFbiTries);
      for (int x = emptied; x < committed; ++x)
        tc::mbar_wait_bounded(&empty[x % FSTAGES], (uint32_t)(x / FSTAGES) & 1u, kFbiTries);
      tc::mbar_arrive(done);
    }
  }
  if (tid == 128) {  // the epilogue's constants (c(q) among them) while thread 0 feeds the tensor cores
    double q[2] = {gd.o[0] + (double)(sh.s[0] * (sh.qlo[0] + mxl)) * gd.h[0],
                   gd.o[1] + (double)(sh.s[1] * (sh.qlo[1] + mzl)) * gd.h[1]};
    const double cq = medium_value<2>(gd, C, q);
    const double hv = gd.h[0] * gd.h[1];
    h2_s = (float)(0.5 * hv);                 // psi_f = hv * acc; psi+ = psi0/2 + ...
    c1_s = (float)(0.5 * hv * sh.eps / cq);   // ... i (eps/(2 c(q) |p|)) hv acc1
  }
  const bool finished = tc::mbar_wait_bounded(done, 0u, tid == 0 ? kFbiTries : (tries > 0 ? tries : 1u));
  const bool ok = __syncthreads_and(finished) && aborted_s == 0;
  if (!ok && tid == 0 && aborted_s == 0) atomicOr(status, kStatusTimeout);
  tc::fence_after_sync();
  // epilogue: TMEM lane 32 quarter + l holds p_z column n0 + 32 quarter + l, TMEM column
  // j the p_x row m0 + j; a warp takes 64 of the rows, 16 at a time, and each of its
  // stores is one contiguous run of 32 p_z columns of a row (FP32 pairs)
  const int lane = tid & 31, quarter = warp & 3, part = warp >> 2;
  const float h2 = h2_s, c1 = c1_s;
  const float psx = psx_s, psz = psz_s;
  float2* out0 = psi + sh.psi_off + ql * sh.np;
  float2* out1 = psi_f1 + sh.psi_off + ql * sh.np;
  const int n = (int)n0 + 32 * quarter + lane;
  const bool nin = n < (int)nbz;
  const int mz = n - (int)(nbz / 2);
  const float pz = (float)mz * psz, pz2 = pz * pz;
  // this thread's values psi+ for the exact maximum below, in the stage buffers (free once
  // the MMAs are done): [value k][thread], NaN where no value was stored
  float2* vs = reinterpret_cast<float2*>(smem);
  float amax = 0.0f;  // largest |Re|, |Im| of the stored values (fmaxf leaves NaN out)
  if (ok) {
#pragma unroll 1
    for (int cb = FCOLS * part; cb < FCOLS * part + FCOLS; cb += 16) {
      if (m0 + cb >= nbx) break;  // uniform over the warp
      const uint32_t lane_base = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)cb;
      uint32_t r0r[16], r0i[16], r1r[16], r1i[16];
      tc::tmem_ld_32x32b_x16(lane_base, r0r);
      tc::tmem_ld_32x32b_x16(lane_base + FT, r0i);
      tc::tmem_ld_32x32b_x16(lane_base + 2 * FT, r1r);
      tc::tmem_ld_32x32b_x16(lane_base + 3 * FT, r1i);
      tc::tmem_ld_wait();
      tc::reg_fence16(r0r);
      tc::reg_fence16(r0i);
      tc::reg_fence16(r1r);
      tc::reg_fence16(r1i);
      const int mb = (int)m0 + cb;                 // p_x row of i = 0
      const float mxf0 = (float)(mb - (int)(nbx / 2));
      float2* vk = vs + (cb - FCOLS * part) * FNT + tid;
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int m = mb + i;
        const bool in = nin && m < (int)nbx;
        const float px = (mxf0 + (float)i) * psx;  // (float) mx, exactly
        // left-out p: the Nyquist index of either axis and p = 0 (as psi_plus<2>)
        const bool valid = m != 0 && n != 0 && !(m == (int)(nbx / 2) && mz == 0);
        const float rr = c1 * rsqrtf(fmaf(px, px, pz2));
        const float r = valid ? rr : 0.0f, hh = valid ? h2 : 0.0f;
        const float tx = -r * __uint_as_float(r1i[i]);
        const float ty = r * __uint_as_float(r1r[i]);
        const float ox = fmaf(hh, __uint_as_float(r0r[i]), tx);
        const float oy = fmaf(hh, __uint_as_float(r0i[i]), ty);
        if (in) {
          const int64_t jp = (int64_t)m * nbz + n;
          out0[jp] = make_float2(ox, oy);
          out1[jp] = make_float2(tx, ty);
          amax = fmaxf(amax, fmaxf(fabsf(ox), fabsf(oy)));
        }
        vk[i * FNT] = in ? make_float2(ox, oy) : make_float2(__int_as_float(0x7fc00000), 0.0f);
      }
    }
  }
  // the largest FP64 |psi+|^2 of the stored values (as the selection computes it). Scaled
  // by s = 2^k so that s max(|Re|, |Im|) lies in [1, 2), the FP32 squares near the largest
  // one are within 2^-22 of the exact scaled squares, so only values within 1e-6 of the
  // largest FP32 square can hold the maximum; only those are squared in FP64. If the
  // components are all zero the maximum is +0; if the largest is below 2^-100 or not
  // finite, every stored value is squared in FP64.
  unsigned long long mymax = 0ull;  // bits of the largest |psi+|^2 (non-negative doubles order as integers)
  if (ok && amax != 0.0f) {
    const bool scaled = amax >= 0x1p-100f && amax < INFINITY;
    const float sc = scaled ? ldexpf(1.0f, -ilogbf(amax)) : 1.0f;
    const int64_t rows = nbx - (m0 + FCOLS * part);  // rows of this warp's part that exist
    const int nk = rows >= FCOLS ? FCOLS : (rows > 0 ? (int)rows : 0);
    float fmx = 0.0f;
    if (scaled) {
#pragma unroll 4
      for (int k = 0; k < nk; ++k) {
        const float2 v = vs[k * FNT + tid];
        const float sx = v.x * sc, sy = v.y * sc;
        fmx = fmaxf(fmx, fmaf(sx, sx, sy * sy));
      }
    }
    const float lim = scaled ? 0.999999f * fmx : 0.0f;
#pragma unroll 4
    for (int k = 0; k < nk; ++k) {
      const float2 v = vs[k * FNT + tid];
      const float sx = v.x * sc, sy = v.y * sc;
      if (fmaf(sx, sx, sy * sy) >= lim) {  // false for NaN (no value stored)
        const double2 o = make_double2(widen_f32(v.x), widen_f32(v.y));
        const unsigned long long a2 = (unsigned long long)__double_as_longlong(abs2_rn(o));
        if (a2 <= 0x7ff0000000000000ull && a2 > mymax) mymax = a2;  // NaN left out, as fmax does
      }
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long o = __shfl_xor_sync(0xffffffffu, mymax, off);
    mymax = o > mymax ? o : mymax;
  }
  if ((tid & 31) == 0) atomic_max_nonneg(max2 + s, __longlong_as_double((long long)mymax));
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 4 * FT);
}

}  // namespace

cudaError_t launch_support_bbox(fga_plan_s* p, const double* u0, const double* u1) {
  int n = p->nshots * p->grid.dim * 2;
  k_bbox_init<<<(n + 255) / 256, 256, 0, p->stream>>>(p->d_bbox, n);
  int64_t blocks = (p->grid.npts + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  k_support_bbox<<<dim3((unsigned)blocks, p->nshots), 256, 0, p->stream>>>(p->grid, u0, u1,
                                                                          p->d_bbox);
  p->launches += 2;
  return cudaGetLastError();
}

namespace {
// One thread per shot: the active q rectangle of the support in bbox, computed as
// fga_decompose computes it on the host, against the one the plan holds.
__global__ void k_check_shapes(GridDev gd, const ShotDev* __restrict__ shots, int nshots,
                               const int* __restrict__ bbox, int* status) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nshots) return;
  const ShotDev& sh = shots[s];
  const int d = gd.dim;
  bool empty = false;
  int64_t qlo[kMaxDim] = {0, 0, 0}, qn[kMaxDim] = {0, 0, 0};
  for (int k = 0; k < d; ++k) {
    const int lo = bbox[(s * d + k) * 2], hi = bbox[(s * d + k) * 2 + 1];
    if (hi < 0) empty = true;
    if (gd.periodic[k]) {
      qlo[k] = 0;
      qn[k] = sh.nq[k];
    } else {
      const int64_t half = sh.nb[k] / 2;
      int64_t mlo = (int64_t)ceil((double)(lo - half + 1) / sh.s[k]);
      int64_t mhi = (int64_t)floor((double)(hi + half) / sh.s[k]);
      mlo = mlo > 0 ? mlo : 0;
      mhi = mhi < sh.nq[k] - 1 ? mhi : sh.nq[k] - 1;
      qlo[k] = mlo;
      qn[k] = mhi - mlo + 1 > 0 ? mhi - mlo + 1 : 0;
    }
  }
  bool same = true;
  for (int k = 0; k < d; ++k) {
    if (empty) qn[k] = 0;
    same = same && qn[k] == sh.qn[k] && (qn[k] == 0 || qlo[k] == sh.qlo[k]);
  }
  if (!same) atomicOr(status, kStatusShape);
}
}  // namespace

cudaError_t launch_check_shapes(fga_plan_s* p) {
  k_check_shapes<<<(p->nshots + 127) / 128, 128, 0, p->stream>>>(p->grid, p->d_shots, p->nshots,
                                                                 p->d_bbox, p->d_status);
  p->launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_fbi(fga_plan_s* p, const double* u0, const double* u1) {
  cudaMemsetAsync(p->d_max2, 0, sizeof(unsigned long long) * p->nshots, p->stream);
  int64_t maxM = 0, maxN = 0, maxQ = 0, maxTiles = 0;
  const int D = p->grid.dim;
  for (const auto& sh : p->shots) {
    int64_t M = (D == 2) ? sh.nrows * sh.qn[1] : sh.qn[0];
    if (sh.qn[0] == 0 || (D == 2 && sh.qn[1] == 0)) continue;
    maxM = std::max(maxM, M);
    maxN = std::max<int64_t>(maxN, sh.nb[D - 1]);
    if (D == 2) {
      maxQ = std::max(maxQ, sh.qn[0] * sh.qn[1]);
      maxTiles = std::max<int64_t>(maxTiles, ((sh.nb[0] + BM - 1) / BM) * ((sh.nb[1] + BN - 1) / BN));
    }
  }
  if (D == 3) {
    bool any = false;
    for (const auto& sh : p->shots) any = any || sh.qn[0] * sh.qn[1] * sh.qn[2] > 0;
    if (!any) return cudaSuccess;
    const unsigned blocks = 1024;
    k_fbi3_stage1<<<dim3(blocks, p->nshots), 256, 0, p->stream>>>(p->grid, p->d_shots, u0, u1, p->d_g1);
    k_fbi3_stage2<<<dim3(blocks, p->nshots), 256, 0, p->stream>>>(p->d_shots, p->d_g1, p->d_g2);
    int64_t qmax = 0;
    for (const auto& sh : p->shots) qmax = std::max<int64_t>(qmax, sh.qn[0] * sh.qn[1] * sh.qn[2]);
    if (qmax >= ((int64_t)1 << 31)) return cudaErrorInvalidConfiguration;
    k_fbi3_stage3<<<dim3((unsigned)qmax, p->nshots), 256, 0, p->stream>>>(p->grid, p->d_shots, p->d_coef,
                                                                          p->d_g2, p->d_psi, p->d_psi_f1,
                                                                          p->d_max2);
    p->launches += 3;
    return cudaGetLastError();
  }
  if (maxM == 0) return cudaSuccess;
  dim3 g1grid((unsigned)((maxN + BN - 1) / BN), (unsigned)((maxM + BM - 1) / BM), p->nshots);
  if (g1grid.y > 65535) return cudaErrorInvalidConfiguration;
  if (D == 1) {
    k_fbi_stage1<1><<<g1grid, NT, 0, p->stream>>>(p->grid, p->d_shots, u0, u1, p->d_coef, p->d_g1,
                                                  p->d_psi, p->d_psi_f1, p->d_max2, 0);
    p->launches += 1;
    return cudaGetLastError();
  }
  if (p->precision == FGA_MIXED_TF32X3)
    k_fbi_stage1<2, float><<<g1grid, NT, 0, p->stream>>>(p->grid, p->d_shots, u0, u1, p->d_coef, p->d_g1,
                                                        p->d_psi, p->d_psi_f1, p->d_max2, 1);
  else
    k_fbi_stage1<2><<<g1grid, NT, 0, p->stream>>>(p->grid, p->d_shots, u0, u1, p->d_coef, p->d_g1,
                                                  p->d_psi, p->d_psi_f1, p->d_max2, 0);
  if (maxQ > 65535) return cudaErrorInvalidConfiguration;
  p->launches += 2;
  if (p->precision == FGA_MIXED_TF32X3) {
    static bool attr_set = false;
    if (!attr_set) {
      cudaError_t e = cudaFuncSetAttribute(k_fbi_stage2_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)kFbiSmem);
      if (e != cudaSuccess) return e;
      attr_set = true;
    }
    int64_t tiles = 0;
    for (const auto& sh : p->shots)
      tiles = std::max<int64_t>(tiles, ((sh.nb[0] + FT - 1) / FT) * ((sh.nb[1] + FT - 1) / FT));
    dim3 tgrid((unsigned)tiles, (unsigned)maxQ, p->nshots);
    k_fbi_stage2_tc<<<tgrid, FNT, kFbiSmem, p->stream>>>(p->grid, p->d_shots, p->d_coef, p->d_g1,
                                                        reinterpret_cast<float2*>(p->d_psi),
                                                        reinterpret_cast<float2*>(p->d_psi_f1), p->d_max2,
                                                        p->d_status,
                                                        p->wait_tries >= 0 ? (uint32_t)p->wait_tries
                                                                           : kFbiTries);
    return cudaGetLastError();
  }
  dim3 g2grid((unsigned)maxTiles, (unsigned)maxQ, p->nshots);
  k_fbi_stage2<<<g2grid, NT, 0, p->stream>>>(p->grid, p->d_shots, p->d_coef, p->d_g1, p->d_psi,
                                             p->d_psi_f1, p->d_max2);
  return cudaGetLastError();
}

}  // namespace fga
