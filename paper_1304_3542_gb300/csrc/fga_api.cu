// C ABI of libfga (declared in include/fga.h): plan set-up, validation, device
// memory, and the order of the three steps of the Algorithm section.
#include <algorithm>
#include <cstdint>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "fga_internal.cuh"

using fga::GridDev;
using fga::ShotDev;

namespace {

thread_local std::string g_plan_error;

const double kPi = 3.14159265358979323846;

fga_status fail(fga_plan_s* p, fga_status st, const std::string& msg, bool mark_failed = false) {
  if (p) {
    p->last_error = msg;
    if (mark_failed) p->failed = true;
  } else {
    g_plan_error = msg;
  }
  return st;
}

#define CUDA_OR_FAIL(p, call)                                                             \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) {                                                              \
      fga_status st_ = (e_ == cudaErrorMemoryAllocation) ? FGA_ERR_OOM : FGA_ERR_CUDA;    \
      return fail(p, st_, std::string(#call) + ": " + cudaGetErrorString(e_), true);      \
    }                                                                                     \
  } while (0)

bool is_device_ptr(const void* ptr) {
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, ptr);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <typename T>
cudaError_t grow(T** ptr, size_t* cap, size_t need) {
  if (need <= *cap && *ptr) return cudaSuccess;
  if (*ptr) cudaFree(*ptr);
  *ptr = nullptr;
  *cap = 0;
  size_t n = std::max<size_t>(need, 1);
  cudaError_t e = cudaMalloc((void**)ptr, n * sizeof(T));
  if (e == cudaSuccess) *cap = n;
  return e;
}

__global__ void k_check_velocity(const double* c, int64_t n, int* bad) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double v = c[i];
    if (!(v > 0.0) || !isfinite(v)) atomicOr(bad, 1);
  }
}

// Window-DFT matrix of one axis: E[jp][j] = w(r_j) exp(-i p_jp r_j/eps), with
// p_jp r_j/eps = 2 pi m r/n_b for the integers m = jp - n_b/2, r = j - n_b/2
// (reduced mod n_b before scaling, so the angle is exact to rounding).
std::vector<double> window_dft(int nb, double h, double eps, bool periodic, double L) {
  std::vector<double> E((size_t)nb * nb * 2);
  std::vector<double> w(nb);
  for (int j = 0; j < nb; ++j) {
    double r = (double)(j - nb / 2) * h;
    if (periodic) {
      double s = 0.0;
      for (int l = -2; l <= 2; ++l) s += std::exp(-(r + l * L) * (r + l * L) / (2.0 * eps));
      w[j] = s;
    } else {
      w[j] = std::exp(-r * r / (2.0 * eps));
    }
  }
  for (int jp = 0; jp < nb; ++jp) {
    long long m = jp - nb / 2;
    for (int j = 0; j < nb; ++j) {
      long long r = j - nb / 2;
      long long k = ((m * r) % nb + nb) % nb;
      double ang = 2.0 * kPi * (double)k / (double)nb;
      E[((size_t)jp * nb + j) * 2 + 0] = w[j] * std::cos(ang);
      E[((size_t)jp * nb + j) * 2 + 1] = -w[j] * std::sin(ang);
    }
  }
  return E;
}

fga_status check_usable(fga_plan_s* p);

// After a replay of the pipeline graph the counts live on the device: bring the host's
// copies (per-shot segments, G) up to date before anything else reads them.
fga_status refresh_host_counts(fga_plan_s* p) {
  if (!p->pipe_host_stale) return FGA_OK;
  p->pipe_host_stale = false;
  std::vector<fga::ShotDev> dev(p->nshots);
  int64_t gm[2] = {0, 0};
  CUDA_OR_FAIL(p, cudaMemcpyAsync(dev.data(), p->d_shots, sizeof(fga::ShotDev) * p->nshots,
                                  cudaMemcpyDeviceToHost, p->stream));
  CUDA_OR_FAIL(p, cudaMemcpyAsync(gm, p->d_gm, sizeof(gm), cudaMemcpyDeviceToHost, p->stream));
  CUDA_OR_FAIL(p, cudaStreamSynchronize(p->stream));
  for (int s = 0; s < p->nshots; ++s) {
    p->shots[s].g_off = dev[s].g_off;
    p->shots[s].g_cnt = dev[s].g_cnt;
  }
  p->G = gm[0];
  return FGA_OK;
}

fga_status check_usable(fga_plan_s* p) {
  if (!p) return fail(nullptr, FGA_ERR_INVALID, "plan is NULL");
  if (p->failed) return FGA_ERR_STATE;
  return refresh_host_counts(p);
}

fga_status read_status(fga_plan_s* p) {
  int st = 0;
  CUDA_OR_FAIL(p, cudaMemcpyAsync(&st, p->d_status, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
  CUDA_OR_FAIL(p, cudaStreamSynchronize(p->stream));
  if (st & fga::kStatusNumeric)
    return fail(p, FGA_ERR_NUMERIC, "a ray met |P| = 0, det Z = 0 or a non-finite value", true);
  if (st & fga::kStatusShape)
    return fail(p, FGA_ERR_CAPACITY,
                "the data's support gives other active q rectangles than the pipeline graph was "
                "captured for (run fga_run_pipeline on a new plan)", true);
  if (st & fga::kStatusCapacity) return fail(p, FGA_ERR_CAPACITY, "a plan capacity was exceeded", true);
  if (st & fga::kStatusTimeout)
    return fail(p, FGA_ERR_TIMEOUT, "a bounded tensor-core completion wait gave up", true);
  return FGA_OK;
}

// One grid line of the interpolating prefilter, v[i * stride], i < n, in place: the
// tridiagonal system (C_{i-1} + 4 C_i + C_{i+1})/6 = c_i with the clamped spline's end
// rows (5 C_0 + C_1)/6, (C_{n-2} + 5 C_{n-1})/6 on an open axis (Thomas algorithm), or
// wrapped indices on a periodic axis (Thomas on the matrix with its corners removed and
// the Sherman-Morrison correction for them). w, x, z: scratch of n values.
void prefilter_line(double* v, int64_t n, int64_t stride, bool periodic, std::vector<double>& w,
                    std::vector<double>& x, std::vector<double>& z) {
  // rows scaled by 6: sub- and super-diagonal 1, diagonal 4 (5 at the ends of an open axis)
  if (!periodic) {
    double m = 5.0;
    w[0] = 1.0 / m;
    x[0] = 6.0 * v[0] / m;
    for (int64_t i = 1; i < n; ++i) {
      m = (i == n - 1 ? 5.0 : 4.0) - w[i - 1];
      w[i] = 1.0 / m;
      x[i] = (6.0 * v[i * stride] - x[i - 1]) / m;
    }
    for (int64_t i = n - 2; i >= 0; --i) x[i] -= w[i] * x[i + 1];
    for (int64_t i = 0; i < n; ++i) v[i * stride] = x[i];
    return;
  }
  // Sherman-Morrison: A = T + u v^T, u = (gamma, 0, ..., 0, 1), v = (1, 0, ..., 0, 1/gamma),
  // gamma = -4, so that T (tridiagonal, diagonal entries 4 - gamma first and 4 - 1/gamma
  // last) holds no corners; solve T x = rhs and T z = u, then
  // x -= z (x_0 + x_{n-1}/gamma)/(1 + z_0 + z_{n-1}/gamma)
  const double gamma = -4.0;
  auto solve_t = [&](const double* rhs, int64_t rstride, std::vector<double>& out) {
    double m = 4.0 - gamma;
    w[0] = 1.0 / m;
    out[0] = rhs[0] / m;
    for (int64_t i = 1; i < n; ++i) {
      m = (i == n - 1 ? 4.0 - 1.0 / gamma : 4.0) - w[i - 1];
      w[i] = 1.0 / m;
      out[i] = (rhs[i * rstride] - out[i - 1]) / m;
    }
    for (int64_t i = n - 2; i >= 0; --i) out[i] -= w[i] * out[i + 1];
  };
  std::vector<double> rhs((size_t)n), u((size_t)n, 0.0);
  for (int64_t i = 0; i < n; ++i) rhs[i] = 6.0 * v[i * stride];
  u[0] = gamma;
  u[n - 1] = 1.0;
  solve_t(rhs.data(), 1, x);
  solve_t(u.data(), 1, z);
  const double f = (x[0] + x[n - 1] / gamma) / (1.0 + z[0] + z[n - 1] / gamma);
  for (int64_t i = 0; i < n; ++i) v[i * stride] = x[i] - f * z[i];
}

// The prefilter on a whole C-order grid, axis by axis.
void prefilter_grid(int d, const int64_t* n, const int* periodic, double* c) {
  int64_t total = 1;
  for (int k = 0; k < d; ++k) total *= n[k];
  for (int k = 0; k < d; ++k) {
    int64_t stride = 1;
    for (int j = k + 1; j < d; ++j) stride *= n[j];
    std::vector<double> w((size_t)n[k]), x((size_t)n[k]), z((size_t)n[k]);
    const int64_t outer = total / (n[k] * stride);
    for (int64_t o = 0; o < outer; ++o)
      for (int64_t in = 0; in < stride; ++in)
        prefilter_line(c + o * n[k] * stride + in, n[k], stride, periodic[k] != 0, w, x, z);
  }
}

}  // namespace

namespace fga {
void set_unbound_error(const std::string& msg) { g_plan_error = msg; }
}  // namespace fga

extern "C" {

const char* fga_status_string(fga_status s) {
  switch (s) {
    case FGA_OK: return "ok";
    case FGA_ERR_INVALID: return "invalid argument";
    case FGA_ERR_OOM: return "out of device memory";
    case FGA_ERR_CUDA: return "CUDA error";
    case FGA_ERR_TIMEOUT: return "device wait timed out";
    case FGA_ERR_STATE: return "call out of order or plan failed";
    case FGA_ERR_NUMERIC: return "numerical failure on a ray";
    case FGA_ERR_CAPACITY: return "capacity exceeded";
  }
  return "unknown status";
}

const char* fga_last_error(fga_plan_t plan) {
  return plan ? plan->last_error.c_str() : g_plan_error.c_str();
}

fga_status fga_destroy(fga_plan_t p) {
  if (!p) return FGA_OK;
  cudaStreamSynchronize(p->stream);
  void* bufs[] = {p->d_coef, p->d_medtab, p->d_shots, p->d_in0, p->d_bbox, p->d_psi, p->d_g1,
                  p->d_max2, p->d_blk, p->d_counts, p->d_blk_first, p->d_gshot, p->d_gq, p->d_gp,
                  p->d_gpsi, p->d_state, p->d_gcoef, p->d_tile_off,
                  p->d_tile_list, p->d_bin_off, p->d_seg_off, p->d_partial, p->d_out, p->d_status,
                  p->d_steps, p->d_rx, p->d_rx_off, p->d_rx_perm, p->d_traces, p->d_gsteps, p->d_g2,
                  p->d_topk, p->d_topk_hist, p->d_blk_eq,
                  p->d_adj_order, p->d_adj_bucket,
                  p->d_run_geo, p->d_run_axis, p->d_run_off, p->d_resid_int,
                  p->d_psi_f1, p->d_gpsi_f1, p->d_adj_scratch, p->d_grad, p->d_resid,
                  p->d_part, p->d_gm, p->d_ganc, p->d_ray_bucket, p->d_rng};
  for (void* b : bufs)
    if (b) cudaFree(b);
  for (double* e : p->E)
    if (e) cudaFree(e);
  for (void* e : p->mixed_tabs)
    if (e) cudaFree(e);
  for (auto& ev : p->ev)
    if (ev) cudaEventDestroy(ev);
  if (p->graph_exec) cudaGraphExecDestroy(p->graph_exec);
  if (p->pipe_exec) cudaGraphExecDestroy(p->pipe_exec);
  delete p;
  return FGA_OK;
}

fga_status fga_plan(const fga_config* cfg, const double* velocity, void* stream, fga_plan_t* out) {
  if (!out) return fail(nullptr, FGA_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!cfg || !velocity) return fail(nullptr, FGA_ERR_INVALID, "cfg or velocity is NULL");
  const int d = cfg->dim;
  if (d < 1 || d > fga::kMaxDim) return fail(nullptr, FGA_ERR_INVALID, "dim must be 1, 2 or 3");
  if (cfg->nshots < 1 || cfg->nshots > fga::kMaxShots)
    return fail(nullptr, FGA_ERR_INVALID, "nshots out of range");
  if (!cfg->eps) return fail(nullptr, FGA_ERR_INVALID, "eps is NULL");
  if (cfg->precision != FGA_FP64 && cfg->precision != FGA_MIXED_TF32X3)
    return fail(nullptr, FGA_ERR_INVALID, "precision must be FGA_FP64 or FGA_MIXED_TF32X3");
  if (cfg->precision == FGA_MIXED_TF32X3) {
    if (d != 2) return fail(nullptr, FGA_ERR_INVALID, "FGA_MIXED_TF32X3 needs a 2D grid");
    if (cfg->periodic[0] || cfg->periodic[1])
      return fail(nullptr, FGA_ERR_INVALID, "FGA_MIXED_TF32X3 needs open (non-periodic) axes");
  }
  if (!(cfg->dt > 0.0) || !(cfg->T >= 0.0) || !std::isfinite(cfg->T))
    return fail(nullptr, FGA_ERR_INVALID, "need T >= 0 and dt > 0");
  double steps = cfg->T / cfg->dt;
  if (std::fabs(steps - std::round(steps)) > 1e-9 * std::max(1.0, steps))
    return fail(nullptr, FGA_ERR_INVALID, "T/dt must be an integer");
  if (steps > 2147483647.0) return fail(nullptr, FGA_ERR_INVALID, "T/dt must be below 2^31");
  if (!(cfg->kappa > 0.0) || !std::isfinite(cfg->kappa))
    return fail(nullptr, FGA_ERR_INVALID, "kappa must be > 0");
  if (!(cfg->tau >= 0.0) || !std::isfinite(cfg->tau))
    return fail(nullptr, FGA_ERR_INVALID, "tau must be >= 0");
  if (cfg->keep_n < 0) return fail(nullptr, FGA_ERR_INVALID, "keep_n must be >= 0");
  if (cfg->interp != FGA_BSPLINE_APPROX && cfg->interp != FGA_BSPLINE_INTERP)
    return fail(nullptr, FGA_ERR_INVALID, "interp must be FGA_BSPLINE_APPROX or FGA_BSPLINE_INTERP");
  if (cfg->z_method != FGA_Z_DYNAMIC && cfg->z_method != FGA_Z_DIVIDED)
    return fail(nullptr, FGA_ERR_INVALID, "z_method must be FGA_Z_DYNAMIC or FGA_Z_DIVIDED");
  if (cfg->z_method == FGA_Z_DIVIDED) {
    if (d > 2) return fail(nullptr, FGA_ERR_INVALID, "FGA_Z_DIVIDED is supported in 1D and 2D");
    if (!(cfg->dz_eta > 0.0 && cfg->dz_eta < 1.0))
      return fail(nullptr, FGA_ERR_INVALID, "FGA_Z_DIVIDED needs 0 < dz_eta < 1");
  }
  GridDev gd;
  std::memset(&gd, 0, sizeof(gd));
  gd.dim = d;
  gd.npts = 1;
  for (int k = 0; k < d; ++k) {
    if (cfg->n[k] < 4 || cfg->n[k] > (int64_t)1 << 30)
      return fail(nullptr, FGA_ERR_INVALID, "grid size out of range");
    if (!(cfg->h[k] > 0.0) || !std::isfinite(cfg->h[k]) || !std::isfinite(cfg->origin[k]))
      return fail(nullptr, FGA_ERR_INVALID, "grid spacing must be finite and > 0");
    gd.n[k] = cfg->n[k];
    gd.h[k] = cfg->h[k];
    gd.o[k] = cfg->origin[k];
    gd.inv_h[k] = 1.0 / cfg->h[k];
    gd.mo[k] = -cfg->origin[k] * gd.inv_h[k];
    gd.periodic[k] = cfg->periodic[k] ? 1 : 0;
    gd.L[k] = gd.periodic[k] ? (double)cfg->n[k] * cfg->h[k] : 0.0;
    gd.npts *= cfg->n[k];
  }
  for (int k = d; k < fga::kMaxDim; ++k) {
    gd.n[k] = 1;
    gd.h[k] = gd.inv_h[k] = 1.0;
  }
  fga_plan_s* p = new fga_plan_s();
  p->grid = gd;
  p->nshots = cfg->nshots;
  p->T = cfg->T;
  p->dt = cfg->dt;
  p->nsteps = (int64_t)std::llround(steps);
  p->kappa = cfg->kappa;
  p->tau = cfg->tau;
  p->precision = cfg->precision;
  p->integrate_exited = cfg->integrate_exited ? 1 : 0;
  p->keep_n = cfg->keep_n;
  p->z_method = cfg->z_method;
  p->interp = cfg->interp;
  p->dz_eta = cfg->z_method == FGA_Z_DIVIDED ? cfg->dz_eta : 0.0;
  p->stream = (cudaStream_t)stream;
  p->nfields = fga::state_fields(d);
  const int TS = cfg->precision == FGA_MIXED_TF32X3 ? fga::tile_edge_tc() : fga::tile_edge(d);
  for (int k = 0; k < fga::kMaxDim; ++k) p->grid.tile[k] = TS;
  int64_t tile_off = 0;
  p->shots.resize(cfg->nshots);
  for (int s = 0; s < cfg->nshots; ++s) {
    ShotDev& sh = p->shots[s];
    std::memset(&sh, 0, sizeof(sh));
    double eps = cfg->eps[s];
    if (!(eps > 0.0) || !std::isfinite(eps)) {
      delete p;
      return fail(nullptr, FGA_ERR_INVALID, "eps must be finite and > 0");
    }
    sh.eps = eps;
    sh.sqrt_eps = std::sqrt(eps);
    sh.inv_eps = 1.0 / eps;
    sh.norm = std::pow(2.0 * kPi * eps, -1.5 * d);
    sh.W = 1.0;
    sh.np = 1;
    for (int k = 0; k < d; ++k) {
      int sk = cfg->q_stride ? cfg->q_stride[s * d + k] : (int)std::lround(0.5 * sh.sqrt_eps / gd.h[k]);
      if (sk < 1) sk = 1;
      int nbk;
      if (gd.periodic[k]) {
        if (!cfg->q_stride)
          while (gd.n[k] % sk) --sk;
        nbk = cfg->box ? cfg->box[s * d + k] : (int)gd.n[k];
        if (nbk != gd.n[k] || gd.n[k] % sk) {
          delete p;
          return fail(nullptr, FGA_ERR_INVALID,
                      "on a periodic axis the box must be one period and n a multiple of the q-stride");
        }
        if (cfg->kappa * sh.sqrt_eps > 2.0 * gd.L[k]) {
          delete p;
          return fail(nullptr, FGA_ERR_INVALID, "kappa sqrt(eps) must not exceed two periods");
        }
      } else {
        nbk = cfg->box ? cfg->box[s * d + k]
                       : 32 * (((int)std::ceil(12.0 * sh.sqrt_eps / gd.h[k]) + 31) / 32);
      }
      if (nbk < 2 || (nbk & 1) || nbk > 4096) {
        delete p;
        return fail(nullptr, FGA_ERR_INVALID, "box must be even, >= 2 and <= 4096");
      }
      if (cfg->precision == FGA_MIXED_TF32X3 && k == 0 && nbk % 8 != 0) {
        delete p;
        return fail(nullptr, FGA_ERR_INVALID,
                    "FGA_MIXED_TF32X3 needs boxes of a multiple of 8 points along the first axis");
      }
      sh.s[k] = sk;
      sh.nb[k] = nbk;
      sh.nq[k] = gd.periodic[k] ? gd.n[k] / sk : (gd.n[k] - 1) / sk + 1;
      sh.pscale[k] = 2.0 * kPi * eps / ((double)nbk * gd.h[k]);
      sh.W *= (double)sk * gd.h[k] * sh.pscale[k];
      sh.np *= nbk;
      sh.ntile[k] = (int)((gd.n[k] + p->grid.tile[k] - 1) / p->grid.tile[k]);
    }
    if (sh.np > ((int64_t)1 << 31) - 1 - fga::kScanBlock) {
      delete p;
      return fail(nullptr, FGA_ERR_INVALID, "a box of 2^31 or more points");
    }
    sh.fd_np = fga::make_fastdiv((uint32_t)sh.np);
    sh.fd_nbl = fga::make_fastdiv((uint32_t)sh.nb[d - 1]);
    sh.fd_nb12 = fga::make_fastdiv((uint32_t)(d == 3 ? sh.nb[1] * sh.nb[2] : 1));
    sh.tile_off = tile_off;
    int64_t nt = 1;
    for (int k = 0; k < d; ++k) nt *= sh.ntile[k];
    tile_off += nt;
  }
  p->ntiles = tile_off;
  // device buffers that do not depend on the data
  cudaError_t e;
#define PLAN_CUDA(call)                                                              \
  do {                                                                               \
    e = (call);                                                                      \
    if (e != cudaSuccess) {                                                          \
      std::string m_ = std::string(#call) + ": " + cudaGetErrorString(e);            \
      fga_destroy(p);                                                                \
      return fail(nullptr, e == cudaErrorMemoryAllocation ? FGA_ERR_OOM : FGA_ERR_CUDA, m_); \
    }                                                                                \
  } while (0)
  PLAN_CUDA(cudaMalloc(&p->d_coef, sizeof(double) * gd.npts));
  PLAN_CUDA(cudaMemcpyAsync(p->d_coef, velocity, sizeof(double) * gd.npts, cudaMemcpyDefault,
                            p->stream));
  PLAN_CUDA(cudaMalloc(&p->d_status, sizeof(int)));
  PLAN_CUDA(cudaMalloc(&p->d_steps, 2 * sizeof(unsigned long long)));
  PLAN_CUDA(cudaMemsetAsync(p->d_status, 0, sizeof(int), p->stream));
  k_check_velocity<<<256, 256, 0, p->stream>>>(p->d_coef, gd.npts, p->d_status);
  p->launches += 1;
  int bad = 0;
  PLAN_CUDA(cudaMemcpyAsync(&bad, p->d_status, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
  PLAN_CUDA(cudaStreamSynchronize(p->stream));
  if (bad) {
    fga_destroy(p);
    return fail(nullptr, FGA_ERR_INVALID, "velocity must be finite and > 0 everywhere");
  }
  if (p->interp == FGA_BSPLINE_INTERP) {
    // the samples were checked; the coefficients are their interpolating prefilter
    std::vector<double> hc((size_t)gd.npts);
    PLAN_CUDA(cudaMemcpyAsync(hc.data(), p->d_coef, sizeof(double) * gd.npts,
                              cudaMemcpyDeviceToHost, p->stream));
    PLAN_CUDA(cudaStreamSynchronize(p->stream));
    prefilter_grid(d, gd.n, gd.periodic, hc.data());
    PLAN_CUDA(cudaMemcpyAsync(p->d_coef, hc.data(), sizeof(double) * gd.npts,
                              cudaMemcpyHostToDevice, p->stream));
    PLAN_CUDA(cudaStreamSynchronize(p->stream));
  }
  PLAN_CUDA(cudaMalloc(&p->d_medtab, sizeof(double) * fga::medium_table_doubles(p->grid)));
  p->grid.tab = p->d_medtab;
  PLAN_CUDA(fga::launch_medium_table(p));
  PLAN_CUDA(cudaMemsetAsync(p->d_status, 0, sizeof(int), p->stream));
  p->E.assign((size_t)cfg->nshots * d, nullptr);
  for (int s = 0; s < cfg->nshots; ++s) {
    for (int k = 0; k < d; ++k) {
      ShotDev& sh = p->shots[s];
      std::vector<double> E = window_dft(sh.nb[k], gd.h[k], sh.eps, gd.periodic[k] != 0, gd.L[k]);
      double* dE = nullptr;
      PLAN_CUDA(cudaMalloc(&dE, sizeof(double) * E.size()));
      p->E[(size_t)s * d + k] = dE;
      PLAN_CUDA(cudaMemcpy(dE, E.data(), sizeof(double) * E.size(), cudaMemcpyHostToDevice));
      sh.E[k] = reinterpret_cast<const double2*>(dE);
      if (k == 0 && cfg->precision == FGA_MIXED_TF32X3) {
        // A operands of the tensor-core stage 2: Re-part rows (Re E, -Im E) and Im-part rows
        // (Im E, Re E) over K = 2 jx, each split into a TF32 head and an FP32 tail, laid
        // out as the shared-memory image one bulk copy fills per K chunk of 8 complex jx,
        // the Re-part and Im-part rows stacked as one 256-row operand:
        // [m tile of 128 p_x][chunk][head, tail][K quad 4][8-row group 32: Re part 0..15,
        // Im part 16..31][row 8][4 floats], rows past n_b zero (fga::fbi_a_image_floats)
        const int nb = sh.nb[0];
        const int mtiles = (nb + 127) / 128, nchunk = nb / 8;
        std::vector<float> A((size_t)mtiles * nchunk * 4 * 4 * 512, 0.0f);
        auto split = [](double v, float& hi, float& lo) {
          float f = (float)v;
          uint32_t bits;
          std::memcpy(&bits, &f, sizeof(bits));
          bits &= 0xFFFFE000u;
          std::memcpy(&hi, &bits, sizeof(hi));
          lo = (float)(v - (double)hi);
        };
        for (int px = 0; px < nb; ++px)
          for (int jx = 0; jx < nb; ++jx) {
            const double er = E[((size_t)px * nb + jx) * 2], ei = E[((size_t)px * nb + jx) * 2 + 1];
            const double vals[2][2] = {{er, -ei}, {ei, er}};
            const int mt = px / 128, row = px % 128, chunk = jx / 8, quad = (jx % 8) / 2, slot = jx % 2;
            for (int part = 0; part < 2; ++part)
              for (int c = 0; c < 2; ++c) {
                float hi, lo;
                split(vals[part][c], hi, lo);
                for (int hl = 0; hl < 2; ++hl) {
                  const size_t at =
                      ((((((size_t)mt * nchunk + chunk) * 2 + hl) * 4 + quad) * 32 + 16 * part +
                        row / 8) * 8 + row % 8) * 4 + 2 * slot + c;
                  A[at] = hl == 0 ? hi : lo;
                }
              }
          }
        float* dA = nullptr;
        PLAN_CUDA(cudaMalloc(&dA, sizeof(float) * A.size()));
        p->mixed_tabs.push_back(dA);
        PLAN_CUDA(cudaMemcpy(dA, A.data(), sizeof(float) * A.size(), cudaMemcpyHostToDevice));
        sh.Etc = dA;
      }
    }
  }
  PLAN_CUDA(cudaMalloc(&p->d_shots, sizeof(ShotDev) * cfg->nshots));
  PLAN_CUDA(cudaMalloc(&p->d_bbox, sizeof(int) * cfg->nshots * d * 2));
  PLAN_CUDA(cudaMalloc(&p->d_max2, sizeof(unsigned long long) * cfg->nshots));
  PLAN_CUDA(cudaMalloc(&p->d_counts, sizeof(int64_t) * cfg->nshots));
  PLAN_CUDA(cudaMalloc(&p->d_blk_first, sizeof(int64_t) * (cfg->nshots + 1)));
  PLAN_CUDA(cudaMalloc(&p->d_tile_off, sizeof(int64_t) * (p->ntiles + 1)));
  PLAN_CUDA(cudaMalloc(&p->d_seg_off, sizeof(int64_t) * (p->ntiles + 1)));
  for (auto& ev : p->ev) PLAN_CUDA(cudaEventCreate(&ev));
#undef PLAN_CUDA
  *out = p;
  return FGA_OK;
}

// Device arrays of the Gaussian list and the ray state for at least cap Gaussians.
static fga_status alloc_gaussians(fga_plan_s* p, size_t need) {
  if (need <= p->g_cap && p->d_gshot) return FGA_OK;
  const size_t cap = std::max<size_t>(need, 1);
  size_t c;
  c = 0; if (p->d_gshot) { cudaFree(p->d_gshot); p->d_gshot = nullptr; }
  CUDA_OR_FAIL(p, grow(&p->d_gshot, &c, cap));
  c = 0; if (p->d_gq) { cudaFree(p->d_gq); p->d_gq = nullptr; }
  CUDA_OR_FAIL(p, grow(&p->d_gq, &c, cap));
  c = 0; if (p->d_gp) { cudaFree(p->d_gp); p->d_gp = nullptr; }
  CUDA_OR_FAIL(p, grow(&p->d_gp, &c, cap));
  c = 0; if (p->d_gpsi) { cudaFree(p->d_gpsi); p->d_gpsi = nullptr; }
  CUDA_OR_FAIL(p, grow(&p->d_gpsi, &c, cap));
  c = 0; if (p->d_gpsi_f1) { cudaFree(p->d_gpsi_f1); p->d_gpsi_f1 = nullptr; }
  CUDA_OR_FAIL(p, grow(&p->d_gpsi_f1, &c, cap));
  c = 0; if (p->d_gcoef) { cudaFree(p->d_gcoef); p->d_gcoef = nullptr; }
  CUDA_OR_FAIL(p, grow(&p->d_gcoef, &c, cap));
  c = 0; if (p->d_state) { cudaFree(p->d_state); p->d_state = nullptr; }
  CUDA_OR_FAIL(p, grow(&p->d_state, &c, cap * p->nfields));
  c = 0; if (p->d_gsteps) { cudaFree(p->d_gsteps); p->d_gsteps = nullptr; }
  CUDA_OR_FAIL(p, grow(&p->d_gsteps, &c, cap));
  c = 0; if (p->d_adj_order) { cudaFree(p->d_adj_order); p->d_adj_order = nullptr; }
  CUDA_OR_FAIL(p, grow(&p->d_adj_order, &c, cap));  // also the rays' longest-first order
  if (!p->d_ray_bucket)
    CUDA_OR_FAIL(p, cudaMalloc(&p->d_ray_bucket,
                               sizeof(int64_t) * (size_t)(p->nsteps / fga::ray_order_width(p->nsteps) + 2)));
  p->g_cap = cap;
  return FGA_OK;
}

fga_status fga_decompose(fga_plan_t p, const double* u0, const double* u1, int64_t* counts_host) {
  fga_status st = check_usable(p);
  if (st != FGA_OK) return st;
  if (!u0 || !u1) return fail(p, FGA_ERR_INVALID, "u0 and u1 must not be NULL");
  const GridDev& gd = p->grid;
  const int d = gd.dim;
  const size_t n_all = (size_t)p->nshots * gd.npts;
  const double* du0 = u0;
  const double* du1 = u1;
  if (!is_device_ptr(u0) || !is_device_ptr(u1)) {
    // host data: one staging buffer holds both fields
    CUDA_OR_FAIL(p, grow(&p->d_in0, &p->in_cap, 2 * n_all));
    p->d_in1 = p->d_in0 + n_all;
    CUDA_OR_FAIL(p, cudaMemcpyAsync(p->d_in0, u0, sizeof(double) * n_all, cudaMemcpyDefault, p->stream));
    CUDA_OR_FAIL(p, cudaMemcpyAsync(p->d_in1, u1, sizeof(double) * n_all, cudaMemcpyDefault, p->stream));
    du0 = p->d_in0;
    du1 = p->d_in1;
  }
  CUDA_OR_FAIL(p, cudaEventRecord(p->ev[0], p->stream));
  CUDA_OR_FAIL(p, fga::launch_support_bbox(p, du0, du1));
  std::vector<int> bbox((size_t)p->nshots * d * 2);
  CUDA_OR_FAIL(p, cudaMemcpyAsync(bbox.data(), p->d_bbox, sizeof(int) * bbox.size(),
                                  cudaMemcpyDeviceToHost, p->stream));
  CUDA_OR_FAIL(p, cudaStreamSynchronize(p->stream));
  // active q rectangle per shot: q whose box meets the data's bounding box
  int64_t psi_total = 0, g1_total = 0, g2_total = 0;
  p->blk_first.assign(p->nshots + 1, 0);
  for (int s = 0; s < p->nshots; ++s) {
    ShotDev& sh = p->shots[s];
    bool empty = false;
    for (int k = 0; k < d; ++k) {
      int lo = bbox[(s * d + k) * 2], hi = bbox[(s * d + k) * 2 + 1];
      if (hi < 0) empty = true;
      if (gd.periodic[k]) {
        sh.qlo[k] = 0;
        sh.qn[k] = sh.nq[k];
      } else {
        int64_t half = sh.nb[k] / 2;
        int64_t mlo = (int64_t)std::ceil((double)(lo - half + 1) / sh.s[k]);
        int64_t mhi = (int64_t)std::floor((double)(hi + half) / sh.s[k]);
        mlo = std::max<int64_t>(mlo, 0);
        mhi = std::min<int64_t>(mhi, sh.nq[k] - 1);
        sh.qlo[k] = mlo;
        sh.qn[k] = std::max<int64_t>(mhi - mlo + 1, 0);
      }
    }
    if (empty)
      for (int k = 0; k < d; ++k) sh.qn[k] = 0;
    int64_t qt = 1;
    for (int k = 0; k < d; ++k) qt *= sh.qn[k];
    sh.psi_off = psi_total;
    sh.psi_len = qt * sh.np;
    psi_total += ((sh.psi_len + fga::kScanBlock - 1) / fga::kScanBlock) * fga::kScanBlock;
    p->blk_first[s] = sh.psi_off / fga::kScanBlock;
    if (d >= 2) {
      sh.row_lo = (int64_t)sh.s[0] * sh.qlo[0] - sh.nb[0] / 2;
      sh.nrows = sh.qn[0] > 0 ? (int64_t)sh.s[0] * (sh.qn[0] - 1) + sh.nb[0] : 0;
      sh.g1_off = g1_total;
    }
    if (d == 2)
      g1_total += p->precision == FGA_MIXED_TF32X3
                      ? (int64_t)(fga::fbi_b_image_floats(sh) / 4)  // float image, in double2
                      : 2 * sh.nrows * sh.qn[1] * sh.nb[1];
    if (d == 3) {
      sh.row_lo1 = (int64_t)sh.s[1] * sh.qlo[1] - sh.nb[1] / 2;
      sh.nrows1 = sh.qn[1] > 0 ? (int64_t)sh.s[1] * (sh.qn[1] - 1) + sh.nb[1] : 0;
      // stage 1: [field][x row][y row][q_z][p_z]; stage 2: [field][x row][q_y][q_z][p_y][p_z]
      g1_total += 2 * sh.nrows * sh.nrows1 * sh.qn[2] * sh.nb[2];
      sh.g2_off = g2_total;
      g2_total += 2 * sh.nrows * sh.qn[1] * sh.qn[2] * sh.nb[1] * sh.nb[2];
    }
    sh.g_off = sh.g_cnt = 0;
  }
  p->blk_first[p->nshots] = psi_total / fga::kScanBlock;
  p->nblocks = psi_total / fga::kScanBlock;
  // psi and psi_1 in double2 units (FP32 pairs in mixed precision take half of them)
  const size_t psi_units = fga::psi_is_f32(p) ? (size_t)psi_total / 2 + 1 : (size_t)psi_total;
  CUDA_OR_FAIL(p, grow(&p->d_psi, &p->psi_cap, psi_units));
  CUDA_OR_FAIL(p, grow(&p->d_psi_f1, &p->psi_f1_cap, psi_units));
  if (d >= 2) CUDA_OR_FAIL(p, grow(&p->d_g1, &p->g1_cap, (size_t)g1_total));
  if (d == 3) CUDA_OR_FAIL(p, grow(&p->d_g2, &p->g2_cap, (size_t)g2_total));
  CUDA_OR_FAIL(p, grow(&p->d_blk, &p->blk_cap, (size_t)p->nblocks + 1));
  CUDA_OR_FAIL(p, cudaMemcpyAsync(p->d_blk_first, p->blk_first.data(),
                                  sizeof(int64_t) * (p->nshots + 1), cudaMemcpyHostToDevice, p->stream));
  CUDA_OR_FAIL(p, cudaMemcpyAsync(p->d_shots, p->shots.data(), sizeof(ShotDev) * p->nshots,
                                  cudaMemcpyHostToDevice, p->stream));
  CUDA_OR_FAIL(p, fga::launch_fbi(p, du0, du1));
  CUDA_OR_FAIL(p, cudaEventRecord(p->ev[1], p->stream));
  if (p->keep_n > 0) {
    if (!p->d_topk) {
      CUDA_OR_FAIL(p, cudaMalloc(&p->d_topk, sizeof(unsigned long long) * 4 * p->nshots));
      CUDA_OR_FAIL(p, cudaMalloc(&p->d_topk_hist, sizeof(unsigned long long) * 256 * p->nshots));
    }
    CUDA_OR_FAIL(p, grow(&p->d_blk_eq, &p->blk_eq_cap, (size_t)p->nblocks + 1));
  }
  CUDA_OR_FAIL(p, fga::launch_select_count(p));
  std::vector<int64_t> counts(p->nshots, 0);
  if (p->nblocks > 0)
    CUDA_OR_FAIL(p, cudaMemcpyAsync(counts.data(), p->d_counts, sizeof(int64_t) * p->nshots,
                                    cudaMemcpyDeviceToHost, p->stream));
  CUDA_OR_FAIL(p, cudaStreamSynchronize(p->stream));
  int64_t G = 0;
  for (int s = 0; s < p->nshots; ++s) {
    p->shots[s].g_off = G;
    p->shots[s].g_cnt = counts[s];
    G += counts[s];
  }
  if (G > ((int64_t)1 << 31) - 1) return fail(p, FGA_ERR_CAPACITY, "more than 2^31-1 Gaussians", true);
  p->G = G;
  p->shape_gen += 1;
  st = alloc_gaussians(p, (size_t)G);
  if (st != FGA_OK) return st;
  CUDA_OR_FAIL(p, fga::launch_select(p));
  CUDA_OR_FAIL(p, cudaEventRecord(p->ev[2], p->stream));
  if (counts_host)
    for (int s = 0; s < p->nshots; ++s) counts_host[s] = counts[s];
  p->stage = 1;
  return FGA_OK;
}

// Device capacity of the block-private trace slices of the next ray launch.
static fga_status trace_capacity(fga_plan_s* p) {
  if (p->nrx == 0 || p->G == 0) return FGA_OK;
  CUDA_OR_FAIL(p, fga::ensure_ray_blocks(p));
  const size_t need = (size_t)(fga::trace_slices(p) * p->nshots * p->rx.nrec * p->rx.nrx);
  CUDA_OR_FAIL(p, grow(&p->d_part, &p->part_cap, need));
  return FGA_OK;
}

fga_status fga_propagate(fga_plan_t p) {
  fga_status st = check_usable(p);
  if (st != FGA_OK) return st;
  if (p->stage < 1) return fail(p, FGA_ERR_STATE, "fga_propagate before fga_decompose");
  st = trace_capacity(p);
  if (st != FGA_OK) return st;
  CUDA_OR_FAIL(p, cudaEventRecord(p->ev[3], p->stream));
  CUDA_OR_FAIL(p, p->z_method == FGA_Z_DIVIDED ? fga::launch_rays_dd(p, p->nsteps) : fga::launch_rays(p));
  CUDA_OR_FAIL(p, cudaEventRecord(p->ev[4], p->stream));
  p->stage = 2;
  return FGA_OK;
}

// Device capacities the reconstruction needs for the current Gaussian set. The tile
// lists: every Gaussian meets at most prod_k m_k tiles, m_k = (floor(window points /
// tile) + 2) per image, times 5 images on periodic axes.
static fga_status reconstruct_capacity(fga_plan_s* p, double headroom = 1.0) {
  const GridDev& gd = p->grid;
  const int d = gd.dim;
  size_t pairs = 0;
  for (const auto& sh : p->shots) {
    size_t per = 1;
    for (int k = 0; k < d; ++k) {
      double wpts = 2.0 * p->kappa * sh.sqrt_eps * gd.inv_h[k] + 6.0;
      size_t mk = (size_t)(wpts / gd.tile[k]) + 2;
      if (gd.periodic[k]) mk *= 5;
      mk = std::min<size_t>(mk, (size_t)sh.ntile[k]);
      per *= mk;
    }
    pairs += per * (size_t)std::ceil(headroom * (double)sh.g_cnt);
  }
  CUDA_OR_FAIL(p, grow(&p->d_tile_list, &p->list_cap, pairs));
  int nsplit;
  int64_t chunk;
  fga::bin_splits(p, &nsplit, &chunk);
  CUDA_OR_FAIL(p, grow(&p->d_bin_off, &p->bin_cap, (size_t)p->ntiles * nsplit + 1));
  CUDA_OR_FAIL(p, grow(&p->d_rng, &p->rng_cap, (size_t)d * 2 * std::max<size_t>(p->g_cap, 1)));
  const bool tc = p->precision == FGA_MIXED_TF32X3;
  CUDA_OR_FAIL(p, grow(&p->d_partial, &p->partial_cap,
                       tc ? (fga::partial_bytes_tc(p) + 7) / 8
                          : fga::partial_items(p) * fga::tile_points(d)));
  if (tc) {
    size_t cap = p->ganc_cap;
    unsigned char* g = static_cast<unsigned char*>(p->d_ganc);
    CUDA_OR_FAIL(p, grow(&g, &cap, fga::anchor_bytes_tc(p)));
    p->d_ganc = g;
    p->ganc_cap = cap;
  }
  return FGA_OK;
}

fga_status fga_run_graph(fga_plan_t p, double* u_dev) {
  fga_status st = check_usable(p);
  if (st != FGA_OK) return st;
  if (p->stage < 1) return fail(p, FGA_ERR_STATE, "fga_run_graph before fga_decompose");
  if (!u_dev || !is_device_ptr(u_dev))
    return fail(p, FGA_ERR_INVALID, "fga_run_graph writes to device memory only");
  if (p->stream == nullptr)
    return fail(p, FGA_ERR_INVALID, "graph mode needs a stream other than the legacy default stream");
  if (p->ray_blocks == 0) {
    // first call: one eager pass sets up every lazily initialised resource
    st = fga_propagate(p);
    if (st != FGA_OK) return st;
    return fga_reconstruct(p, u_dev);
  }
  st = reconstruct_capacity(p);
  if (st != FGA_OK) return st;
  st = trace_capacity(p);
  if (st != FGA_OK) return st;
  int nsplit;
  int64_t chunk;
  fga::bin_splits(p, &nsplit, &chunk);
  int64_t key[13] = {p->G, (int64_t)p->g_cap, (int64_t)p->list_cap, (int64_t)p->partial_cap,
                    (int64_t)(uintptr_t)u_dev, p->nrx, p->seg, p->ray_blocks,
                    (int64_t)(uintptr_t)p->d_part, p->ray_variant, nsplit, chunk,
                    (int64_t)(uintptr_t)p->d_bin_off};
  bool same = p->graph_exec != nullptr;
  for (int i = 0; i < 13; ++i) same = same && key[i] == p->graph_key[i];
  if (!same) {
    if (p->graph_exec) {
      cudaGraphExecDestroy(p->graph_exec);
      p->graph_exec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    CUDA_OR_FAIL(p, cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = p->z_method == FGA_Z_DIVIDED ? fga::launch_rays_dd(p, p->nsteps) : fga::launch_rays(p);
    if (e == cudaSuccess) e = fga::launch_binning(p);
    if (e == cudaSuccess) e = fga::launch_binning_fill(p);
    if (e == cudaSuccess)
      e = p->precision == FGA_MIXED_TF32X3 ? fga::launch_reconstruct_tc(p, u_dev)
                                           : fga::launch_reconstruct(p, u_dev);
    cudaError_t e2 = cudaStreamEndCapture(p->stream, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return fail(p, FGA_ERR_CUDA, std::string("graph capture: ") +
                                       cudaGetErrorString(e != cudaSuccess ? e : e2), true);
    }
    e = cudaGraphInstantiate(&p->graph_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      p->graph_exec = nullptr;
      return fail(p, FGA_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e), true);
    }
    for (int i = 0; i < 13; ++i) p->graph_key[i] = key[i];
  }
  CUDA_OR_FAIL(p, cudaGraphLaunch(p->graph_exec, p->stream));
  p->launches += 12;
  p->stage = 2;
  return FGA_OK;
}

// Headroom of the pipeline graph's capacities over the counts of its sizing pass.
constexpr double kPipeHeadroom = 1.25;

fga_status fga_run_pipeline(fga_plan_t p, const double* u0, const double* u1, double* u_dev) {
  // no refresh of the host's counts here: a replay needs none, and reading them back
  // would wait for the stream
  if (!p) return fail(nullptr, FGA_ERR_INVALID, "plan is NULL");
  if (p->failed) return FGA_ERR_STATE;
  fga_status st = FGA_OK;
  if (!u0 || !u1 || !u_dev || !is_device_ptr(u0) || !is_device_ptr(u1) || !is_device_ptr(u_dev))
    return fail(p, FGA_ERR_INVALID, "fga_run_pipeline takes device pointers only");
  if (p->stream == nullptr)
    return fail(p, FGA_ERR_INVALID, "graph mode needs a stream other than the legacy default stream");
  if (p->nrx > 0) return fail(p, FGA_ERR_INVALID, "fga_run_pipeline records no traces: the plan has receivers");
  if (p->z_method != FGA_Z_DYNAMIC)
    return fail(p, FGA_ERR_INVALID, "fga_run_pipeline needs the dynamic-ray Z (FGA_Z_DYNAMIC)");
  auto key_now = [&]() {
    return std::vector<int64_t>{
        (int64_t)(uintptr_t)u0, (int64_t)(uintptr_t)u1, (int64_t)(uintptr_t)u_dev, p->shape_gen,
        (int64_t)p->g_cap, (int64_t)p->list_cap, (int64_t)p->partial_cap, (int64_t)p->bin_cap,
        (int64_t)(uintptr_t)p->d_gshot, (int64_t)(uintptr_t)p->d_state,
        (int64_t)(uintptr_t)p->d_tile_list, (int64_t)(uintptr_t)p->d_partial,
        (int64_t)(uintptr_t)p->d_bin_off, (int64_t)(uintptr_t)p->d_psi, (int64_t)(uintptr_t)p->d_g1,
        p->seg, p->ray_blocks, p->ray_variant};
  };
  if (p->pipe_exec && key_now() == p->pipe_key) {
    CUDA_OR_FAIL(p, cudaGraphLaunch(p->pipe_exec, p->stream));
    p->launches += p->pipe_kernels;
    p->pipe_host_stale = true;
    p->stage = 2;
    return FGA_OK;
  }
  if (p->pipe_exec) {
    cudaGraphExecDestroy(p->pipe_exec);
    p->pipe_exec = nullptr;
  }
  // sizing pass (eager; its result is this call's result): the data's active q
  // rectangles and counts, then capacities with headroom for the counts of later data
  st = fga_decompose(p, u0, u1, nullptr);
  if (st != FGA_OK) return st;
  const size_t want = (size_t)std::ceil(kPipeHeadroom * (double)p->G) + 1024;
  if (want > p->g_cap) {
    st = alloc_gaussians(p, want);  // the new arrays are empty: select into them again
    if (st != FGA_OK) return st;
    st = fga_decompose(p, u0, u1, nullptr);
    if (st != FGA_OK) return st;
  }
  if (!p->d_gm) CUDA_OR_FAIL(p, cudaMalloc(&p->d_gm, 2 * sizeof(int64_t)));
  st = fga_propagate(p);
  if (st != FGA_OK) return st;
  p->dev_counts = true;  // binning splits over the whole capacity
  st = reconstruct_capacity(p, kPipeHeadroom);
  p->dev_counts = false;
  if (st != FGA_OK) return st;
  st = fga_reconstruct(p, u_dev);
  if (st != FGA_OK) return st;
  // capture: every launch sizes itself from the device-side counts
  cudaGraph_t graph = nullptr;
  CUDA_OR_FAIL(p, cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal));
  p->dev_counts = true;
  const int64_t launches0 = p->launches;
  cudaError_t e = fga::launch_support_bbox(p, u0, u1);
  if (e == cudaSuccess) e = fga::launch_check_shapes(p);
  if (e == cudaSuccess) e = fga::launch_fbi(p, u0, u1);
  if (e == cudaSuccess) e = fga::launch_select_count(p);
  if (e == cudaSuccess) e = fga::launch_counts_finish(p);
  if (e == cudaSuccess) e = fga::launch_select(p);
  if (e == cudaSuccess) e = fga::launch_rays(p);
  if (e == cudaSuccess) e = fga::launch_binning(p);
  if (e == cudaSuccess) e = fga::launch_binning_fill(p);
  if (e == cudaSuccess)
    e = p->precision == FGA_MIXED_TF32X3 ? fga::launch_reconstruct_tc(p, u_dev)
                                         : fga::launch_reconstruct(p, u_dev);
  p->dev_counts = false;
  cudaError_t e2 = cudaStreamEndCapture(p->stream, &graph);
  p->launches = launches0;
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return fail(p, FGA_ERR_CUDA, std::string("pipeline graph capture: ") +
                                     cudaGetErrorString(e != cudaSuccess ? e : e2), true);
  }
  size_t nnodes = 0;
  p->pipe_kernels = 0;
  if (cudaGraphGetNodes(graph, nullptr, &nnodes) == cudaSuccess && nnodes > 0) {
    std::vector<cudaGraphNode_t> nodes(nnodes);
    if (cudaGraphGetNodes(graph, nodes.data(), &nnodes) == cudaSuccess)
      for (size_t i = 0; i < nnodes; ++i) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel)
          p->pipe_kernels += 1;
      }
  }
  e = cudaGraphInstantiate(&p->pipe_exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    p->pipe_exec = nullptr;
    return fail(p, FGA_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e), true);
  }
  p->pipe_key = key_now();
  return FGA_OK;
}

// Milliseconds between two events recorded around `launch` on the plan's stream (the
// best of `reps` runs after one untimed run).
extern "C++" template <class F>
cudaError_t time_best(fga_plan_s* p, int reps, F launch, float* best_ms) {
  cudaError_t e = launch();
  *best_ms = 3.0e38f;
  for (int r = 0; r < reps && e == cudaSuccess; ++r) {
    e = cudaEventRecord(p->ev[8], p->stream);
    if (e == cudaSuccess) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(p->ev[9], p->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(p->ev[9]);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, p->ev[8], p->ev[9]);
    if (e == cudaSuccess && ms < *best_ms) *best_ms = ms;
  }
  return e;
}

fga_status fga_autotune(fga_plan_t p, double* u_dev, int64_t* choice) {
  fga_status st = check_usable(p);
  if (st != FGA_OK) return st;
  if (p->stage < 1) return fail(p, FGA_ERR_STATE, "fga_autotune before fga_decompose");
  if (!u_dev || !is_device_ptr(u_dev))
    return fail(p, FGA_ERR_INVALID, "fga_autotune writes to device memory only");
  // 1. register budget and blocks per SM of the persistent ray kernel, timed on a short
  //    integration
  const int64_t probe = std::min<int64_t>(p->nsteps, 64);
  int best_variant = 0, best_sm = 0;
  float best = 3.0e38f;
  if (p->G > 0 && probe > 0 && p->z_method == FGA_Z_DYNAMIC) {  // the divided-difference kernel has no variants
    for (int variant = 0; variant < 2; ++variant) {
      p->ray_variant = variant;
      const int max_sm = fga::ray_max_per_sm(p);
      for (int per_sm = max_sm; per_sm >= 1 && per_sm >= max_sm - 3; --per_sm) {
        p->ray_per_sm = per_sm;
        p->ray_blocks = 0;
        float ms = 0.0f;
        CUDA_OR_FAIL(p, time_best(p, 2, [&] { return fga::launch_rays_steps(p, probe, false); }, &ms));
        if (ms < best * 0.98f) {  // prefer the earlier candidate unless clearly slower
          best = ms;
          best_sm = per_sm;
          best_variant = variant;
        }
      }
    }
  }
  p->ray_variant = best_variant;
  p->ray_per_sm = best_sm;
  p->ray_blocks = 0;
  // 2. the full integration with the chosen launch shape
  st = fga_propagate(p);
  if (st != FGA_OK) return st;
  // 3. split-K segment length of the gather, timed on the real Gaussian set
  const bool tc = p->precision == FGA_MIXED_TF32X3;
  const int d = p->grid.dim;
  // (tensor cores: at most 2048 Gaussians per work item, since the FP32 accumulation in
  // tensor memory loses accuracy with the number of products it sums: rel-L2 against the
  // FP64 path about 2e-5 at 2048 and 3e-5 at 4096 on the layered model)
  const int64_t base = tc ? 128 : (d == 1 ? 128 : 256);
  int64_t best_seg = 0;
  best = 3.0e38f;
  for (int k = 0; k < 5; ++k) {
    p->seg = base << k;
    st = reconstruct_capacity(p);
    if (st != FGA_OK) return st;
    float ms = 0.0f;
    CUDA_OR_FAIL(p, time_best(p, 2, [&] {
      cudaError_t e = fga::launch_binning(p);
      if (e == cudaSuccess) e = fga::launch_binning_fill(p);
      if (e == cudaSuccess)
        e = tc ? fga::launch_reconstruct_tc(p, u_dev) : fga::launch_reconstruct(p, u_dev);
      return e;
    }, &ms));
    if (ms < best) {
      best = ms;
      best_seg = p->seg;
    }
  }
  p->seg = best_seg;
  // 4. the field with the chosen segment length
  st = fga_reconstruct(p, u_dev);
  if (st != FGA_OK) return st;
  if (choice) {
    choice[0] = p->ray_per_sm;
    choice[1] = p->precision == FGA_MIXED_TF32X3 ? fga::segment_len_tc(p) : fga::segment_len(p);
    choice[2] = p->ray_variant;
  }
  return read_status(p);
}

fga_status fga_tuning(fga_plan_t p, int64_t* choice) {
  if (!p || !choice) return fail(p, FGA_ERR_INVALID, "NULL plan or output");
  choice[0] = p->ray_per_sm;
  choice[1] = p->precision == FGA_MIXED_TF32X3 ? fga::segment_len_tc(p) : fga::segment_len(p);
  choice[2] = p->ray_variant;
  return FGA_OK;
}

fga_status fga_set_tuning(fga_plan_t p, const int64_t* choice) {
  fga_status st = check_usable(p);
  if (st != FGA_OK) return st;
  if (!choice || choice[0] < 0 || choice[0] > 64 || choice[1] < 0 || choice[1] > ((int64_t)1 << 20) ||
      choice[2] < 0 || choice[2] > 1)
    return fail(p, FGA_ERR_INVALID,
                "tuning values out of range (0 <= blocks/SM <= 64, 0 <= segment <= 2^20, variant 0 or 1)");
  p->ray_per_sm = (int)choice[0];
  p->ray_blocks = 0;
  p->seg = choice[1];
  p->ray_variant = (int)choice[2];
  return FGA_OK;
}

fga_status fga_reconstruct(fga_plan_t p, double* u_out) {
  fga_status st = check_usable(p);
  if (st != FGA_OK) return st;
  if (p->stage < 2) return fail(p, FGA_ERR_STATE, "fga_reconstruct before fga_propagate");
  if (!u_out) return fail(p, FGA_ERR_INVALID, "u_out must not be NULL");
  st = reconstruct_capacity(p);
  if (st != FGA_OK) return st;
  const GridDev& gd = p->grid;
  const bool tc = p->precision == FGA_MIXED_TF32X3;
  CUDA_OR_FAIL(p, cudaEventRecord(p->ev[5], p->stream));
  CUDA_OR_FAIL(p, fga::launch_binning(p));
  CUDA_OR_FAIL(p, fga::launch_binning_fill(p));
  CUDA_OR_FAIL(p, cudaEventRecord(p->ev[6], p->stream));
  const size_t n_all = (size_t)p->nshots * gd.npts;
  double* dst = u_out;
  bool host_out = !is_device_ptr(u_out);
  if (host_out) {
    CUDA_OR_FAIL(p, grow(&p->d_out, &p->out_cap, n_all));
    dst = p->d_out;
  }
  CUDA_OR_FAIL(p, tc ? fga::launch_reconstruct_tc(p, dst) : fga::launch_reconstruct(p, dst));
  CUDA_OR_FAIL(p, cudaEventRecord(p->ev[7], p->stream));
  if (host_out) {
    CUDA_OR_FAIL(p, cudaMemcpyAsync(u_out, dst, sizeof(double) * n_all, cudaMemcpyDeviceToHost,
                                    p->stream));
    return read_status(p);
  }
  return FGA_OK;
}

fga_status fga_set_wait_budget(fga_plan_t p, int64_t tries) {
  fga_status st = check_usable(p);
  if (st != FGA_OK) return st;
  if (tries > (int64_t)UINT32_MAX) return fail(p, FGA_ERR_INVALID, "tries must be below 2^32");
  p->wait_tries = tries < 0 ? -1 : tries;
  return FGA_OK;
}

fga_status fga_set_adjoint_checkpointing(fga_plan_t p, int mode) {
  fga_status st = check_usable(p);
  if (st != FGA_OK) return st;
  if (mode != 0 && mode != 1) return fail(p, FGA_ERR_INVALID, "mode must be 0 or 1");
  p->adj_force_segments = mode;
  return FGA_OK;
}

fga_status fga_sync(fga_plan_t p) {
  fga_status st = check_usable(p);
  if (st != FGA_OK) return st;
  return read_status(p);
}

int64_t fga_count(fga_plan_t p, int shot) {
  if (!p || shot < 0 || shot >= p->nshots || p->stage < 1) return -1;
  return p->shots[shot].g_cnt;
}

fga_status fga_shot_grid(fga_plan_t p, int shot, int64_t* nq, int64_t* np, int64_t* nb, int64_t* s) {
  if (!p || shot < 0 || shot >= p->nshots) return fail(p, FGA_ERR_INVALID, "bad plan or shot");
  const ShotDev& sh = p->shots[shot];
  for (int k = 0; k < p->grid.dim; ++k) {
    if (nq) nq[k] = sh.nq[k];
    if (np) np[k] = sh.nb[k];
    if (nb) nb[k] = sh.nb[k];
    if (s) s[k] = sh.s[k];
  }
  return FGA_OK;
}

fga_status fga_psi(fga_plan_t p, int shot, double* psi_host, double* max_abs) {
  fga_status st = check_usable(p);
  if (st != FGA_OK) return st;
  if (shot < 0 || shot >= p->nshots) return fail(p, FGA_ERR_INVALID, "bad shot");
  if (p->stage < 1) return fail(p, FGA_ERR_STATE, "no decomposition yet");
  const ShotDev& sh = p->shots[shot];
  const int d = p->grid.dim;
  int64_t nqt = 1;
  for (int k = 0; k < d; ++k) nqt *= sh.nq[k];
  if (psi_host) {
    std::memset(psi_host, 0, sizeof(double) * 2 * nqt * sh.np);
    std::vector<double> seg((size_t)sh.psi_len * 2);
    if (fga::psi_is_f32(p)) {  // FP32 pairs (mixed precision), widened exactly
      std::vector<float> segf((size_t)sh.psi_len * 2);
      if (sh.psi_len > 0)
        CUDA_OR_FAIL(p, cudaMemcpyAsync(segf.data(), reinterpret_cast<const float2*>(p->d_psi) + sh.psi_off,
                                        sizeof(float2) * sh.psi_len, cudaMemcpyDeviceToHost, p->stream));
      CUDA_OR_FAIL(p, cudaStreamSynchronize(p->stream));
      for (size_t i = 0; i < segf.size(); ++i) seg[i] = (double)segf[i];
    } else {
      if (sh.psi_len > 0)
        CUDA_OR_FAIL(p, cudaMemcpyAsync(seg.data(), p->d_psi + sh.psi_off, sizeof(double2) * sh.psi_len,
                                        cudaMemcpyDeviceToHost, p->stream));
      CUDA_OR_FAIL(p, cudaStreamSynchronize(p->stream));
    }
    int64_t qtl = sh.psi_len / std::max<int64_t>(sh.np, 1);
    for (int64_t ql = 0; ql < qtl; ++ql) {
      int64_t qf;
      if (d == 1) {
        qf = sh.qlo[0] + ql;
      } else if (d == 2) {
        int64_t mx = ql / sh.qn[1], mz = ql % sh.qn[1];
        qf = (sh.qlo[0] + mx) * sh.nq[1] + sh.qlo[1] + mz;
      } else {
        const int64_t qn12 = sh.qn[1] * sh.qn[2];
        int64_t mx = ql / qn12, my = (ql % qn12) / sh.qn[2], mz = ql % sh.qn[2];
        qf = ((sh.qlo[0] + mx) * sh.nq[1] + sh.qlo[1] + my) * sh.nq[2] + sh.qlo[2] + mz;
      }
      std::memcpy(psi_host + 2 * qf * sh.np, seg.data() + 2 * ql * sh.np, sizeof(double) * 2 * sh.np);
    }
  }
  if (max_abs) {
    unsigned long long bits = 0;
    CUDA_OR_FAIL(p, cudaMemcpyAsync(&bits, p->d_max2 + shot, sizeof(bits), cudaMemcpyDeviceToHost,
                                    p->stream));
    CUDA_OR_FAIL(p, cudaStreamSynchronize(p->stream));
    double m2;
    std::memcpy(&m2, &bits, sizeof(m2));
    *max_abs = std::sqrt(m2);
  }
  return FGA_OK;
}

fga_status fga_gaussians(fga_plan_t p, int shot, int64_t* qidx, int64_t* pidx, double* psi) {
  fga_status st = check_usable(p);
  if (st != FGA_OK) return st;
  if (shot < 0 || shot >= p->nshots) return fail(p, FGA_ERR_INVALID, "bad shot");
  if (p->stage < 1) return fail(p, FGA_ERR_STATE, "no decomposition yet");
  const ShotDev& sh = p->shots[shot];
  int64_t n = sh.g_cnt;
  if (n == 0) return FGA_OK;
  if (qidx)
    CUDA_OR_FAIL(p, cudaMemcpyAsync(qidx, p->d_gq + sh.g_off, sizeof(int64_t) * n,
                                    cudaMemcpyDeviceToHost, p->stream));
  if (pidx) {
    std::vector<int32_t> tmp(n);
    CUDA_OR_FAIL(p, cudaMemcpyAsync(tmp.data(), p->d_gp + sh.g_off, sizeof(int32_t) * n,
                                    cudaMemcpyDeviceToHost, p->stream));
    CUDA_OR_FAIL(p, cudaStreamSynchronize(p->stream));
    for (int64_t i = 0; i < n; ++i) pidx[i] = tmp[i];
  }
  if (psi)
    CUDA_OR_FAIL(p, cudaMemcpyAsync(psi, p->d_gpsi + sh.g_off, sizeof(double2) * n,
                                    cudaMemcpyDeviceToHost, p->stream));
  CUDA_OR_FAIL(p, cudaStreamSynchronize(p->stream));
  return FGA_OK;
}

fga_status fga_state(fga_plan_t p, int shot, double* Q, double* P, double* A, double* B, double* a,
                     double* S) {
  fga_status st = check_usable(p);
  if (st != FGA_OK) return st;
  if (shot < 0 || shot >= p->nshots) return fail(p, FGA_ERR_INVALID, "bad shot");
  if (p->stage < 2) return fail(p, FGA_ERR_STATE, "not propagated yet");
  const ShotDev& sh = p->shots[shot];
  const int d = p->grid.dim;
  const int64_t n = sh.g_cnt;
  if (n == 0) return FGA_OK;
  std::vector<double> f((size_t)p->nfields * n);
  for (int i = 0; i < p->nfields; ++i)
    CUDA_OR_FAIL(p, cudaMemcpyAsync(f.data() + (size_t)i * n, p->d_state + (size_t)i * p->g_cap + sh.g_off,
                                    sizeof(double) * n, cudaMemcpyDeviceToHost, p->stream));
  CUDA_OR_FAIL(p, cudaStreamSynchronize(p->stream));
  auto F = [&](int field, int64_t g) { return f[(size_t)field * n + g]; };
  const int AR = 2 * d, AI = AR + d * d, BR = AI + d * d, BI = BR + d * d, aR = BI + d * d;
  for (int64_t g = 0; g < n; ++g) {
    for (int k = 0; k < d; ++k) {
      if (Q) Q[g * d + k] = F(k, g);
      if (P) P[g * d + k] = F(d + k, g);
      for (int l = 0; l < d; ++l) {
        int e = k * d + l;
        if (A) {
          A[((g * d + k) * d + l) * 2] = F(AR + e, g);
          A[((g * d + k) * d + l) * 2 + 1] = F(AI + e, g);
        }
        if (B) {
          B[((g * d + k) * d + l) * 2] = F(BR + e, g);
          B[((g * d + k) * d + l) * 2 + 1] = F(BI + e, g);
        }
      }
    }
    if (a) {
      a[2 * g] = F(aR, g);
      a[2 * g + 1] = F(aR + 1, g);
    }
    if (S) S[g] = F(aR + 2, g);
  }
  return FGA_OK;
}

fga_status fga_set_receivers(fga_plan_t p, int64_t nrx, const double* xr, int64_t record_every) {
  fga_status st = check_usable(p);
  if (st != FGA_OK) return st;
  const GridDev& gd = p->grid;
  const int d = gd.dim;
  if (p->graph_exec) {  // a captured graph holds the old receiver buffers
    cudaGraphExecDestroy(p->graph_exec);
    p->graph_exec = nullptr;
  }
  for (void* b : {(void*)p->d_rx, (void*)p->d_rx_off, (void*)p->d_rx_perm, (void*)p->d_traces,
                  (void*)p->d_run_geo, (void*)p->d_run_axis, (void*)p->d_run_off})
    if (b) cudaFree(b);
  p->d_rx = nullptr;
  p->d_rx_off = nullptr;
  p->d_rx_perm = nullptr;
  p->d_traces = nullptr;
  p->d_run_geo = nullptr;
  p->d_run_axis = nullptr;
  p->d_run_off = nullptr;
  p->nrx = 0;
  std::memset(&p->rx, 0, sizeof(p->rx));
  if (nrx == 0) return FGA_OK;
  if (nrx < 0 || nrx > (((int64_t)1 << 31) - 1) || !xr)
    return fail(p, FGA_ERR_INVALID, "need 0 < nrx < 2^31 and receiver positions");
  if (record_every < 1 || p->nsteps % record_every != 0)
    return fail(p, FGA_ERR_INVALID, "record_every must be >= 1 and divide T/dt");
  if (p->z_method != FGA_Z_DYNAMIC)
    return fail(p, FGA_ERR_INVALID, "receivers (traces, fga_grad) need z_method FGA_Z_DYNAMIC");
  for (int k = 0; k < d; ++k)
    if (gd.periodic[k]) return fail(p, FGA_ERR_INVALID, "receivers need open axes");
  std::vector<double> x((size_t)nrx * d);
  CUDA_OR_FAIL(p, cudaMemcpy(x.data(), xr, sizeof(double) * x.size(), cudaMemcpyDefault));
  for (int64_t r = 0; r < nrx; ++r)
    for (int k = 0; k < d; ++k) {
      double v = x[(size_t)r * d + k];
      if (!std::isfinite(v) || v < gd.o[k] || v > gd.o[k] + (double)(gd.n[k] - 1) * gd.h[k])
        return fail(p, FGA_ERR_INVALID, "receivers must lie inside the grid");
    }
  // runs: receivers sharing the coordinate across an axis, equally spaced along it
  std::vector<double> run_geo;
  std::vector<int32_t> run_axis, run_rx;
  std::vector<int64_t> run_off(1, 0);
  std::vector<char> in_run((size_t)nrx, 0);
  const int64_t kMinRun = 4;
  for (int a = 0; a < (d <= 2 ? d : 0); ++a) {  // in 3D no runs: every receiver by its tile
    std::map<uint64_t, std::vector<int32_t>> groups;  // by the exact coordinate across axis a
    for (int64_t r = 0; r < nrx; ++r) {
      if (in_run[r]) continue;
      uint64_t key = 0;
      if (d == 2) std::memcpy(&key, &x[(size_t)r * d + (1 - a)], sizeof(double));
      groups[key].push_back((int32_t)r);
    }
    for (auto& kv : groups) {
      std::vector<int32_t>& g = kv.second;
      if ((int64_t)g.size() < kMinRun) continue;
      std::stable_sort(g.begin(), g.end(), [&](int32_t u, int32_t v) {
        return x[(size_t)u * d + a] < x[(size_t)v * d + a];
      });
      size_t i = 0;
      while (i + 1 < g.size()) {
        const double x0 = x[(size_t)g[i] * d + a];
        const double dl = x[(size_t)g[i + 1] * d + a] - x0;
        size_t j = i + 1;
        if (dl > 0.0)
          while (j + 1 < g.size() &&
                 std::fabs((x[(size_t)g[j + 1] * d + a] - x[(size_t)g[j] * d + a]) - dl) <= 1e-9 * dl)
            ++j;
        bool ok = dl > 0.0 && (int64_t)(j - i + 1) >= kMinRun;
        // spacing from the end points; every position of the run x0 + m * step must be
        // within a few ulps of the given coordinate (the kernels use the former)
        const double step = ok ? (x[(size_t)g[j] * d + a] - x0) / (double)(j - i) : 0.0;
        if (ok) {
          const double tol = 8.0 * 2.220446049250313e-16 *
                             std::max(std::fabs(x0), std::fabs(x[(size_t)g[j] * d + a]));
          for (size_t m = i; m <= j && ok; ++m)
            ok = std::fabs(std::fma((double)(m - i), step, x0) - x[(size_t)g[m] * d + a]) <= tol;
        }
        if (ok) {
          run_geo.push_back(x0);
          run_geo.push_back(step);
          run_geo.push_back(d == 2 ? x[(size_t)g[i] * d + (1 - a)] : 0.0);
          run_axis.push_back(a);
          for (size_t m = i; m <= j; ++m) {
            run_rx.push_back(g[m]);
            in_run[g[m]] = 1;
          }
          run_off.push_back((int64_t)run_rx.size());
          i = j + 1;
        } else {
          ++i;
        }
      }
    }
  }
  const int64_t nruns = (int64_t)run_axis.size();
  const int64_t nin_runs = (int64_t)run_rx.size();
  // the other receivers, grouped by output tile, after the runs in the internal order
  const int* nt = p->shots[0].ntile;
  int64_t nbins = 1;
  for (int k = 0; k < d; ++k) nbins *= nt[k];
  std::vector<int64_t> bin((size_t)nrx, -1), off((size_t)nbins + 1, 0);
  for (int64_t r = 0; r < nrx; ++r) {
    if (in_run[r]) continue;
    int64_t b = 0;
    for (int k = 0; k < d; ++k) {
      double v = x[(size_t)r * d + k];
      int64_t i = (int64_t)std::floor((v - gd.o[k]) * gd.inv_h[k]);
      i = std::min<int64_t>(std::max<int64_t>(i, 0), gd.n[k] - 1);
      b = b * nt[k] + i / gd.tile[k];
    }
    bin[r] = b;
    off[b + 1] += 1;
  }
  off[0] = nin_runs;
  for (int64_t b = 0; b < nbins; ++b) off[b + 1] += off[b];
  std::vector<int32_t> perm(run_rx);  // internal index -> caller's index
  perm.resize((size_t)nrx);
  std::vector<int64_t> fill(off.begin(), off.end() - 1);
  for (int64_t r = 0; r < nrx; ++r)
    if (bin[r] >= 0) perm[fill[bin[r]]++] = (int32_t)r;
  std::vector<double> xi((size_t)nrx * d);
  for (int64_t i = 0; i < nrx; ++i)
    for (int k = 0; k < d; ++k) xi[(size_t)i * d + k] = x[(size_t)perm[i] * d + k];
  const int64_t nrec = p->nsteps / record_every + 1;
  CUDA_OR_FAIL(p, cudaMalloc(&p->d_rx, sizeof(double) * xi.size()));
  CUDA_OR_FAIL(p, cudaMalloc(&p->d_rx_off, sizeof(int64_t) * off.size()));
  CUDA_OR_FAIL(p, cudaMalloc(&p->d_rx_perm, sizeof(int32_t) * perm.size()));
  CUDA_OR_FAIL(p, cudaMalloc(&p->d_traces, sizeof(double) * p->nshots * nrec * nrx));
  CUDA_OR_FAIL(p, cudaMemcpy(p->d_rx, xi.data(), sizeof(double) * xi.size(), cudaMemcpyHostToDevice));
  CUDA_OR_FAIL(p, cudaMemcpy(p->d_rx_off, off.data(), sizeof(int64_t) * off.size(), cudaMemcpyHostToDevice));
  CUDA_OR_FAIL(p, cudaMemcpy(p->d_rx_perm, perm.data(), sizeof(int32_t) * perm.size(), cudaMemcpyHostToDevice));
  if (nruns > 0) {
    CUDA_OR_FAIL(p, cudaMalloc(&p->d_run_geo, sizeof(double) * run_geo.size()));
    CUDA_OR_FAIL(p, cudaMalloc(&p->d_run_axis, sizeof(int32_t) * run_axis.size()));
    CUDA_OR_FAIL(p, cudaMalloc(&p->d_run_off, sizeof(int64_t) * run_off.size()));
    CUDA_OR_FAIL(p, cudaMemcpy(p->d_run_geo, run_geo.data(), sizeof(double) * run_geo.size(),
                               cudaMemcpyHostToDevice));
    CUDA_OR_FAIL(p, cudaMemcpy(p->d_run_axis, run_axis.data(), sizeof(int32_t) * run_axis.size(),
                               cudaMemcpyHostToDevice));
    CUDA_OR_FAIL(p, cudaMemcpy(p->d_run_off, run_off.data(), sizeof(int64_t) * run_off.size(),
                               cudaMemcpyHostToDevice));
  }
  p->nrx = nrx;
  p->rx.nrx = nrx;
  p->rx.nrec = nrec;
  p->rx.every = record_every;
  p->rx.x = p->d_rx;
  p->rx.off = p->d_rx_off;
  p->rx.nruns = nruns;
  p->rx.run_geo = p->d_run_geo;
  p->rx.run_axis = p->d_run_axis;
  p->rx.run_off = p->d_run_off;
  for (int k = 0; k < fga::kMaxDim; ++k) p->rx.ntile[k] = k < d ? nt[k] : 1;
  if (p->stage >= 2) p->stage = 1;  // traces need a new propagation
  return FGA_OK;
}

fga_status fga_traces(fga_plan_t p, double* traces) {
  fga_status st = check_usable(p);
  if (st != FGA_OK) return st;
  if (p->nrx == 0) return fail(p, FGA_ERR_STATE, "no receivers set");
  if (p->stage < 2) return fail(p, FGA_ERR_STATE, "not propagated since the receivers were set");
  if (!traces) return fail(p, FGA_ERR_INVALID, "traces must not be NULL");
  size_t n = (size_t)p->nshots * p->rx.nrec * p->rx.nrx;
  CUDA_OR_FAIL(p, cudaMemcpyAsync(traces, p->d_traces, sizeof(double) * n, cudaMemcpyDefault, p->stream));
  return read_status(p);
}

fga_status fga_grad(fga_plan_t p, const double* residual, double* grad) {
  fga_status st = check_usable(p);
  if (st != FGA_OK) return st;
  if (p->nrx == 0) return fail(p, FGA_ERR_STATE, "fga_grad needs receivers (fga_set_receivers)");
  if (p->stage < 2) return fail(p, FGA_ERR_STATE, "fga_grad before fga_propagate");
  if (!residual || !grad) return fail(p, FGA_ERR_INVALID, "residual and grad must not be NULL");
  const GridDev& gd = p->grid;
  const size_t nres = (size_t)p->nshots * p->rx.nrec * p->rx.nrx;
  const double* d_res = residual;
  if (!is_device_ptr(residual)) {
    CUDA_OR_FAIL(p, grow(&p->d_resid, &p->resid_cap, nres));
    CUDA_OR_FAIL(p, cudaMemcpyAsync(p->d_resid, residual, sizeof(double) * nres, cudaMemcpyDefault,
                                    p->stream));
    d_res = p->d_resid;
  }
  // to the internal receiver order of the kernels
  CUDA_OR_FAIL(p, grow(&p->d_resid_int, &p->resid_int_cap, nres));
  CUDA_OR_FAIL(p, fga::launch_gather_rows(p, d_res, p->d_rx_perm, (int64_t)p->nshots * p->rx.nrec,
                                          p->rx.nrx, p->d_resid_int));
  d_res = p->d_resid_int;
  const int64_t nthr = fga::adjoint_threads(p);
  if (nthr <= 0) return fail(p, FGA_ERR_CUDA, "occupancy query for the adjoint kernel failed", true);
  // Every state and stage state of a ray recorded by the forward pass (one segment) when
  // that fits in half of the free device memory; otherwise checkpoints every
  // kseg ~ sqrt(nsteps) steps and one segment of kseg states (and their stage states)
  // recomputed at a time. Per resident thread: ncheck checkpoints + 4 kseg states.
  int64_t kseg = p->nsteps + 1, ncheck = 0;
  {
    size_t free_b = 0, total_b = 0;
    CUDA_OR_FAIL(p, cudaMemGetInfo(&free_b, &total_b));
    const double full = (double)nthr * (double)(4 * kseg) * (double)p->nfields * sizeof(double);
    const double avail = (double)free_b + (double)p->adj_scratch_cap * sizeof(double);
    if (p->adj_force_segments || full > 0.5 * avail) {
      kseg = std::max<int64_t>(1, (int64_t)std::ceil(std::sqrt((double)std::max<int64_t>(p->nsteps, 1))));
      ncheck = p->nsteps / kseg + 2;
    }
  }
  const size_t need = (size_t)nthr * (size_t)(ncheck + 4 * kseg) * (size_t)p->nfields;
  CUDA_OR_FAIL(p, grow(&p->d_adj_scratch, &p->adj_scratch_cap, need));
  double* dst = grad;
  bool host_out = !is_device_ptr(grad);
  if (host_out) {
    if (!p->d_grad) CUDA_OR_FAIL(p, cudaMalloc(&p->d_grad, sizeof(double) * gd.npts));
    dst = p->d_grad;
  }
  CUDA_OR_FAIL(p, grow(&p->d_part, &p->part_cap,
                       (size_t)(fga::adjoint_slices(p, nthr) * gd.npts)));
  CUDA_OR_FAIL(p, grow(&p->d_adj_bucket, &p->adj_bucket_cap,
                       (size_t)(p->nsteps / fga::adjoint_sort_width(p->nsteps) + 2)));
  CUDA_OR_FAIL(p, fga::launch_adjoint(p, d_res, dst, p->d_adj_scratch, nthr, kseg, ncheck));
  if (p->interp == FGA_BSPLINE_INTERP) {
    // dJ/dc = B^{-T} dJ/dC for C = B^{-1} c; B is symmetric, so this is the prefilter again
    std::vector<double> hg((size_t)gd.npts);
    CUDA_OR_FAIL(p, cudaMemcpyAsync(hg.data(), dst, sizeof(double) * gd.npts, cudaMemcpyDeviceToHost,
                                    p->stream));
    CUDA_OR_FAIL(p, cudaStreamSynchronize(p->stream));
    prefilter_grid(gd.dim, gd.n, gd.periodic, hg.data());
    if (host_out) {
      std::memcpy(grad, hg.data(), sizeof(double) * gd.npts);
    } else {
      CUDA_OR_FAIL(p, cudaMemcpyAsync(grad, hg.data(), sizeof(double) * gd.npts,
                                      cudaMemcpyHostToDevice, p->stream));
      CUDA_OR_FAIL(p, cudaStreamSynchronize(p->stream));
    }
    return read_status(p);
  }
  if (host_out)
    CUDA_OR_FAIL(p, cudaMemcpyAsync(grad, dst, sizeof(double) * gd.npts, cudaMemcpyDeviceToHost,
                                    p->stream));
  return read_status(p);
}

int64_t fga_ray_steps(fga_plan_t p) {
  if (!p || p->stage < 2 || p->failed) return -1;
  unsigned long long v = 0;
  if (cudaMemcpyAsync(&v, p->d_steps, sizeof(v), cudaMemcpyDeviceToHost, p->stream) != cudaSuccess ||
      cudaStreamSynchronize(p->stream) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  return (int64_t)v;
}

fga_status fga_stage_times(fga_plan_t p, double* ms5, int64_t* launches) {
  if (!p) return fail(nullptr, FGA_ERR_INVALID, "plan is NULL");
  if (ms5) {
    CUDA_OR_FAIL(p, cudaStreamSynchronize(p->stream));
    const int from[5] = {0, 1, 3, 5, 6}, to[5] = {1, 2, 4, 6, 7};
    for (int i = 0; i < 5; ++i) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, p->ev[from[i]], p->ev[to[i]]) != cudaSuccess) {
        cudaGetLastError();
        ms = -1.f;
      }
      ms5[i] = ms;
    }
  }
  if (launches) *launches = p->launches;
  return FGA_OK;
}

fga_status fga_spline_prefilter(int dim, const int64_t* n, const int* periodic,
                                const double* samples, double* coef) {
  if (dim < 1 || dim > fga::kMaxDim || !n || !periodic || !samples || !coef)
    return fail(nullptr, FGA_ERR_INVALID, "fga_spline_prefilter: bad arguments");
  int64_t total = 1;
  for (int k = 0; k < dim; ++k) {
    if (n[k] < 4 || n[k] > ((int64_t)1 << 30))
      return fail(nullptr, FGA_ERR_INVALID, "fga_spline_prefilter: grid size out of range");
    total *= n[k];
  }
  if (coef != samples) std::memmove(coef, samples, sizeof(double) * total);
  prefilter_grid(dim, n, periodic, coef);
  return FGA_OK;
}

}  // extern "C"
