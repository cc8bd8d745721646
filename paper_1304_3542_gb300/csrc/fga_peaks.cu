// Measured fused multiply-add throughput of the current GPU in FP64 and FP32: the
// denominator of the roofline of the FP64-bound kernels (the ray integrator, the FP64
// FBI and gather) is checked against it. Not part of the method.
//
// Each thread runs 8 independent FMA chains x = fma(x, a, b) (so the pipe, not the
// dependency latency, sets the rate) for iters x 16 rounds; a and b come from the host,
// so nothing can be folded, and the result is stored only under a condition the
// compiler cannot decide. The grid is 8 blocks of 256 threads per SM.
#include <cuda_runtime.h>

#include <string>

#include "fga_internal.cuh"

namespace {

template <class T>
__global__ void __launch_bounds__(256) k_fma_chains(T* out, int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) x[u] = (T)(threadIdx.x + 7 * u) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 16; ++r)
#pragma unroll
      for (int u = 0; u < 8; ++u) x[u] = fma(x[u], a, b);
  }
  T s = 0;
#pragma unroll
  for (int u = 0; u < 8; ++u) s += x[u];
  if (s == (T)-1.0) out[blockIdx.x] = s;
}

}  // namespace

extern "C" fga_status fga_fma_peak(int bits, int iters, double* tflops, double* ms) {
  if ((bits != 32 && bits != 64) || iters < 1 || !tflops || !ms) {
    fga::set_unbound_error("fga_fma_peak: bits must be 32 or 64, iters >= 1, outputs non-NULL");
    return FGA_ERR_INVALID;
  }
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  void* out = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&out, 1 << 16);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const int blocks = 8 * sms, threads = 256;
  float t = 0.0f;
  if (e == cudaSuccess) {
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // the first launch warms up
      e = cudaEventRecord(e0, 0);
      if (bits == 64)
        k_fma_chains<double><<<blocks, threads>>>((double*)out, iters, 0.999999, 1e-7);
      else
        k_fma_chains<float><<<blocks, threads>>>((float*)out, iters, 0.999999f, 1e-7f);
      if (e == cudaSuccess) e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaEventRecord(e1, 0);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (out) cudaFree(out);
  if (e != cudaSuccess) {
    fga::set_unbound_error(std::string("fga_fma_peak: ") + cudaGetErrorString(e));
    return FGA_ERR_CUDA;
  }
  const double flops = 2.0 * 8.0 * 16.0 * (double)iters * (double)blocks * threads;
  *ms = (double)t;
  *tflops = flops / ((double)t * 1e-3) / 1e12;
  return FGA_OK;
}
