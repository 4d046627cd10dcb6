// Float64 FMA throughput of the current device, the unit that bounds the
// outer Krylov operator (eight float64 FMAs per finest point, one neighbour
// load each) on GPUs whose float64 pipe is narrow.  A measurement helper for
// roofline figures; no solve calls it.  What it times is a lower bound on the
// pipe's rate: on GB300 long launches of the float64 operator run faster.
//
// Every thread runs PK_CHAINS independent recurrences a <- a * m + c, so the
// float64 pipe has independent instructions to issue.  With m = 1 - 2^-10 and
// c = 2^-10 every chain stays in [1, 2) (its fixed point is 1): no overflow,
// no subnormals.
#include <cuda_runtime.h>

#include <algorithm>

#include "mg.h"

namespace {

constexpr int PK_THREADS = 256;
constexpr int PK_BLOCKS_PER_SM = 4;  // 1024 resident threads per SM
constexpr int PK_CHAINS = 8;
constexpr int PK_ITERS = 8192;       // about 16 ms per launch at 2 FMAs per clock per SM

__global__ void __launch_bounds__(PK_THREADS) k_fp64_fma_chains(int iters, double m, double c, double* out) {
  double a[PK_CHAINS];
#pragma unroll
  for (int u = 0; u < PK_CHAINS; ++u) a[u] = 1.0 + 0.0625 * u + 1e-6 * threadIdx.x;
#pragma unroll 4
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < PK_CHAINS; ++u) a[u] = fma(a[u], m, c);
  }
  double s = 0.0;
#pragma unroll
  for (int u = 0; u < PK_CHAINS; ++u) s += a[u];
  // Never true (every chain stays in [1, 2)); the store keeps the chains live.
  if (s < 0.0) out[blockIdx.x * PK_THREADS + threadIdx.x] = s;
}

}  // namespace

extern "C" mg_status mg_fp64_fma_peak(int launches, double* tflops) {
  if (launches < 1 || launches > 100 || !tflops) return MG_ERR_ARG;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MG_ERR_CUDA;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return MG_ERR_CUDA;
  const int blocks = nsm * PK_BLOCKS_PER_SM;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  double* out = nullptr;
  mg_status st = MG_OK;
  double best_ms = 0.0;
  const double m = 1.0 - 1.0 / 1024.0, c = 1.0 / 1024.0;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
      cudaMalloc(&out, sizeof(double) * (size_t)blocks * PK_THREADS) != cudaSuccess) {
    st = MG_ERR_CUDA;
  } else {
    k_fp64_fma_chains<<<blocks, PK_THREADS, 0, s>>>(PK_ITERS, m, c, out);  // untimed: clocks ramp up
    for (int t = 0; t < launches && st == MG_OK; ++t) {
      float ms = 0.0f;
      if (cudaEventRecord(e0, s) != cudaSuccess) st = MG_ERR_CUDA;
      k_fp64_fma_chains<<<blocks, PK_THREADS, 0, s>>>(PK_ITERS, m, c, out);
      if (st == MG_OK && (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1, s) != cudaSuccess ||
                          cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
        st = MG_ERR_CUDA;
      if (st == MG_OK && ms > 0.0f) best_ms = best_ms > 0.0 ? std::min(best_ms, (double)ms) : (double)ms;
    }
    if (st == MG_OK && !(best_ms > 0.0)) st = MG_ERR_CUDA;
  }
  if (st == MG_OK) {
    const double fmas = (double)blocks * PK_THREADS * PK_CHAINS * PK_ITERS;
    *tflops = 2.0 * fmas / (best_ms * 1e-3) / 1e12;
  }
  if (s) cudaStreamSynchronize(s);
  if (out) cudaFree(out);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  return st;
}
