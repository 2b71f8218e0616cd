// bminres_fp64_peak: measured FP64 fused multiply-add throughput of the current GPU, the denominator
// of the arithmetic roofline that the FP64 solve is reported against (GB300's FP64 units, not its
// HBM, bound that solve).  A measurement helper of the library, not a step of the method.
//
// Every thread runs NCH independent FMA chains x <- x * m + c (m slightly below 1, so the values stay
// finite and normal), the loop unrolled by 4; the probe times three shapes (8 or 16 chains per
// thread, 4 or 8 blocks of 256 threads per SM) and reports the fastest, so that neither the FP64
// pipe's latency nor loop overhead hides its throughput.  Each shape is timed by CUDA events around
// one launch after one warm-up launch.
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/bminres.h"

namespace {

constexpr int NT = 256;

template <int NCH>
__global__ void __launch_bounds__(NT) fp64_fma_chains(int iters, double* out) {
  double x[NCH];
#pragma unroll
  for (int k = 0; k < NCH; ++k) x[k] = 1.0 + 1e-3 * k + 1e-9 * threadIdx.x;
  const double m = 0.9999999999, c = 1e-12;
#pragma unroll 4
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < NCH; ++k) x[k] = fma(x[k], m, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < NCH; ++k) s += x[k];
  if (s == 12345.678) out[0] = s;  // keeps the chains live; never true for these inputs
}

template <int NCH>
bool time_shape(int iters, int grid, cudaStream_t s, double* out, cudaEvent_t e0, cudaEvent_t e1, double* gflops,
                float* ms) {
  const int it = std::max(1, iters * 8 / NCH);
  fp64_fma_chains<NCH><<<grid, NT, 0, s>>>(std::max(1, it / 8), out);  // warm-up
  cudaEventRecord(e0, s);
  fp64_fma_chains<NCH><<<grid, NT, 0, s>>>(it, out);
  cudaEventRecord(e1, s);
  float t = 0.f;
  if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
      cudaEventElapsedTime(&t, e0, e1) != cudaSuccess || !(t > 0.f))
    return false;
  const double g = 2.0 * NCH * (double)it * (double)grid * NT / (t * 1e-3) / 1e9;
  if (g > *gflops) {
    *gflops = g;
    *ms = t;
  }
  return true;
}

}  // namespace

extern "C" bminres_status bminres_fp64_peak(int iters, bminres_stream stream, double* gflops, double* ms_out) {
  if (!gflops || iters <= 0) return BMINRES_ERR_INVALID;
  *gflops = 0.0;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return BMINRES_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  double* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  bminres_status st = BMINRES_ERR_CUDA;
  float ms = 0.f;
  if (cudaMalloc(&out, sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return BMINRES_ERR_OOM;
  }
  if (cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess &&
      time_shape<8>(iters, 8 * sms, s, out, e0, e1, gflops, &ms) &&
      time_shape<16>(iters, 8 * sms, s, out, e0, e1, gflops, &ms) &&
      time_shape<16>(iters, 4 * sms, s, out, e0, e1, gflops, &ms)) {
    if (ms_out) *ms_out = ms;
    st = BMINRES_OK;
  }
  cudaGetLastError();
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  return st;
}
