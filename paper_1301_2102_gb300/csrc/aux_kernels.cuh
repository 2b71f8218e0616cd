// Non-persistent kernels around the solve: residual R = B - A X (FP64) written as column vectors,
// the block product Y = A X, the sampled outer product for the adjoint, and X += D.  Defined in
// this header with internal linkage so that each translation unit that launches them has its own.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "dword.cuh"

namespace bmr {

constexpr int AUX_NT = 256;
constexpr int AUX_CH = 8;  // right-hand-side columns handled per sweep of a row

// F[c] = B[:, c] - (A X)[:, c] for c < p, stored as column vectors of type V (stride ld), and the
// per-block partial sums of ||F[:, c]||^2 (computed from the FP64 values) into part[c][block].
template <typename V>
__global__ void __launch_bounds__(AUX_NT) residual_kernel(int64_t n, int p, const int32_t* __restrict__ rowptr,
                                                          const int32_t* __restrict__ colidx,
                                                          const double* __restrict__ vals, const double* B,
                                                          const double* X, V* F, int64_t ld, double* part) {
  __shared__ double red[AUX_NT / 32][32];
  const int64_t r = (int64_t)blockIdx.x * AUX_NT + threadIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int c0 = 0; c0 < p; c0 += AUX_CH) {
    double acc[AUX_CH];
#pragma unroll
    for (int c = 0; c < AUX_CH; ++c) acc[c] = 0.0;
    if (r < n) {
      const int32_t k0 = rowptr[r], k1 = rowptr[r + 1];
      for (int32_t k = k0; k < k1; ++k) {
        const double a = vals[k];
        const double* xr = X + (int64_t)colidx[k] * p + c0;
#pragma unroll
        for (int c = 0; c < AUX_CH; ++c)
          if (c0 + c < p) acc[c] += a * xr[c];
      }
#pragma unroll
      for (int c = 0; c < AUX_CH; ++c)
        if (c0 + c < p) {
          double f = B[r * p + c0 + c] - acc[c];
          acc[c] = f;
          F[(int64_t)(c0 + c) * ld + r] = (V)f;
        }
    }
    // block partial of ||f_c||^2 in a fixed order
#pragma unroll
    for (int c = 0; c < AUX_CH; ++c) {
      double s = (r < n && c0 + c < p) ? acc[c] * acc[c] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) red[warp][c] = s;
    }
    __syncthreads();
    if (threadIdx.x < AUX_CH && c0 + (int)threadIdx.x < p) {
      double s = 0.0;
      for (int w = 0; w < AUX_NT / 32; ++w) s += red[w][threadIdx.x];
      part[(int64_t)(c0 + threadIdx.x) * gridDim.x + blockIdx.x] = s;
    }
    __syncthreads();
  }
}

// out[c] = sqrt(sum_b part[c][b]) for c < p (one block, fixed order).
static __global__ void finish_norms_kernel(int p, int nparts, const double* part, double* out) {
  __shared__ double red[AUX_NT];
  for (int c = 0; c < p; ++c) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nparts; b += AUX_NT) s += part[(int64_t)c * nparts + b];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = AUX_NT / 2; h > 0; h >>= 1) {
      if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[c] = sqrt(red[0]);
    __syncthreads();
  }
}

// Y = A X for row-major n x p blocks, FP64, CSR summation order.
static __global__ void __launch_bounds__(AUX_NT) spmm_kernel(int64_t n, int p, const int32_t* __restrict__ rowptr,
                                                      const int32_t* __restrict__ colidx,
                                                      const double* __restrict__ vals, const double* X, double* Y) {
  const int64_t r = (int64_t)blockIdx.x * AUX_NT + threadIdx.x;
  if (r >= n) return;
  const int32_t k0 = rowptr[r], k1 = rowptr[r + 1];
  for (int c0 = 0; c0 < p; c0 += AUX_CH) {
    double acc[AUX_CH];
#pragma unroll
    for (int c = 0; c < AUX_CH; ++c) acc[c] = 0.0;
    for (int32_t k = k0; k < k1; ++k) {
      const double a = vals[k];
      const double* xr = X + (int64_t)colidx[k] * p + c0;
#pragma unroll
      for (int c = 0; c < AUX_CH; ++c)
        if (c0 + c < p) acc[c] += a * xr[c];
    }
#pragma unroll
    for (int c = 0; c < AUX_CH; ++c)
      if (c0 + c < p) Y[r * p + c0 + c] = acc[c];
  }
}

// dA[k] = -sum_c L[row_k, c] * X[col_k, c] for every stored entry k (row-major n x p L and X).
static __global__ void __launch_bounds__(AUX_NT) sddmm_kernel(int64_t n, int p, const int32_t* __restrict__ rowptr,
                                                       const int32_t* __restrict__ colidx, const double* Lm,
                                                       const double* X, double* dA) {
  const int64_t r = (int64_t)blockIdx.x * AUX_NT + threadIdx.x;
  if (r >= n) return;
  const double* lr = Lm + r * p;
  for (int32_t k = rowptr[r]; k < rowptr[r + 1]; ++k) {
    const double* xr = X + (int64_t)colidx[k] * p;
    double s = 0.0;
    for (int c = 0; c < p; ++c) s += lr[c] * xr[c];
    dA[k] = -s;
  }
}

__device__ __forceinline__ double as_double(double x) { return x; }
__device__ __forceinline__ double as_double(float x) { return (double)x; }
__device__ __forceinline__ double as_double(dw x) { return to_double(x); }

// X += D (FP64 += inner vector type), row-major n x p, and D = 0.
template <typename V>
__global__ void add_correction_kernel(int64_t total, double* X, V* D) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    X[i] += as_double(D[i]);
    D[i] = V(0);
  }
}

// Copy of the matrix values in the inner vector type (rounded to nearest).
template <typename V>
__global__ void to_vec_kernel(int64_t total, const double* a, V* b) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = V(a[i]);
}

}  // namespace bmr
