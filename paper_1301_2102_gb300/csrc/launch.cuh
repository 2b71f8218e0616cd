// Host-side launchers of the persistent solve kernel, one explicit instantiation per
// (vector type, maximum block size PM) in the solver_*.cu translation units.
#pragma once
#include <cuda_runtime.h>
#include "solver.cuh"

namespace bmr {

constexpr int SOLVE_NT = 256;  // 7 streaming warps + 1 control warp

template <typename V, int PM>
struct SolveLauncher {
  static size_t smem() { return solve_smem_bytes<V, PM, SOLVE_NT>(); }
  // blocks of the kernel that fit on one SM (0 if it cannot run)
  static int blocks_per_sm();
  static cudaError_t launch(const SolveArgs<V>& args, int grid, cudaStream_t stream);
};

#define BMR_DEFINE_LAUNCHER(V, PM)                                                                        \
  template <>                                                                                             \
  int SolveLauncher<V, PM>::blocks_per_sm() {                                                             \
    auto fn = bminres_solve_kernel<V, PM, SOLVE_NT>;                                                      \
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem()) != cudaSuccess) \
      return 0;                                                                                           \
    int nb = 0;                                                                                           \
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, SOLVE_NT, smem()) != cudaSuccess) return 0; \
    return nb;                                                                                            \
  }                                                                                                       \
  template <>                                                                                             \
  cudaError_t SolveLauncher<V, PM>::launch(const SolveArgs<V>& args, int grid, cudaStream_t stream) {     \
    auto fn = bminres_solve_kernel<V, PM, SOLVE_NT>;                                                      \
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem());  \
    if (e != cudaSuccess) return e;                                                                       \
    SolveArgs<V> a = args;                                                                                \
    void* kargs[] = {(void*)&a};                                                                          \
    return cudaLaunchCooperativeKernel((const void*)fn, dim3(grid), dim3(SOLVE_NT), kargs, smem(), stream); \
  }

}  // namespace bmr
