// Device helpers shared by the block MINRES kernels: bounded grid barrier, timers, counter-based
// bench generator, and the status codes the kernels report.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace bmr {

constexpr int NBMAX = 8;  // maximum bench vectors (and removed-vector slots)

// status values written by the kernels (same numbering as bminres_status)
enum : int {
  ST_OK = 0,
  ST_NOT_CONVERGED = 1,
  ST_ERR_BREAKDOWN = -4,
  ST_ERR_BENCH = -5,
  ST_ERR_NONFINITE = -6,
  ST_ERR_TIMEOUT = -7,
};

// Device-global control block, one per handle.  Zeroed before every persistent launch.
struct Ctl {
  unsigned bar_count;  // arrivals at the current barrier
  unsigned bar_gen;    // barrier generation
  int err;             // set to ST_ERR_TIMEOUT by a block whose wait ran out
  int status;          // final status (block 0)
  int iters;           // band iterations
  int cycles;          // block products
  int deflations;
  int setup_deflations;
  int bench_used;
  int pad0;
  double relres_est_max;
  // coarse timeline of block 0 (nanoseconds): streaming passes, reductions incl. barriers,
  // scalar work (band QR and coefficient bookkeeping)
  unsigned long long t_stream, t_reduce, t_scalar, t_total;
  unsigned long long t_qr;  // band QR steps of the control warp (overlapped with streaming)
};

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_volatile_int(const int* p) { return *(volatile const int*)p; }

// Grid-wide barrier for a cooperative launch (all blocks co-resident).  Every wait is bounded:
// after `limit_ns` the waiting block records ST_ERR_TIMEOUT in ctl->err and returns false, so a
// broken schedule ends the kernel instead of hanging the GPU.  Returns false if any block has
// recorded an error.
__device__ __forceinline__ bool grid_barrier(Ctl* ctl, unsigned nblocks, unsigned long long limit_ns) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    unsigned gen = ld_acquire(&ctl->bar_gen);
    __threadfence();
    unsigned arrived = atomicAdd(&ctl->bar_count, 1u) + 1u;
    if (arrived == nblocks) {
      atomicExch(&ctl->bar_count, 0u);
      __threadfence();
      st_release(&ctl->bar_gen, gen + 1u);
    } else {
      unsigned long long t0 = gtimer();
      unsigned spins = 0;
      while (ld_acquire(&ctl->bar_gen) == gen) {
        if ((++spins & 63u) == 0u) {
          if (gtimer() - t0 > limit_ns) {
            atomicExch(&ctl->err, ST_ERR_TIMEOUT);
            ok = 0;
            break;
          }
          if (ld_volatile_int(&ctl->err) != 0) {
            ok = 0;
            break;
          }
        }
      }
    }
    __threadfence();
    if (ld_volatile_int(&ctl->err) != 0) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) used counter-style: value t of the stream with
// seed s is mix(s + (t + 1) * golden).  Bench vector k, row r uses t = k * n + r.  Returns a
// uniform double in [-1, 1) carrying 53 random bits.
__device__ __forceinline__ double bench_value(uint64_t seed, int64_t k, int64_t n, int64_t r) {
  uint64_t t = (uint64_t)k * (uint64_t)n + (uint64_t)r;
  uint64_t z = seed + (t + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z = z ^ (z >> 31);
  return __dmul_rn((double)(z >> 11), 0x1.0p-52) - 1.0;
}

}  // namespace bmr
