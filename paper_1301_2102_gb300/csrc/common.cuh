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
  unsigned long long bar_arrived;  // grid-barrier arrivals since the launch (nblocks per barrier)
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
  unsigned long long t_sp, t_dir;  // block-product and direction passes (t_stream: the fused passes)
};

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int ld_volatile_int(const int* p) { return *(volatile const int*)p; }

__device__ __forceinline__ unsigned long long ld_acquire64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add64(unsigned long long* p, unsigned long long v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Grid-wide barrier for a cooperative launch (all blocks co-resident).  Thread 0 of each block adds
// one to a 64-bit arrival counter (release: the block's writes, ordered before it by the block
// barrier, become visible with it) and waits (acquire) until the counter reaches nblocks * epoch,
// `epoch` counting the barriers this block has passed (the same sequence in every block).  Every
// wait is bounded: after `limit_ns` the block records ST_ERR_TIMEOUT in ctl->err and returns false,
// so a broken schedule ends the kernel instead of hanging the GPU.  Returns false if any block has
// recorded an error.
__device__ __forceinline__ bool grid_barrier(Ctl* ctl, unsigned nblocks, unsigned long long& epoch,
                                             unsigned long long limit_ns) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    epoch += 1;
    const unsigned long long target = epoch * nblocks;
    red_release_add64(&ctl->bar_arrived, 1ull);
    if (ld_acquire64(&ctl->bar_arrived) < target) {
      const unsigned long long t0 = gtimer();
      unsigned spins = 0;
      while (ld_acquire64(&ctl->bar_arrived) < target) {
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
    if (ld_volatile_int(&ctl->err) != 0) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// ---- bulk copies global -> shared completed on an mbarrier (PTX: cp.async.bulk, mbarrier) -------
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// make initialised mbarriers visible to the async proxy
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// order this thread's earlier generic-proxy accesses before its later async-proxy (bulk) accesses
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async;" ::: "memory"); }
// the single arrival of a phase, announcing `bytes` of bulk copies that complete on it
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\tselp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait until the phase with the given parity has completed; gives up after limit_ns.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, unsigned long long limit_ns) {
  if (mbar_test(bar, parity)) return true;
  const unsigned long long t0 = gtimer();
  while (!mbar_test(bar, parity))
    if (gtimer() - t0 > limit_ns) return false;
  return true;
}
// bytes (a multiple of 16) from 16-byte aligned global src to 16-byte aligned shared dst
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
// named barrier `id` over `count` threads (a multiple of 32)
__device__ __forceinline__ void named_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
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
