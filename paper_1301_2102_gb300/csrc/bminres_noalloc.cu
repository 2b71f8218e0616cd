// bminres_solve_noalloc: the FP64 solve with every piece of workspace carved out of one static
// device array, for callers that cannot call cudaMalloc: code whose device memory belongs to another
// framework's pool (a raw allocation fragments it or breaks its budget) and latency-critical loops
// that cannot take the implicit device-wide synchronisation of cudaMalloc / cudaFree.  It launches
// the same kernels as bminres_solve (residual, persistent solve, residual); nothing here allocates
// device or host memory, events or streams.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "../../include/bminres.h"
#include "aux_kernels.cuh"
#include "launch.cuh"
#include "pointer_kind.h"

namespace {

// The scratch array.  In host code `g_noalloc_scratch` names a host-side stand-in, not device
// memory: its device address comes from cudaGetSymbolAddress, once per device.
__device__ __align__(256) unsigned char g_noalloc_scratch[BMINRES_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up on first use).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

// true for device memory of the current device (or managed memory); false for host memory and
// for memory of another GPU, which the kernels cannot read without peer access
bool on_device(const void* p) {
  cudaPointerAttributes at;
  if (!p || cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) cudaGetLastError();
  return bmr::mem_kind(true, (int)at.type, at.device, dev) == bmr::MemKind::device;
}

int pm_of(int p) {
  int pm = 1;
  while (pm < p) pm <<= 1;
  return pm;
}

int blocks_per_sm_f64(int pm) {
  switch (pm) {
    case 1: return bmr::SolveLauncher<double, 1>::blocks_per_sm();
    case 2: return bmr::SolveLauncher<double, 2>::blocks_per_sm();
    case 4: return bmr::SolveLauncher<double, 4>::blocks_per_sm();
    case 8: return bmr::SolveLauncher<double, 8>::blocks_per_sm();
    case 16: return bmr::SolveLauncher<double, 16>::blocks_per_sm();
    case 32: return bmr::SolveLauncher<double, 32>::blocks_per_sm();
  }
  return 0;
}

cudaError_t launch_f64(int pm, const bmr::SolveArgs<double>& a, int grid, cudaStream_t s) {
  switch (pm) {
    case 1: return bmr::SolveLauncher<double, 1>::launch(a, grid, s);
    case 2: return bmr::SolveLauncher<double, 2>::launch(a, grid, s);
    case 4: return bmr::SolveLauncher<double, 4>::launch(a, grid, s);
    case 8: return bmr::SolveLauncher<double, 8>::launch(a, grid, s);
    case 16: return bmr::SolveLauncher<double, 16>::launch(a, grid, s);
    case 32: return bmr::SolveLauncher<double, 32>::launch(a, grid, s);
  }
  return cudaErrorInvalidValue;
}

int nvmax_of(int pm) {
  switch (pm) {
    case 1: return bmr::Layout<1>::NVMAX;
    case 2: return bmr::Layout<2>::NVMAX;
    case 4: return bmr::Layout<4>::NVMAX;
    case 8: return bmr::Layout<8>::NVMAX;
    case 16: return bmr::Layout<16>::NVMAX;
    case 32: return bmr::Layout<32>::NVMAX;
  }
  return 0;
}

constexpr size_t align256(size_t b) { return (b + 255) / 256 * 256; }

bminres_status status_of(int st) {
  switch (st) {
    case bmr::ST_OK: return BMINRES_OK;
    case bmr::ST_NOT_CONVERGED: return BMINRES_NOT_CONVERGED;
    case bmr::ST_ERR_BREAKDOWN: return BMINRES_ERR_BREAKDOWN;
    case bmr::ST_ERR_BENCH: return BMINRES_ERR_BENCH_EXHAUSTED;
    case bmr::ST_ERR_NONFINITE: return BMINRES_ERR_NONFINITE;
    case bmr::ST_ERR_TIMEOUT: return BMINRES_ERR_TIMEOUT;
  }
  return BMINRES_ERR_CUDA;
}

#define NA_TRY(expr)                                                    \
  do {                                                                  \
    if ((expr) != cudaSuccess) return BMINRES_ERR_CUDA;                 \
  } while (0)

}  // namespace

extern "C" bminres_status bminres_solve_noalloc(int64_t n, int64_t nnz, const int32_t* rowptr,
                                                const int32_t* colidx, const double* vals, int p,
                                                const double* B, double* X, double tol, int maxit,
                                                const bminres_opts* opts, bminres_stream stream,
                                                double* relres_true, bminres_info* info) {
  if (info) memset(info, 0, sizeof(*info));
  bminres_opts o;
  bminres_default_opts(&o);
  if (opts) o = *opts;
  if (n < 0 || nnz < 0 || nnz >= ((int64_t)1 << 31) || n >= ((int64_t)1 << 31) || p < 0 || p > 32 ||
      maxit < 0 || !(tol > 0.0) || o.precision != BMINRES_FP64 || o.bench < 0 || o.bench > bmr::NBMAX ||
      !(o.gamma >= 0.0))
    return BMINRES_ERR_INVALID;
  if (n == 0 || p == 0) return BMINRES_OK;
  if (p > n) return BMINRES_ERR_INVALID;

  // workspace layout inside the scratch array (same pieces as a handle's workspace)
  const int pm = pm_of(p);
  const int64_t ld = (n + 63) / 64 * 64;
  const int nb = std::max(o.bench, 1);
  int num_sms = 0, dev = 0;
  NA_TRY(cudaGetDevice(&dev));
  NA_TRY(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev));
  const int bps = blocks_per_sm_f64(pm);
  if (bps <= 0) return BMINRES_ERR_CUDA;
  const int64_t grid64 =
      std::max<int64_t>(1, std::min<int64_t>((int64_t)bps * num_sms, (n + 511) / 512));
  const int grid = (int)(o.max_blocks > 0 ? std::min<int64_t>(grid64, o.max_blocks) : grid64);
  const int nres = (int)((n + bmr::AUX_NT - 1) / bmr::AUX_NT);
  // the control block and both sets of column norms sit side by side, so that one copy at the end
  // brings every result the host needs
  size_t off = 0;
  const size_t oCtl = off; off += align256(sizeof(bmr::Ctl));
  const size_t oNo0 = off; off += sizeof(double) * 64;  // ||f0_i||
  const size_t oNo1 = off; off += sizeof(double) * 64;  // ||b_i - A x_i|| after the solve
  const size_t tail_bytes = off;
  off = align256(off);
  const size_t oU = off; off += align256(sizeof(double) * 2 * p * ld);
  const size_t oW = off; off += align256(sizeof(double) * p * ld);
  const size_t oM = off; off += align256(sizeof(double) * 2 * p * ld);
  const size_t oB = off; off += align256(sizeof(double) * nb * ld);
  const size_t oG = off; off += align256(sizeof(double) * nb * ld);
  const size_t oF = off; off += align256(sizeof(double) * p * ld);
  const size_t oP = off; off += align256(sizeof(double) * 2 * (size_t)nvmax_of(pm) * grid);
  const size_t oN = off; off += align256(sizeof(double) * (size_t)p * nres);
  if (off > BMINRES_NOALLOC_SCRATCH_BYTES) return BMINRES_ERR_INVALID;  // does not fit the array
  if (!on_device(rowptr) || (nnz > 0 && (!on_device(colidx) || !on_device(vals))) || !on_device(B) ||
      !on_device(X))
    return BMINRES_ERR_INVALID;

  void* base = nullptr;
  NA_TRY(scratch_address(&base));
  char* sb = static_cast<char*>(base);
  bmr::Ctl* ctl = reinterpret_cast<bmr::Ctl*>(sb + oCtl);
  double* U = reinterpret_cast<double*>(sb + oU);
  double* W = reinterpret_cast<double*>(sb + oW);
  double* M = reinterpret_cast<double*>(sb + oM);
  double* Bench = reinterpret_cast<double*>(sb + oB);
  double* Ghost = reinterpret_cast<double*>(sb + oG);
  double* F = reinterpret_cast<double*>(sb + oF);
  double* part = reinterpret_cast<double*>(sb + oP);
  double* npart = reinterpret_cast<double*>(sb + oN);
  double* norms0 = reinterpret_cast<double*>(sb + oNo0);
  double* norms1 = reinterpret_cast<double*>(sb + oNo1);
  cudaStream_t s = (cudaStream_t)stream;

  // the array keeps the previous call's contents: clear what the solve expects to start at zero
  NA_TRY(cudaMemsetAsync(U, 0, sizeof(double) * 2 * p * ld, s));
  NA_TRY(cudaMemsetAsync(M, 0, sizeof(double) * 2 * p * ld, s));
  NA_TRY(cudaMemsetAsync(Ghost, 0, sizeof(double) * nb * ld, s));
  NA_TRY(cudaMemsetAsync(ctl, 0, sizeof(bmr::Ctl), s));

  // F0 = B - A X0 (FP64) and its column norms
  bmr::residual_kernel<double><<<nres, bmr::AUX_NT, 0, s>>>(n, p, rowptr, colidx, vals, B, X, F, ld, npart);
  NA_TRY(cudaGetLastError());
  bmr::finish_norms_kernel<<<1, bmr::AUX_NT, 0, s>>>(p, nres, npart, norms0);
  NA_TRY(cudaGetLastError());

  bmr::SolveArgs<double> a;
  memset(&a, 0, sizeof(a));
  a.n = n;
  a.ld = ld;
  a.p = p;
  a.nbench = o.bench;
  a.ghost = o.ghost;
  a.maxit = maxit;
  a.tol = tol;
  a.gamma = o.gamma;
  a.seed = o.seed;
  a.rowptr = rowptr;
  a.colidx = colidx;
  a.vals = vals;
  a.F = F;
  a.X = X;
  a.U = U;
  a.W = W;
  a.M = M;
  a.Bench = Bench;
  a.Ghost = Ghost;
  a.part = part;
  a.ctl = ctl;
  a.barrier_limit_ns = 10ull * 1000 * 1000 * 1000;
  NA_TRY(launch_f64(pm, a, grid, s));

  // FP64 true residual of the result
  bmr::residual_kernel<double><<<nres, bmr::AUX_NT, 0, s>>>(n, p, rowptr, colidx, vals, B, X, F, ld, npart);
  NA_TRY(cudaGetLastError());
  bmr::finish_norms_kernel<<<1, bmr::AUX_NT, 0, s>>>(p, nres, npart, norms1);
  NA_TRY(cudaGetLastError());
  // one copy of the control block and both norm sets (a stack buffer: nothing is allocated)
  alignas(16) unsigned char tail[align256(sizeof(bmr::Ctl)) + 2 * 64 * sizeof(double)];
  NA_TRY(cudaMemcpyAsync(tail, sb + oCtl, tail_bytes, cudaMemcpyDeviceToHost, s));
  NA_TRY(cudaStreamSynchronize(s));
  bmr::Ctl r;
  memcpy(&r, tail, sizeof(bmr::Ctl));
  const double* f0 = reinterpret_cast<const double*>(tail + oNo0);
  const double* rt = reinterpret_cast<const double*>(tail + oNo1);

  double worst = 0.0;
  for (int i = 0; i < p; ++i) {
    const double rel = f0[i] > 0.0 ? rt[i] / f0[i] : 0.0;
    if (relres_true) relres_true[i] = rel;
    worst = std::max(worst, rel);
  }
  bminres_status st = status_of(r.status);
  // the solve stops on the recursive residual (Eq. (comp-resid)); say so when the true one missed
  if (st == BMINRES_OK && worst > tol) st = BMINRES_RESIDUAL_GAP;
  if (info) {
    info->status = st;
    info->iters = r.iters;
    info->cycles = r.cycles;
    info->outer = 1;
    info->deflations = r.deflations;
    info->setup_deflations = r.setup_deflations;
    info->bench_used = r.bench_used;
    info->grid_blocks = grid;
    info->relres_est_max = r.relres_est_max;
    info->relres_true_max = worst;
    info->stream_ms = (r.t_stream + r.t_sp + r.t_dir) * 1e-6;
    info->spmm_ms = r.t_sp * 1e-6;
    info->dir_ms = r.t_dir * 1e-6;
    info->reduce_ms = r.t_reduce * 1e-6;
    info->scalar_ms = r.t_scalar * 1e-6;
    info->timeline_ms = r.t_total * 1e-6;
    info->qr_ms = r.t_qr * 1e-6;
    info->launches = 5;
  }
  return st;
}
