// Host implementation of the C ABI declared in include/bminres.h.
//
// A solve is: residual kernel F0 = B - A X0 (FP64 arithmetic, stored in the vector precision) ->
// one cooperative launch of the persistent solve kernel -> residual kernel for the FP64 true
// residual.  The mixed mode wraps the FP32 persistent kernel in an FP64 iterative-refinement loop.
#include <cuda_runtime.h>

#include <algorithm>
#include <initializer_list>
#include <type_traits>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/bminres.h"
#include "aux_kernels.cuh"
#include "launch.cuh"
#include "pointer_kind.h"

namespace bmr {

struct Workspace {
  int p = 0;
  int prec = -1;
  int grid = 0;
  size_t bytes = 0;
  void* base = nullptr;
  void* U = nullptr;
  void* W = nullptr;
  void* M = nullptr;
  void* Bench = nullptr;
  void* Ghost = nullptr;
  void* F = nullptr;
  void* D = nullptr;      // mixed: correction, row-major n x p, inner vector type
  double* part = nullptr; // reductions of the persistent kernel
  double* npart = nullptr;// residual-norm partials
  double* norms = nullptr;// p norms (device)
  double* Xtmp = nullptr; // adjoint solve / staging
  double* Btmp = nullptr;
};

}  // namespace bmr

struct bminres_handle_s {
  int device = 0;
  int num_sms = 0;
  int64_t n = 0, nnz = 0;
  bminres_opts opts;
  int32_t* rowptr = nullptr;
  int32_t* colidx = nullptr;
  double* vals = nullptr;
  float* vals32 = nullptr;   // FP32 copy of the values (MIXED)
  bmr::dw* vals_dw = nullptr; // double-word copy of the values (MIXED_DW)
  bmr::Ctl* ctl = nullptr;      // device
  bmr::Ctl* ctl_host = nullptr; // pinned
  double* norms_host = nullptr; // pinned, 2 * 32
  bmr::Workspace ws;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, evk0 = nullptr, evk1 = nullptr;
  int launches = 0;  // kernels launched by the current call
  int hist_cap = 0;
  double* hist = nullptr;  // device, hist_cap * 32
  int hist_count = 0, hist_p = 0;
};

namespace {

using bmr::Ctl;

constexpr int PMAX = 32;
constexpr unsigned long long BARRIER_LIMIT_NS = 10ull * 1000 * 1000 * 1000;  // 10 s per wait

bminres_status from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return BMINRES_OK;
  if (e == cudaErrorMemoryAllocation) return BMINRES_ERR_OOM;
  return BMINRES_ERR_CUDA;
}
#define BMR_TRY(expr)                            \
  do {                                           \
    cudaError_t _e = (expr);                     \
    if (_e != cudaSuccess) return from_cuda(_e); \
  } while (0)

// Where a caller's pointer lives: host memory (pageable or pinned), device or managed memory of
// the current device, or memory of another device (rejected).
using Mem = bmr::MemKind;
static_assert(cudaMemoryTypeDevice == 2 && cudaMemoryTypeManaged == 3, "memory type numbering of mem_kind");
Mem classify(const void* p) {
  cudaPointerAttributes at;
  if (!p || cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return Mem::host;
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) cudaGetLastError();
  return bmr::mem_kind(true, (int)at.type, at.device, dev);
}
bool is_device_ptr(const void* p) { return classify(p) == Mem::device; }
// true if any of the pointers is device memory of another GPU
bool foreign(std::initializer_list<const void*> ps) {
  for (const void* p : ps)
    if (p && classify(p) == Mem::other_device) return true;
  return false;
}

int pm_for(int p) {
  int pm = 1;
  while (pm < p) pm <<= 1;
  return pm;
}

int64_t padded_ld(int64_t n) { return (n + 63) / 64 * 64; }

// largest block size with a kernel instantiation for vector type V (double-word: 16, the
// coefficient copies of p = 32 leave too little shared memory for staging)
template <typename V>
constexpr int pmax_of() { return std::is_same<V, bmr::dw>::value ? 16 : 32; }

template <typename V>
int blocks_per_sm(int pm) {
  switch (pm) {
    case 1: return bmr::SolveLauncher<V, 1>::blocks_per_sm();
    case 2: return bmr::SolveLauncher<V, 2>::blocks_per_sm();
    case 4: return bmr::SolveLauncher<V, 4>::blocks_per_sm();
    case 8: return bmr::SolveLauncher<V, 8>::blocks_per_sm();
    case 16: return bmr::SolveLauncher<V, 16>::blocks_per_sm();
    case 32:
      if constexpr (pmax_of<V>() >= 32) return bmr::SolveLauncher<V, 32>::blocks_per_sm();
  }
  return 0;
}
template <typename V>
cudaError_t launch_solve(int pm, const bmr::SolveArgs<V>& a, int grid, cudaStream_t s) {
  switch (pm) {
    case 1: return bmr::SolveLauncher<V, 1>::launch(a, grid, s);
    case 2: return bmr::SolveLauncher<V, 2>::launch(a, grid, s);
    case 4: return bmr::SolveLauncher<V, 4>::launch(a, grid, s);
    case 8: return bmr::SolveLauncher<V, 8>::launch(a, grid, s);
    case 16: return bmr::SolveLauncher<V, 16>::launch(a, grid, s);
    case 32:
      if constexpr (pmax_of<V>() >= 32) return bmr::SolveLauncher<V, 32>::launch(a, grid, s);
  }
  return cudaErrorInvalidValue;
}
int nvmax_for(int pm) {
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

// grid of the persistent kernel: one wave of co-resident blocks, fewer for small n
int solve_grid(bminres_handle h, int pm, int prec) {
  int bps = prec == 1 ? blocks_per_sm<float>(pm) : (prec == 2 ? blocks_per_sm<bmr::dw>(pm) : blocks_per_sm<double>(pm));
  if (bps <= 0) return 0;
  int64_t full = (int64_t)bps * h->num_sms;
  int64_t want = (h->n + 511) / 512;  // at least two rows per thread and pass
  int64_t g = std::max<int64_t>(1, std::min<int64_t>(full, want));
  if (h->opts.max_blocks > 0) g = std::min<int64_t>(g, h->opts.max_blocks);
  return (int)g;
}

void free_ws(bmr::Workspace& w) {
  if (w.base) cudaFree(w.base);
  w = bmr::Workspace();
}

// vector precision of the solves of a handle: 0 = FP64, 1 = FP32, 2 = double-word, 3 = FP64 refined
int prec_of(bminres_handle h) {
  switch (h->opts.precision) {
    case BMINRES_MIXED: return 1;
    case BMINRES_MIXED_DW: return 2;
    case BMINRES_FP64_REFINED: return 3;
  }
  return 0;
}

// (Re)allocate the workspace for block size p and vector precision prec (see prec_of).
bminres_status ensure_ws(bminres_handle h, int p, int prec) {
  bmr::Workspace& w = h->ws;
  const int pm = pm_for(p);
  const bool f32 = (prec == 1);
  const int grid = solve_grid(h, pm, prec);
  if (grid <= 0) return BMINRES_ERR_CUDA;
  if (w.base && w.p == p && w.prec == prec && w.grid == grid) return BMINRES_OK;
  free_ws(w);
  const int64_t ld = padded_ld(h->n);
  const size_t es = f32 ? sizeof(float) : sizeof(double);
  const int nb = std::max(h->opts.bench, 1);
  const size_t vecs = (size_t)(2 * p + p + 2 * p + nb + nb + p);
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  size_t off = 0;
  size_t oU = off; off += al(2 * p * ld * es);
  size_t oW = off; off += al(p * ld * es);
  size_t oM = off; off += al(2 * p * ld * es);
  size_t oB = off; off += al(nb * ld * es);
  size_t oG = off; off += al(nb * ld * es);
  size_t oF = off; off += al(p * ld * es);
  size_t oD = off; off += prec != 0 ? al((size_t)h->n * p * es) : 0;
  size_t oP = off; off += al((size_t)2 * nvmax_for(pm) * grid * sizeof(double));
  const int nres = (int)((h->n + bmr::AUX_NT - 1) / bmr::AUX_NT);
  size_t oN = off; off += al((size_t)p * std::max(nres, 1) * sizeof(double));
  size_t oNo = off; off += al((size_t)64 * sizeof(double));
  size_t oX = off; off += al((size_t)h->n * p * sizeof(double));
  size_t oBt = off; off += al((size_t)h->n * p * sizeof(double));
  (void)vecs;
  void* base = nullptr;
  cudaError_t e = cudaMalloc(&base, off);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return BMINRES_ERR_OOM;
  }
  char* b = (char*)base;
  w.base = base;
  w.bytes = off;
  w.p = p;
  w.prec = prec;
  w.grid = grid;
  w.U = b + oU;
  w.W = b + oW;
  w.M = b + oM;
  w.Bench = b + oB;
  w.Ghost = b + oG;
  w.F = b + oF;
  w.D = prec != 0 ? (void*)(b + oD) : nullptr;
  w.part = (double*)(b + oP);
  w.npart = (double*)(b + oN);
  w.norms = (double*)(b + oNo);
  w.Xtmp = (double*)(b + oX);
  w.Btmp = (double*)(b + oBt);
  return BMINRES_OK;
}

// residual F = B - A X (FP64), stored in the precision of the workspace; norms into h->norms_host
// when `norms_to_host` (synchronises the stream).
template <typename V>
bminres_status residual(bminres_handle h, int p, const double* B, const double* X, V* F, cudaStream_t s,
                        bool norms_to_host) {
  bmr::Workspace& w = h->ws;
  const int nres = (int)((h->n + bmr::AUX_NT - 1) / bmr::AUX_NT);
  const int64_t ld = padded_ld(h->n);
  if (nres > 0)
    bmr::residual_kernel<V><<<nres, bmr::AUX_NT, 0, s>>>(h->n, p, h->rowptr, h->colidx, h->vals, B, X, F, ld,
                                                          w.npart);
  BMR_TRY(cudaGetLastError());
  bmr::finish_norms_kernel<<<1, bmr::AUX_NT, 0, s>>>(p, nres, w.npart, w.norms);
  BMR_TRY(cudaGetLastError());
  h->launches += (nres > 0) ? 2 : 1;
  if (norms_to_host) {
    BMR_TRY(cudaMemcpyAsync(h->norms_host, w.norms, sizeof(double) * p, cudaMemcpyDeviceToHost, s));
    BMR_TRY(cudaStreamSynchronize(s));
  }
  return BMINRES_OK;
}

// One persistent solve on F (vectors of type V), updating Xout (row-major n x p of type V).
// Dependence threshold for a vector precision: FP32 Gram-Schmidt leaves ~1e-7 of an exactly
// dependent vector, so an FP32 inner solve cannot resolve gamma below ~1e-5.
template <typename V>
double effective_gamma(double gamma) {
  return std::is_same<V, float>::value ? std::max(gamma, 1e-5) : gamma;
}

template <typename V> const V* vals_of(bminres_handle h);
template <> const double* vals_of<double>(bminres_handle h) { return h->vals; }
template <> const float* vals_of<float>(bminres_handle h) { return h->vals32; }
template <> const bmr::dw* vals_of<bmr::dw>(bminres_handle h) { return h->vals_dw; }

template <typename V>
bminres_status persistent_solve(bminres_handle h, int p, V* Xout, double tol, int maxit, cudaStream_t s,
                                const V* vals, Ctl* result, double* kernel_ms) {
  bmr::Workspace& w = h->ws;
  const int64_t ld = padded_ld(h->n);
  const size_t es = sizeof(V);
  const int nb = std::max(h->opts.bench, 1);
  BMR_TRY(cudaMemsetAsync(w.U, 0, 2 * p * ld * es, s));
  BMR_TRY(cudaMemsetAsync(w.M, 0, 2 * p * ld * es, s));
  BMR_TRY(cudaMemsetAsync(w.Ghost, 0, nb * ld * es, s));
  BMR_TRY(cudaMemsetAsync(h->ctl, 0, sizeof(Ctl), s));
  bmr::SolveArgs<V> a;
  memset(&a, 0, sizeof(a));
  a.n = h->n;
  a.ld = ld;
  a.p = p;
  a.nbench = h->opts.bench;
  a.ghost = h->opts.ghost;
  a.maxit = maxit;
  a.tol = tol;
  a.gamma = effective_gamma<V>(h->opts.gamma);
  a.seed = h->opts.seed;
  a.rowptr = h->rowptr;
  a.colidx = h->colidx;
  a.vals = vals;
  a.F = (const V*)w.F;
  a.X = Xout;
  a.U = (V*)w.U;
  a.W = (V*)w.W;
  a.M = (V*)w.M;
  a.Bench = (V*)w.Bench;
  a.Ghost = (V*)w.Ghost;
  a.part = w.part;
  a.ctl = h->ctl;
  a.rho_hist = h->hist;
  a.hist_cap = h->hist_cap;
  a.barrier_limit_ns = BARRIER_LIMIT_NS;
  // Fault injection for tests of the bounded waits (no GPU fault involved): with
  // BMINRES_DEBUG_BARRIER_TIMEOUT_MS set, every grid barrier waits for one block more than the
  // grid has and gives up after that many milliseconds, so the solve ends with BMINRES_ERR_TIMEOUT.
  if (const char* e = getenv("BMINRES_DEBUG_BARRIER_TIMEOUT_MS")) {
    const long ms = strtol(e, nullptr, 10);
    if (ms > 0) {
      a.barrier_limit_ns = (unsigned long long)ms * 1000000ull;
      a.barrier_extra = 1;
    }
  }
  BMR_TRY(cudaEventRecord(h->evk0, s));
  BMR_TRY(launch_solve<V>(pm_for(p), a, w.grid, s));
  BMR_TRY(cudaEventRecord(h->evk1, s));
  h->launches++;
  BMR_TRY(cudaMemcpyAsync(h->ctl_host, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
  BMR_TRY(cudaStreamSynchronize(s));
  float kms = 0.f;
  if (cudaEventElapsedTime(&kms, h->evk0, h->evk1) == cudaSuccess) *kernel_ms += kms;
  *result = *h->ctl_host;
  h->hist_count = std::min(result->iters, h->hist_cap);
  h->hist_p = p;
  return BMINRES_OK;
}

void add_timeline(bminres_info& inf, const Ctl& r) {
  inf.stream_ms += (r.t_stream + r.t_sp + r.t_dir) * 1e-6;
  inf.spmm_ms += r.t_sp * 1e-6;
  inf.dir_ms += r.t_dir * 1e-6;
  inf.reduce_ms += r.t_reduce * 1e-6;
  inf.scalar_ms += r.t_scalar * 1e-6;
  inf.timeline_ms += r.t_total * 1e-6;
  inf.qr_ms += r.t_qr * 1e-6;
}

bminres_status map_kernel_status(int st) {
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

// FP64 iterative refinement around inner block MINRES solves with vectors of type V (FP32 or
// double-word): R = B - A X in FP64 (stored as V), solve A D = R to opts.tol_inner, X += D, until
// the FP64 residual meets tol.  f0 receives the initial residual norms.
template <typename V>
bminres_status refine(bminres_handle h, int p, const double* B, double* X, double tol, int maxit, cudaStream_t s,
                      double* f0, bminres_info& inf) {
  bmr::Workspace& w = h->ws;
  V* D = (V*)w.D;
  BMR_TRY(cudaMemsetAsync(D, 0, sizeof(V) * h->n * p, s));
  bminres_status st = BMINRES_NOT_CONVERGED;
  int used = 0;
  for (int outer = 0; outer < h->opts.max_outer; ++outer) {
    bminres_status rs = residual<V>(h, p, B, X, (V*)w.F, s, true);
    if (rs != BMINRES_OK) return rs;
    if (outer == 0)
      for (int i = 0; i < p; ++i) f0[i] = h->norms_host[i];
    double worst = 0.0;
    for (int i = 0; i < p; ++i) worst = std::max(worst, f0[i] > 0 ? h->norms_host[i] / f0[i] : 0.0);
    inf.relres_true_max = worst;
    if (worst < tol) {
      st = BMINRES_OK;
      break;
    }
    if (used >= maxit) break;
    Ctl r;
    rs = persistent_solve<V>(h, p, D, h->opts.tol_inner, maxit - used, s, vals_of<V>(h), &r, &inf.kernel_ms);
    if (rs != BMINRES_OK) return rs;
    used += r.iters;
    inf.iters += r.iters;
    inf.cycles += r.cycles;
    inf.outer = outer + 1;
    inf.deflations += r.deflations;
    inf.setup_deflations += r.setup_deflations;
    inf.bench_used = std::max(inf.bench_used, r.bench_used);
    inf.relres_est_max = r.relres_est_max;
    add_timeline(inf, r);
    bminres_status ks = map_kernel_status(r.status);
    if (ks != BMINRES_OK && ks != BMINRES_NOT_CONVERGED) {
      st = ks;
      break;
    }
    const int64_t total = h->n * p;
    bmr::add_correction_kernel<V><<<std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 4096)), 256, 0, s>>>(
        total, X, D);
    BMR_TRY(cudaGetLastError());
    h->launches++;
    if (r.iters == 0) break;  // inner solve could not make progress
  }
  return st;
}

// The solve on device-resident B and X.
bminres_status solve_device(bminres_handle h, int p, const double* B, double* X, double tol, int maxit,
                            cudaStream_t s, double* relres_true, bminres_info* info) {
  bminres_info inf;
  memset(&inf, 0, sizeof(inf));
  h->launches = 0;
  const int prec = prec_of(h);
  if (prec == 2 && p > pmax_of<bmr::dw>()) return BMINRES_ERR_INVALID;
  bminres_status st = ensure_ws(h, p, prec);
  if (st != BMINRES_OK) return st;
  bmr::Workspace& w = h->ws;
  inf.grid_blocks = w.grid;
  double f0[PMAX];
  BMR_TRY(cudaEventRecord(h->ev0, s));
  if (prec == 0) {
    st = residual<double>(h, p, B, X, (double*)w.F, s, true);
    if (st != BMINRES_OK) return st;
    for (int i = 0; i < p; ++i) f0[i] = h->norms_host[i];
    Ctl r;
    st = persistent_solve<double>(h, p, X, tol, maxit, s, h->vals, &r, &inf.kernel_ms);
    if (st != BMINRES_OK) return st;
    inf.iters = r.iters;
    inf.cycles = r.cycles;
    inf.outer = 1;
    inf.deflations = r.deflations;
    inf.setup_deflations = r.setup_deflations;
    inf.bench_used = r.bench_used;
    inf.relres_est_max = r.relres_est_max;
    add_timeline(inf, r);
    st = map_kernel_status(r.status);
  } else if (prec == 1) {
    st = refine<float>(h, p, B, X, tol, maxit, s, f0, inf);
  } else if (prec == 2) {
    st = refine<bmr::dw>(h, p, B, X, tol, maxit, s, f0, inf);
  } else {
    st = refine<double>(h, p, B, X, tol, maxit, s, f0, inf);
  }
  // FP64 true residual of the result
  {
    bminres_status rs = prec == 1   ? residual<float>(h, p, B, X, (float*)w.F, s, true)
                        : prec == 2 ? residual<bmr::dw>(h, p, B, X, (bmr::dw*)w.F, s, true)
                                    : residual<double>(h, p, B, X, (double*)w.F, s, true);
    if (rs != BMINRES_OK) return rs;
    double worst = 0.0;
    for (int i = 0; i < p; ++i) {
      double rel = f0[i] > 0 ? h->norms_host[i] / f0[i] : 0.0;
      if (relres_true) relres_true[i] = rel;
      worst = std::max(worst, rel);
    }
    inf.relres_true_max = worst;
    // FP64 mode stops on the recursive residual (Eq. (comp-resid)); say so when the true one missed
    if (prec == 0 && st == BMINRES_OK && worst > tol) st = BMINRES_RESIDUAL_GAP;
  }
  BMR_TRY(cudaEventRecord(h->ev1, s));
  BMR_TRY(cudaEventSynchronize(h->ev1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, h->ev0, h->ev1);
  inf.device_ms = ms;
  inf.launches = h->launches;
  inf.status = st;
  if (info) *info = inf;
  return st;
}

}  // namespace

extern "C" {

void bminres_default_opts(bminres_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->precision = BMINRES_FP64;
  o->gamma = 1e-8;
  o->bench = 4;
  o->seed = 0;
  o->ghost = 0;
  o->tol_inner = 1e-5;
  o->max_outer = 20;
  o->max_blocks = 0;
}

const char* bminres_status_string(bminres_status s) {
  switch (s) {
    case BMINRES_OK: return "BMINRES_OK";
    case BMINRES_NOT_CONVERGED: return "BMINRES_NOT_CONVERGED";
    case BMINRES_RESIDUAL_GAP: return "BMINRES_RESIDUAL_GAP";
    case BMINRES_ERR_INVALID: return "BMINRES_ERR_INVALID";
    case BMINRES_ERR_CUDA: return "BMINRES_ERR_CUDA";
    case BMINRES_ERR_OOM: return "BMINRES_ERR_OOM";
    case BMINRES_ERR_BREAKDOWN: return "BMINRES_ERR_BREAKDOWN";
    case BMINRES_ERR_BENCH_EXHAUSTED: return "BMINRES_ERR_BENCH_EXHAUSTED";
    case BMINRES_ERR_NONFINITE: return "BMINRES_ERR_NONFINITE";
    case BMINRES_ERR_TIMEOUT: return "BMINRES_ERR_TIMEOUT";
  }
  return "BMINRES_UNKNOWN_STATUS";
}

bminres_status bminres_create(bminres_handle* out, int64_t n, int64_t nnz, const int32_t* rowptr,
                              const int32_t* colidx, const double* vals, const bminres_opts* opts) {
  if (!out) return BMINRES_ERR_INVALID;
  *out = nullptr;
  if (n < 0 || nnz < 0 || nnz >= ((int64_t)1 << 31) || n >= ((int64_t)1 << 31)) return BMINRES_ERR_INVALID;
  if (!rowptr || (nnz > 0 && (!colidx || !vals))) return BMINRES_ERR_INVALID;
  if (foreign({rowptr, colidx, vals})) return BMINRES_ERR_INVALID;
  bminres_opts o;
  bminres_default_opts(&o);
  if (opts) o = *opts;
  if (o.bench < 0 || o.bench > bmr::NBMAX || !(o.gamma >= 0.0) || (o.precision < BMINRES_FP64 || o.precision > BMINRES_FP64_REFINED))
    return BMINRES_ERR_INVALID;
  if (o.max_outer <= 0) o.max_outer = 20;
  if (!(o.tol_inner > 0.0)) o.tol_inner = 1e-5;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return BMINRES_ERR_CUDA;
  }
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return BMINRES_ERR_CUDA;
  if (prop.major != 10 || prop.minor != 3 || !prop.cooperativeLaunch) return BMINRES_ERR_CUDA;
  // validate the CSR structure on the host
  std::vector<int32_t> rp(n + 1);
  std::vector<int32_t> ci(nnz);
  if (is_device_ptr(rowptr)) {
    if (cudaMemcpy(rp.data(), rowptr, sizeof(int32_t) * (n + 1), cudaMemcpyDeviceToHost) != cudaSuccess) return BMINRES_ERR_CUDA;
  } else {
    memcpy(rp.data(), rowptr, sizeof(int32_t) * (n + 1));
  }
  if (nnz > 0) {
    if (is_device_ptr(colidx)) {
      if (cudaMemcpy(ci.data(), colidx, sizeof(int32_t) * nnz, cudaMemcpyDeviceToHost) != cudaSuccess) return BMINRES_ERR_CUDA;
    } else {
      memcpy(ci.data(), colidx, sizeof(int32_t) * nnz);
    }
  }
  if (rp[0] != 0 || rp[n] != nnz) return BMINRES_ERR_INVALID;
  for (int64_t r = 0; r < n; ++r)
    if (rp[r + 1] < rp[r]) return BMINRES_ERR_INVALID;
  for (int64_t k = 0; k < nnz; ++k)
    if (ci[k] < 0 || ci[k] >= n) return BMINRES_ERR_INVALID;

  bminres_handle h = new (std::nothrow) bminres_handle_s();
  if (!h) return BMINRES_ERR_OOM;
  h->device = dev;
  h->num_sms = prop.multiProcessorCount;
  h->n = n;
  h->nnz = nnz;
  h->opts = o;
  auto fail = [&](bminres_status s) {
    bminres_destroy(h);
    return s;
  };
  if (cudaMalloc(&h->rowptr, sizeof(int32_t) * (n + 1)) != cudaSuccess) return fail(BMINRES_ERR_OOM);
  if (cudaMalloc(&h->colidx, sizeof(int32_t) * std::max<int64_t>(nnz, 1)) != cudaSuccess) return fail(BMINRES_ERR_OOM);
  if (cudaMalloc(&h->vals, sizeof(double) * std::max<int64_t>(nnz, 1)) != cudaSuccess) return fail(BMINRES_ERR_OOM);
  if (o.precision == BMINRES_MIXED &&
      cudaMalloc(&h->vals32, sizeof(float) * std::max<int64_t>(nnz, 1)) != cudaSuccess)
    return fail(BMINRES_ERR_OOM);
  if (o.precision == BMINRES_MIXED_DW &&
      cudaMalloc(&h->vals_dw, sizeof(bmr::dw) * std::max<int64_t>(nnz, 1)) != cudaSuccess)
    return fail(BMINRES_ERR_OOM);
  if (cudaMalloc(&h->ctl, sizeof(Ctl)) != cudaSuccess) return fail(BMINRES_ERR_OOM);
  if (cudaMallocHost(&h->ctl_host, sizeof(Ctl)) != cudaSuccess) return fail(BMINRES_ERR_OOM);
  if (cudaMallocHost(&h->norms_host, sizeof(double) * 64) != cudaSuccess) return fail(BMINRES_ERR_OOM);
  if (cudaEventCreate(&h->ev0) != cudaSuccess || cudaEventCreate(&h->ev1) != cudaSuccess ||
      cudaEventCreate(&h->evk0) != cudaSuccess || cudaEventCreate(&h->evk1) != cudaSuccess)
    return fail(BMINRES_ERR_CUDA);
  if (cudaMemcpy(h->rowptr, rp.data(), sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(BMINRES_ERR_CUDA);
  if (nnz > 0 && cudaMemcpy(h->colidx, ci.data(), sizeof(int32_t) * nnz, cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(BMINRES_ERR_CUDA);
  *out = h;
  bminres_status s = bminres_set_values(h, vals, nullptr);
  if (s != BMINRES_OK) {
    *out = nullptr;
    return fail(s);
  }
  if (cudaDeviceSynchronize() != cudaSuccess) {
    *out = nullptr;
    return fail(BMINRES_ERR_CUDA);
  }
  return BMINRES_OK;
}

bminres_status bminres_set_values(bminres_handle h, const double* vals, bminres_stream stream) {
  if (!h) return BMINRES_ERR_INVALID;
  if (h->nnz == 0) return BMINRES_OK;
  if (!vals || foreign({vals})) return BMINRES_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  BMR_TRY(cudaMemcpyAsync(h->vals, vals, sizeof(double) * h->nnz, cudaMemcpyDefault, s));
  const int cb = (int)std::min<int64_t>((h->nnz + 255) / 256, 4096);
  if (h->vals32) {
    bmr::to_vec_kernel<float><<<cb, 256, 0, s>>>(h->nnz, h->vals, h->vals32);
    BMR_TRY(cudaGetLastError());
  }
  if (h->vals_dw) {
    bmr::to_vec_kernel<bmr::dw><<<cb, 256, 0, s>>>(h->nnz, h->vals, h->vals_dw);
    BMR_TRY(cudaGetLastError());
  }
  BMR_TRY(cudaStreamSynchronize(s));
  return BMINRES_OK;
}

void bminres_destroy(bminres_handle h) {
  if (!h) return;
  free_ws(h->ws);
  if (h->rowptr) cudaFree(h->rowptr);
  if (h->colidx) cudaFree(h->colidx);
  if (h->vals) cudaFree(h->vals);
  if (h->vals32) cudaFree(h->vals32);
  if (h->vals_dw) cudaFree(h->vals_dw);
  if (h->ctl) cudaFree(h->ctl);
  if (h->ctl_host) cudaFreeHost(h->ctl_host);
  if (h->norms_host) cudaFreeHost(h->norms_host);
  if (h->ev0) cudaEventDestroy(h->ev0);
  if (h->ev1) cudaEventDestroy(h->ev1);
  if (h->evk0) cudaEventDestroy(h->evk0);
  if (h->evk1) cudaEventDestroy(h->evk1);
  if (h->hist) cudaFree(h->hist);
  delete h;
}

bminres_status bminres_solve(bminres_handle h, int p, const double* B, double* X, double tol, int maxit,
                             bminres_stream stream, double* relres_true, bminres_info* info) {
  if (info) memset(info, 0, sizeof(*info));
  if (!h) return BMINRES_ERR_INVALID;
  if (h->n == 0 || p == 0) return BMINRES_OK;
  if (p < 0 || p > PMAX || p > h->n || !B || !X || !(tol > 0.0) || maxit < 0) return BMINRES_ERR_INVALID;
  if (foreign({B, X})) return BMINRES_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  const bool dB = is_device_ptr(B), dX = is_device_ptr(X);
  if (dB && dX) return solve_device(h, p, B, X, tol, maxit, s, relres_true, info);
  // host buffers: stage through handle-owned device memory (copies are part of the call)
  bminres_status st = ensure_ws(h, p, prec_of(h));
  if (st != BMINRES_OK) return st;
  const size_t bytes = sizeof(double) * h->n * p;
  double* Bd = dB ? (double*)B : h->ws.Btmp;
  double* Xd = dX ? X : h->ws.Xtmp;
  if (!dB) BMR_TRY(cudaMemcpyAsync(Bd, B, bytes, cudaMemcpyHostToDevice, s));
  if (!dX) BMR_TRY(cudaMemcpyAsync(Xd, X, bytes, cudaMemcpyHostToDevice, s));
  st = solve_device(h, p, Bd, Xd, tol, maxit, s, relres_true, info);
  if (st != BMINRES_OK && st != BMINRES_NOT_CONVERGED && st != BMINRES_RESIDUAL_GAP) return st;
  if (!dX) {
    BMR_TRY(cudaMemcpyAsync(X, Xd, bytes, cudaMemcpyDeviceToHost, s));
    BMR_TRY(cudaStreamSynchronize(s));
  }
  return st;
}

bminres_status bminres_set_history(bminres_handle h, int cap) {
  if (!h || cap < 0) return BMINRES_ERR_INVALID;
  if (h->hist) cudaFree(h->hist);
  h->hist = nullptr;
  h->hist_cap = 0;
  h->hist_count = 0;
  if (cap == 0) return BMINRES_OK;
  if (cudaMalloc(&h->hist, sizeof(double) * (size_t)cap * PMAX) != cudaSuccess) {
    cudaGetLastError();
    return BMINRES_ERR_OOM;
  }
  h->hist_cap = cap;
  return BMINRES_OK;
}

bminres_status bminres_get_history(bminres_handle h, double* out, int* count) {
  if (!h || !count) return BMINRES_ERR_INVALID;
  *count = h->hist_count;
  if (h->hist_count == 0) return BMINRES_OK;
  if (!out) return BMINRES_ERR_INVALID;
  BMR_TRY(cudaMemcpy(out, h->hist, sizeof(double) * (size_t)h->hist_count * h->hist_p, cudaMemcpyDefault));
  return BMINRES_OK;
}

bminres_status bminres_spmm(bminres_handle h, int p, const double* X, double* Y, bminres_stream stream) {
  if (!h) return BMINRES_ERR_INVALID;
  if (h->n == 0 || p == 0) return BMINRES_OK;
  if (p < 0 || p > PMAX || !X || !Y) return BMINRES_ERR_INVALID;
  if (foreign({X, Y})) return BMINRES_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  const bool dx = is_device_ptr(X), dy = is_device_ptr(Y);
  const size_t bytes = sizeof(double) * h->n * p;
  double *Xd = (double*)X, *Yd = Y, *tmp = nullptr;
  if (!dx || !dy) {
    BMR_TRY(cudaMalloc(&tmp, 2 * bytes));
    if (!dx) {
      Xd = tmp;
      cudaMemcpyAsync(Xd, X, bytes, cudaMemcpyHostToDevice, s);
    }
    if (!dy) Yd = tmp + h->n * p;
  }
  bmr::spmm_kernel<<<(int)((h->n + bmr::AUX_NT - 1) / bmr::AUX_NT), bmr::AUX_NT, 0, s>>>(h->n, p, h->rowptr, h->colidx,
                                                                                           h->vals, Xd, Yd);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && !dy) e = cudaMemcpyAsync(Y, Yd, bytes, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (tmp) cudaFree(tmp);
  return from_cuda(e);
}

bminres_status bminres_backward(bminres_handle h, int p, const double* G, const double* X, double* dB,
                                double* dA_vals, double tol, int maxit, bminres_stream stream, bminres_info* info) {
  if (info) memset(info, 0, sizeof(*info));
  if (!h) return BMINRES_ERR_INVALID;
  if (h->n == 0 || p == 0) return BMINRES_OK;
  if (p < 0 || p > PMAX || !G || !dB || (dA_vals && !X) || !(tol > 0.0) || maxit < 0) return BMINRES_ERR_INVALID;
  if (foreign({G, X, dB, dA_vals})) return BMINRES_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = sizeof(double) * h->n * p;
  // dB = A^{-1} G by a block solve from zero (A symmetric, so A^{-T} = A^{-1})
  const bool dG = is_device_ptr(G), ddB = is_device_ptr(dB), dXp = X ? is_device_ptr(X) : true;
  const bool dA = dA_vals ? is_device_ptr(dA_vals) : true;
  double *tmp = nullptr, *Gd = (double*)G, *dBd = dB, *Xd = (double*)X, *dAd = dA_vals;
  size_t need = (dG ? 0 : bytes) + (ddB ? 0 : bytes) + (dXp ? 0 : bytes) + (dA ? 0 : sizeof(double) * h->nnz);
  if (need) BMR_TRY(cudaMalloc(&tmp, need));
  char* cur = (char*)tmp;
  if (!dG) { Gd = (double*)cur; cur += bytes; cudaMemcpyAsync(Gd, G, bytes, cudaMemcpyHostToDevice, s); }
  if (!ddB) { dBd = (double*)cur; cur += bytes; }
  if (!dXp) { Xd = (double*)cur; cur += bytes; cudaMemcpyAsync(Xd, X, bytes, cudaMemcpyHostToDevice, s); }
  if (!dA) { dAd = (double*)cur; }
  bminres_status st = BMINRES_OK;
  cudaError_t e = cudaMemsetAsync(dBd, 0, bytes, s);
  if (e != cudaSuccess) st = from_cuda(e);
  if (st == BMINRES_OK) st = solve_device(h, p, Gd, dBd, tol, maxit, s, nullptr, info);
  if (st == BMINRES_OK || st == BMINRES_NOT_CONVERGED || st == BMINRES_RESIDUAL_GAP) {
    bminres_status keep = st;
    if (dA_vals) {
      bmr::sddmm_kernel<<<(int)((h->n + bmr::AUX_NT - 1) / bmr::AUX_NT), bmr::AUX_NT, 0, s>>>(h->n, p, h->rowptr,
                                                                                                h->colidx, dBd, Xd, dAd);
      e = cudaGetLastError();
      if (e == cudaSuccess && !dA) e = cudaMemcpyAsync(dA_vals, dAd, sizeof(double) * h->nnz, cudaMemcpyDeviceToHost, s);
    }
    if (e == cudaSuccess && !ddB) e = cudaMemcpyAsync(dB, dBd, bytes, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    st = (e == cudaSuccess) ? keep : from_cuda(e);
  }
  if (tmp) {
    cudaStreamSynchronize(s);
    cudaFree(tmp);
  }
  return st;
}

}  // extern "C"
