/*
 * bminres.h -- C ABI of the GB300 (sm_103a) block MINRES library.
 *
 * The library solves A X = B for a sparse symmetric (indefinite) A and a block of p right-hand
 * sides with the band-Lanczos block MINRES method (K. M. Soodhalter, "A block MINRES algorithm
 * based on the band Lanczos method", Algorithm 2).  At band iteration j, column i of X_j
 * minimises ||b_i - A x|| over x in x0_i + span(U_j), where U_j holds the first j band-Lanczos
 * vectors generated from the orthonormalised initial block residual (Sec. 3, Eq. (min-resid)).
 *
 * Conventions for every entry point:
 *  - Dense blocks (B, X, G, dB) are row-major n x p arrays of double: entry (r, c) at [r*p + c].
 *  - A pointer argument may be host or device memory; host data is staged through buffers the
 *    handle owns.  Device memory must belong to the current device (memory of another GPU is
 *    rejected with BMINRES_ERR_INVALID).  The caller keeps ownership of every pointer it passes.
 *  - Work is enqueued on `stream` (a cudaStream_t; NULL = the legacy default stream).  Entry
 *    points that fill an info struct or return a solve status synchronise that stream first.
 *  - Errors are returned as bminres_status codes; no exception crosses the ABI.  After any
 *    status other than BMINRES_OK / BMINRES_NOT_CONVERGED the contents of output arrays are
 *    unspecified, but the handle stays usable unless the status is BMINRES_ERR_CUDA.
 *  - A handle is not thread safe: calls on one handle must not overlap.
 */
#ifndef BMINRES_H
#define BMINRES_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bminres_handle_s* bminres_handle;
typedef void* bminres_stream; /* cudaStream_t */

typedef enum {
  BMINRES_OK = 0,                  /* converged: every column met the stopping test */
  BMINRES_NOT_CONVERGED = 1,       /* maxit reached; X holds the last iterate */
  BMINRES_RESIDUAL_GAP = 2,        /* FP64 mode: the recursive residual met tol (the paper's stopping
                                      test) but the FP64 true residual recomputed after the solve did
                                      not (finite-precision residual gap, or a dropped dependent
                                      direction); X holds the final iterate.  The refined forms
                                      restart on this condition instead of returning it */
  BMINRES_ERR_INVALID = -1,        /* bad argument (sizes, CSR structure, null pointer) */
  BMINRES_ERR_CUDA = -2,           /* a CUDA runtime call failed, or no usable sm_103 device */
  BMINRES_ERR_OOM = -3,            /* device allocation failed */
  BMINRES_ERR_BREAKDOWN = -4,      /* r_jj = 0 in the band QR (singular R_j) */
  BMINRES_ERR_BENCH_EXHAUSTED = -5,/* a dependence was met with no bench vector left (Sec. 5.1) */
  BMINRES_ERR_NONFINITE = -6,      /* NaN or Inf in a norm or coefficient */
  BMINRES_ERR_TIMEOUT = -7         /* a device-side wait hit its time limit; results invalid */
} bminres_status;

typedef enum { BMINRES_FP64 = 0, BMINRES_MIXED = 1, BMINRES_MIXED_DW = 2, BMINRES_FP64_REFINED = 3 } bminres_precision;

typedef struct {
  int precision;     /* BMINRES_FP64 (default); BMINRES_MIXED: FP32 Lanczos vectors, block
                        product and orthogonalisation inside an FP64 iterative-refinement loop;
                        the residual B - A X, coefficients, band QR and dependence test in FP64;
                        BMINRES_MIXED_DW: the same loop with double-word vectors (pairs of FP32
                        values, about 48 significant bits, arithmetic on the FP32 units), p <= 16
                        (larger p: BMINRES_ERR_INVALID); BMINRES_FP64_REFINED: the same loop with
                        FP64 inner solves (restarts until the FP64 true residual meets tol).
                        None of the refined forms is in the paper */
  double gamma;      /* dependence tolerance, relative: a new vector is dependent when its norm
                        after orthogonalisation is <= gamma * ||A u_j|| (Sec. 5).  Default 1e-8;
                        FP32 inner solves (MIXED) use max(gamma, 1e-5) */
  int bench;         /* size of the dynamic substitutes bench (Sec. 5.1), 0..8.  Default 4 */
  uint64_t seed;     /* seed of the counter-based SplitMix64 stream for bench vectors */
  int ghost;         /* 1: keep a removed vector and orthogonalise against it for the next 2p
                        iterations (end of Sec. 5.1).  Its coefficients are not part of H, so the
                        recursive residual can then drift from the true one.  Default 0 */
  double tol_inner;  /* refined forms: relative tolerance of each inner solve.  Default 1e-5 */
  int max_outer;     /* refined forms: maximum refinement steps.  Default 20 */
  int max_blocks;    /* upper bound on the persistent kernel's grid (0 = one wave of the GPU) */
} bminres_opts;

typedef struct {
  int status;            /* same as the return value */
  int iters;             /* band iterations (summed over the inner solves of the refined forms) */
  int cycles;            /* block products A [u_j .. u_{j+p-1}] */
  int outer;             /* refinement steps (MIXED, MIXED_DW, FP64_REFINED); 1 in FP64 mode */
  int deflations;        /* dependent vectors replaced during the iteration */
  int setup_deflations;  /* dependent columns of the initial block residual */
  int bench_used;        /* bench vectors consumed */
  int grid_blocks;       /* blocks of the persistent solve kernel */
  double relres_est_max; /* max_i of the recursive residual ||Shat(j+1:j+p, i)|| / ||f0_i||
                            (Eq. (comp-resid)); for the refined forms, of the last inner solve */
  double relres_true_max;/* max_i ||b_i - A x_i|| / ||b_i - A x0_i||, recomputed in FP64 */
  double device_ms;      /* device time from the first to the last kernel of the solve */
  double kernel_ms;      /* CUDA-event time of the persistent solve kernel launches (summed) */
  double stream_ms;      /* timeline of the persistent kernel's block 0 (global timer, summed over
                            launches): streaming passes over the vectors, */
  double reduce_ms;      /* grid reductions including barriers, */
  double scalar_ms;      /* coefficient bookkeeping between passes, */
  double timeline_ms;    /* the whole kernel, */
  double qr_ms;          /* and the band QR steps of the control warp (overlapped with streaming) */
  int launches;          /* kernels launched by this call */
  double spmm_ms;        /* part of stream_ms: block-product passes (SpMM fused with an A step) */
  double dir_ms;         /* part of stream_ms: direction and iterate passes */
} bminres_info;

/* Fill *opts with the defaults listed above. */
void bminres_default_opts(bminres_opts* opts);

/* Create a solver handle for the n x n CSR matrix (rowptr[n+1], colidx[nnz], vals[nnz]; int32
 * indices, the full symmetric pattern, any column order within a row).  The arrays are copied
 * into handle-owned device memory (host or device pointers accepted); opts may be NULL.
 * Checks: n >= 0, 0 <= nnz < 2^31, rowptr monotone with rowptr[0] = 0, rowptr[n] = nnz,
 * 0 <= colidx < n.  Symmetry is the caller's responsibility (it is not checked).
 * Returns BMINRES_ERR_CUDA when no sm_103 device is present. */
bminres_status bminres_create(bminres_handle* handle, int64_t n, int64_t nnz, const int32_t* rowptr,
                              const int32_t* colidx, const double* vals, const bminres_opts* opts);

/* Replace the nnz values of A (same order as at create time; same pattern). */
bminres_status bminres_set_values(bminres_handle handle, const double* vals, bminres_stream stream);

/* Solve A X = B by block MINRES (Algorithm 2).  B: n x p, X: n x p (in: X0, out: X).
 * Stops after the first band iteration j with max_i rho_i / ||f0_i|| < tol, where rho_i is the
 * recursive residual of column i (Eq. (comp-resid)) and f0 = B - A X0 (FP64 mode), or when the
 * FP64 true relative residual of every column is < tol (refined forms), or after maxit band
 * iterations (status NOT_CONVERGED, X = last iterate).  In FP64 mode the status is
 * BMINRES_RESIDUAL_GAP instead of BMINRES_OK when the FP64 true residual of some column is above
 * tol although the recursive one met it.  relres_true (host, length p, may be NULL)
 * receives ||b_i - A x_i|| / ||b_i - A x0_i|| computed in FP64 after the solve.  info may be
 * NULL.  p must satisfy 1 <= p <= 32 (<= 16 for MIXED_DW) and p <= n; n = 0 or p = 0 returns
 * BMINRES_OK at once. */
bminres_status bminres_solve(bminres_handle handle, int p, const double* B, double* X, double tol,
                             int maxit, bminres_stream stream, double* relres_true, bminres_info* info);

/* Adjoint of the solve (not in the paper): given G = dL/dX for X = A^{-1} B, compute
 * dB = A^{-1} G (a second block solve from zero, A being symmetric) and
 * dA_vals[k] = -sum_c dB[row_k, c] * X[colidx_k, c] for every stored entry k (same order as the
 * CSR given at create time), i.e. -(dB X^T) restricted to the sparsity pattern.  G, X, dB: n x p;
 * dA_vals: nnz (may be NULL to skip).  tol / maxit apply to the adjoint solve. */
bminres_status bminres_backward(bminres_handle handle, int p, const double* G, const double* X,
                                double* dB, double* dA_vals, double tol, int maxit,
                                bminres_stream stream, bminres_info* info);

/* Record the recursive residual norms ||Shat(j+1:j+p, i)|| (Eq. (comp-resid)) of band iterations
 * j = 1 .. cap of the following solves (cap = 0 switches recording off).  For the refined forms
 * the record is that of the last inner solve. */
bminres_status bminres_set_history(bminres_handle handle, int cap);

/* Copy the record of the last solve to host memory: out[(j-1)*p + i] for j = 1 .. *count
 * (count = min(iterations, cap)); out must hold cap * p doubles. */
bminres_status bminres_get_history(bminres_handle handle, double* out, int* count);

/* Y = A X for an n x p block (FP64, CSR summation order).  1 <= p <= 32. */
bminres_status bminres_spmm(bminres_handle handle, int p, const double* X, double* Y, bminres_stream stream);

/* Size of the static device scratch array used by bminres_solve_noalloc (64 MiB).  Every GPU on
 * which the library is loaded holds this array until the process exits. */
#define BMINRES_NOALLOC_SCRATCH_BYTES (64ull << 20)

/* FP64 solve of A X = B that allocates nothing (the paper has no counterpart; this is a service
 * entry point of the library).  It is meant for callers that must not call cudaMalloc: code whose
 * device memory is owned by another framework's pool (a raw cudaMalloc there fragments the pool or
 * exceeds its budget), and latency-critical loops that cannot accept the implicit device-wide
 * synchronisation of cudaMalloc / cudaFree.  The result is the same as bminres_create +
 * bminres_solve in FP64 mode with the default options (or *opts, whose precision must be FP64).
 *  - rowptr, colidx, vals (CSR of A, int32 indices, full symmetric pattern), B and X (row-major
 *    n x p; X in: X0, out: X) must be device pointers of the current device; the caller owns them.  The CSR is not
 *    validated beyond n >= 0 and 0 <= nnz < 2^31.
 *  - All workspace lives in one static device array of BMINRES_NOALLOC_SCRATCH_BYTES; the call
 *    fits when (6 p + 2 bench) * 8 * round_up(n, 64) bytes plus ~1 MiB do not exceed it (about
 *    n <= 140,000 at p = 8 with 4 bench vectors); larger problems are rejected with
 *    BMINRES_ERR_INVALID before any device work.
 *  - The first call on a device looks up the array's device address (cudaGetSymbolAddress) with
 *    that device current; make that first call before any stream capture.
 *  - Every call shares the array and it keeps the last call's contents: calls that overlap on the
 *    GPU (other streams, other host threads) race and must not be issued.
 *  - relres_true (host, p doubles) and info may be NULL; info->device_ms is 0 (no event is
 *    created); info->timeline_ms carries the kernel's own device timer.  The status follows
 *    bminres_solve in FP64 mode (BMINRES_RESIDUAL_GAP included). */
bminres_status bminres_solve_noalloc(int64_t n, int64_t nnz, const int32_t* rowptr, const int32_t* colidx,
                                     const double* vals, int p, const double* B, double* X, double tol,
                                     int maxit, const bminres_opts* opts, bminres_stream stream,
                                     double* relres_true, bminres_info* info);

/* Measurement helper, not a step of the method (the paper has no counterpart): FP64 fused
 * multiply-add throughput of the current GPU, in GFLOP/s (2 flops per FMA): the fastest of three
 * timed launches of independent FMA chains (8 or 16 chains per thread, 4 or 8 blocks of 256 threads
 * per SM, about 8 * `iters` FMAs per thread), each after a warm-up launch, on `stream`.  It is the
 * denominator of the arithmetic roofline against which the FP64 solve is reported.  ms (may be NULL)
 * receives the fastest timed launch's duration.  Allocates 8 bytes of device memory for the
 * duration of the call. */
bminres_status bminres_fp64_peak(int iters, bminres_stream stream, double* gflops, double* ms);

/* Release the handle and everything it owns.  NULL is ignored. */
void bminres_destroy(bminres_handle handle);

/* Static, human-readable name of a status code. */
const char* bminres_status_string(bminres_status status);

#ifdef __cplusplus
}
#endif

#endif /* BMINRES_H */
