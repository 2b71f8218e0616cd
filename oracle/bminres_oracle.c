/*
 * Block MINRES (band Lanczos version) -- plain FP64 CPU ORACLE.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is used by the tests, by the smoke check and by the
 * benchmark's CPU-baseline leg.  The library's solve path never calls it, and it shares no
 * code, headers or constants with the CUDA implementation.
 *
 * What it computes (Soodhalter, "A block MINRES algorithm based on the band Lanczos method"):
 * at band iteration j, column i of X_j minimises ||b_i - A x|| over x in x0_i + R(U_j), where
 * U_j holds the first j band-Lanczos vectors started from the orthonormalised initial block
 * residual (Sec. 3, Eq. (min-resid), Eq. (minres-approx)).  The steps follow Algorithm 2
 * ("Block MINRES (band Lanczos version)") in the paper's order, with these readings of the
 * printed algorithm (each is also listed in the design notes):
 *   R1  "QR-Factorization B V_p S" is F0 = U_p S with F0 = B - A X0 (Eq. (init-QR)); the
 *       right-hand-side block is Shat = [S; 0] (Eq. (E1.block)).
 *   R2  The loop runs while max_i ||Shat(j+1:j+p, i)|| / ||f0_i|| >= eps and j <= M
 *       (Eq. (comp-resid)); the printed condition is inverted.
 *   R3  The block product fires when (j-1) mod p == 0, on u_j .. u_{j+p-1}.
 *   R4  "w <- h w" and "w <- h v_i" mean w <- w - h_{i,j} u_i; the new vector is u_{j+p};
 *       loop bounds printed with min{1, .} mean max{1, .}.
 *   R5  The new reflector is also applied to rows j..j+p of Shat (Sec. 4), which the printed
 *       algorithm leaves out.
 *   R6  "If m = 1" means "if j = 1".
 *   R7  Dependence test (Sec. 5): h_{j+p,j} <= gamma * ||A u_j||, relative to the norm of the
 *       block-product column.  At set-up a column is dependent when its orthogonalised norm is
 *       <= gamma * ||f0_i||; it is replaced the same way and gets S_ii = 0.
 *   R8  Dynamic substitutes bench (Sec. 5.1): `bench` vectors drawn before the iteration from a
 *       counter-based SplitMix64 stream and orthogonalised against every Lanczos vector as it
 *       is created.  On a dependence a bench vector gets one more modified Gram-Schmidt pass
 *       against u_{j-p+1} .. u_{j+p-1} and the active removed vectors, is normalised and
 *       becomes u_{j+p}; h_{j+p,j} is set to 0 (so h_{j,j+p} = 0 by symmetry).
 *   R9  A removed vector is kept and new Lanczos vectors are orthogonalised against it for the
 *       next 2p iterations, after which it would have left the band (end of Sec. 5.1); its
 *       coefficients are not entered in H.  The kept vector is w after one more MGS pass against
 *       u_{j-p+1}..u_{j+p-1} and the removed vectors still active, normalised (dropped if
 *       nothing is left).  It is kept only when ||w|| > 1e-12 ||A u_j||: for a dependence that is
 *       exact to rounding, w is noise and carries no direction.
 *   R10 Lanczos orthogonalisation uses modified Gram-Schmidt in the order of Algorithm 1:
 *       known (symmetric) coefficients first, then the p new inner products.
 * The band QR uses Householder reflectors (Sec. 4) by default; qr_mode = 1 selects Givens
 * rotations instead (used only to check that X does not depend on the choice).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Build variants of this one source (the arithmetic of the default build is plain FP64):
 *   ORACLE_ACC   accumulator type of inner products, norms and the CSR matvec sums (default
 *                double).  `long double` gives a second reference whose only difference is the
 *                rounding of those sums; the tests use it to measure how much the iteration count
 *                at which the tolerance is met depends on summation rounding.
 *   ORACLE_FMA   vector updates y + a x rounded once (C99 fma) instead of twice; with ORACLE_ACC =
 *                long double this is the most accurately rounded build of the same steps.
 *   ORACLE_OMP   (with -fopenmp) the vector loops and the matvec run on all host cores, the inner
 *                products as fixed chunks summed in chunk order, so the result does not depend on
 *                the thread count.  Used only to time the oracle on the host cores. */
#ifndef ORACLE_ACC
#define ORACLE_ACC double
#endif
typedef ORACLE_ACC acc_t;
#if defined(ORACLE_OMP) && defined(_OPENMP)
#define OMP_FOR _Pragma("omp parallel for schedule(static)")
#define DOT_CHUNKS 256
#else
#define OMP_FOR
#endif

#define OR_OK 0
#define OR_NOT_CONVERGED 1
#define OR_ERR_INVALID -1
#define OR_ERR_OOM -3
#define OR_ERR_BREAKDOWN -4
#define OR_ERR_BENCH_EXHAUSTED -5
#define OR_ERR_NONFINITE -6

/* reading R9: a removed vector is kept only for a near-dependence; at ||w|| <= 1e-12 ||A u_j|| the
 * dependence is exact to rounding and w carries no direction */
#define GHOST_FLOOR 1e-12

typedef struct {
  int status;            /* OR_* code */
  int iters;             /* band iterations performed (the final j) */
  int deflations;        /* dependences met during the iteration */
  int setup_deflations;  /* dependent columns in the initial QR */
  int bench_used;        /* bench vectors consumed */
} oracle_info;

/* ---------------------------------------------------------------------------------------- */
/* SplitMix64 (Steele, Lea, Flood, OOPSLA 2014), used as a counter-based generator: the value
 * with index t of the stream seeded with s is mix(s + (t + 1) * 0x9E3779B97F4A7C15).          */
static uint64_t splitmix64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* Entry `row` of bench vector k: uniform in [-1, 1) with 53 random bits. */
double oracle_bench_value(uint64_t seed, int64_t k, int64_t n, int64_t row) {
  uint64_t t = (uint64_t)k * (uint64_t)n + (uint64_t)row;
  uint64_t z = splitmix64_mix(seed + (t + 1ULL) * 0x9E3779B97F4A7C15ULL);
  return (double)(z >> 11) * (1.0 / 4503599627370496.0) - 1.0; /* (z>>11) * 2^-52 - 1 */
}

/* ---------------------------------------------------------------------------------------- */
static double dot(int64_t n, const double* x, const double* y) {
#ifdef DOT_CHUNKS
  double part[DOT_CHUNKS];
  OMP_FOR
  for (int c = 0; c < DOT_CHUNKS; ++c) {
    acc_t s = 0.0;
    for (int64_t r = n * c / DOT_CHUNKS; r < n * (c + 1) / DOT_CHUNKS; ++r) s += (acc_t)x[r] * y[r];
    part[c] = (double)s;
  }
  double s = 0.0;
  for (int c = 0; c < DOT_CHUNKS; ++c) s += part[c];
  return s;
#else
  acc_t s = 0.0;
  for (int64_t r = 0; r < n; ++r) s += (acc_t)x[r] * y[r];
  return (double)s;
#endif
}
static void axpy(int64_t n, double a, const double* x, double* y) {
  OMP_FOR
#ifdef ORACLE_FMA
  for (int64_t r = 0; r < n; ++r) y[r] = fma(a, x[r], y[r]);
#else
  for (int64_t r = 0; r < n; ++r) y[r] += a * x[r];
#endif
}
static double nrm2(int64_t n, const double* x) { return sqrt(dot(n, x, x)); }
static void scal(int64_t n, double a, double* x) {
  OMP_FOR
  for (int64_t r = 0; r < n; ++r) x[r] *= a;
}
static void vcopy(int64_t n, const double* x, double* y) {
  OMP_FOR
  for (int64_t r = 0; r < n; ++r) y[r] = x[r];
}
/* y = A x for CSR A */
static void csr_matvec(int64_t n, const int32_t* rowptr, const int32_t* colidx, const double* vals,
                       const double* x, double* y) {
  OMP_FOR
  for (int64_t r = 0; r < n; ++r) {
    acc_t s = 0.0;
    for (int32_t k = rowptr[r]; k < rowptr[r + 1]; ++k) s += (acc_t)vals[k] * x[colidx[k]];
    y[r] = (double)s;
  }
}

/* Householder reflector H = I - tau v v^T, v[0] = 1, with H x = (beta, 0, ..., 0)^T
 * (the LAPACK dlarfg convention: beta = -sign(alpha) ||x||).  x has m entries; on return
 * v holds the reflector and *beta the new leading entry. */
static void house_gen(int m, const double* x, double* v, double* tau, double* beta) {
  double alpha = x[0];
  double xn = 0.0;
  for (int t = 1; t < m; ++t) xn += x[t] * x[t];
  xn = sqrt(xn);
  v[0] = 1.0;
  if (xn == 0.0) {
    *tau = 0.0;
    *beta = alpha;
    for (int t = 1; t < m; ++t) v[t] = 0.0;
    return;
  }
  double b = -copysign(sqrt(alpha * alpha + xn * xn), alpha);
  *tau = (b - alpha) / b;
  double sc = 1.0 / (alpha - b);
  for (int t = 1; t < m; ++t) v[t] = x[t] * sc;
  *beta = b;
}
/* y <- (I - tau v v^T) y over m entries with stride `ld` between consecutive entries */
static void house_apply(int m, const double* v, double tau, double* y, int ld) {
  if (tau == 0.0) return;
  acc_t sa = 0.0;
  for (int t = 0; t < m; ++t) sa += (acc_t)v[t] * y[(int64_t)t * ld];
  double s = (double)sa * tau;
  for (int t = 0; t < m; ++t) y[(int64_t)t * ld] -= s * v[t];
}

/* Givens rotation zeroing b against a: [c s; -s c] [a; b] = [r; 0]. */
static void givens_gen(double a, double b, double* c, double* s, double* r) {
  if (b == 0.0) {
    *c = 1.0;
    *s = 0.0;
    *r = a;
    return;
  }
  double h = hypot(a, b);
  *c = a / h;
  *s = b / h;
  *r = h;
}

/* ---------------------------------------------------------------------------------------- */
typedef struct {
  int64_t n;
  const int32_t* rowptr;
  const int32_t* colidx;
  const double* vals;
} csr_t;

/* Orthogonalise r against q (unit vector) by one modified Gram-Schmidt step. */
static void mgs_step(int64_t n, const double* q, double* r) { axpy(n, -dot(n, q, r), q, r); }

int oracle_bminres(int64_t n, const int32_t* rowptr, const int32_t* colidx, const double* vals,
                   int p, const double* B, double* X, double tol, int maxit, double gamma,
                   int bench, uint64_t seed, int ghost, int qr_mode,
                   /* optional histories; pass NULL / 0 to skip */
                   int hist_cap, double* rho_hist, double* H_band, double* R_band,
                   int xhist_cap, double* X_hist, int ucap, double* U_hist, int defl_cap,
                   int* defl_iters, double* f0norm_out, oracle_info* info) {
  memset(info, 0, sizeof(*info));
  if (n < 0 || p < 0 || maxit < 0 || bench < 0 || !(tol > 0.0) || gamma < 0.0) {
    info->status = OR_ERR_INVALID;
    return OR_ERR_INVALID;
  }
  if (n == 0 || p == 0) {
    info->status = OR_OK;
    return OR_OK;
  }
  if (p > n) {
    info->status = OR_ERR_INVALID;
    return OR_ERR_INVALID;
  }
  csr_t A = {n, rowptr, colidx, vals};
  const int P1 = p + 1, W2 = 2 * p + 1; /* W2: ring length for Lanczos vectors and directions */
  int status = OR_OK;

  double* F0 = malloc(sizeof(double) * n * p);      /* initial residual, column-major */
  double* f0n = malloc(sizeof(double) * p);
  double* U = calloc((size_t)n * W2, sizeof(double));  /* u_i in slot i mod (2p+1)          */
  double* M = calloc((size_t)n * W2, sizeof(double));  /* m_i in slot i mod (2p+1)          */
  double* Wb = malloc(sizeof(double) * n * p);      /* block product W = A [u_j .. ]        */
  double* w = malloc(sizeof(double) * n);
  double* tmp = malloc(sizeof(double) * n);
  int nb = bench;
  double* Bench = malloc(sizeof(double) * (size_t)n * (nb > 0 ? nb : 1));
  double* Ghost = malloc(sizeof(double) * (size_t)n * (nb > 0 ? nb : 1));
  int* ghost_born = malloc(sizeof(int) * (nb > 0 ? nb : 1));
  double* S = calloc((size_t)p * p, sizeof(double));      /* S row-major p x p            */
  double* Shat = calloc((size_t)P1 * p, sizeof(double));  /* rows j..j+p of Shat          */
  double* hsub = calloc((size_t)p * p, sizeof(double));   /* C queue: h_{i+k,i}, k=1..p   */
  double* col = malloc(sizeof(double) * (3 * p + 1));     /* rows j-2p .. j+p              */
  double* hv = malloc(sizeof(double) * (size_t)2 * p * P1); /* reflectors of 2p columns   */
  double* htau = calloc(2 * p, sizeof(double));
  double* gc = malloc(sizeof(double) * (size_t)2 * p * p); /* Givens c, s of 2p columns     */
  double* gs = malloc(sizeof(double) * (size_t)2 * p * p);
  double* z = malloc(sizeof(double) * p);
  if (!F0 || !f0n || !U || !M || !Wb || !w || !tmp || !Bench || !Ghost || !ghost_born || !S ||
      !Shat || !hsub || !col || !hv || !htau || !gc || !gs || !z) {
    status = OR_ERR_OOM;
    goto done;
  }
#define USLOT(i) (U + (size_t)(((i) % W2 + W2) % W2) * n)
#define MSLOT(i) (M + (size_t)(((i) % W2 + W2) % W2) * n)

  /* ---- set-up: F0 = B - A X0 (Algorithm 2, first lines) ---- */
  for (int i = 0; i < p; ++i) {
    for (int64_t r = 0; r < n; ++r) tmp[r] = X[r * p + i];
    csr_matvec(n, A.rowptr, A.colidx, A.vals, tmp, w);
    double* f = F0 + (size_t)i * n;
    for (int64_t r = 0; r < n; ++r) f[r] = B[r * p + i] - w[r];
    f0n[i] = nrm2(n, f);
    if (f0norm_out) f0norm_out[i] = f0n[i];
  }
  {
    int all_zero = 1;
    for (int i = 0; i < p; ++i) all_zero &= (f0n[i] == 0.0);
    if (all_zero) { status = OR_OK; info->iters = 0; goto done; }
  }
  /* bench vectors, drawn before the iteration (Sec. 5.1) */
  for (int k = 0; k < nb; ++k) {
    OMP_FOR
    for (int64_t r = 0; r < n; ++r) Bench[(size_t)k * n + r] = oracle_bench_value(seed, k, n, r);
  }
  int bench_next = 0, n_ghost = 0;

  /* ---- economy QR F0 = U_p S by modified Gram-Schmidt with one re-orthogonalisation pass,
   *      with the dependence test of reading R7 (Eq. (init-QR)) ---- */
  int ucount = 0;
  for (int i = 0; i < p; ++i) {
    double* v = USLOT(i + 1);
    vcopy(n, F0 + (size_t)i * n, v);
    for (int pass = 0; pass < 2; ++pass)
      for (int k = 0; k < i; ++k) {
        double c = dot(n, USLOT(k + 1), v);
        S[k * p + i] += c;
        axpy(n, -c, USLOT(k + 1), v);
      }
    double nv = nrm2(n, v);
    if (!isfinite(nv)) { status = OR_ERR_NONFINITE; goto done; }
    if (nv <= gamma * f0n[i]) {
      /* dependent column: substitute a bench vector orthogonalised against u_1..u_{i} */
      info->setup_deflations++;
      S[i * p + i] = 0.0;
      if (bench_next >= nb) { status = OR_ERR_BENCH_EXHAUSTED; goto done; }
      vcopy(n, Bench + (size_t)bench_next * n, v);
      bench_next++;
      for (int pass = 0; pass < 2; ++pass)
        for (int k = 0; k < i; ++k) mgs_step(n, USLOT(k + 1), v);
      double nr = nrm2(n, v);
      if (!(nr > 0.0)) { status = OR_ERR_BENCH_EXHAUSTED; goto done; }
      scal(n, 1.0 / nr, v);
    } else {
      S[i * p + i] = nv;
      scal(n, 1.0 / nv, v);
    }
    /* remaining bench vectors are kept orthogonal to every new basis vector */
    for (int k = bench_next; k < nb; ++k) mgs_step(n, v, Bench + (size_t)k * n);
    if (U_hist && ucount < ucap) memcpy(U_hist + (size_t)ucount * n, v, sizeof(double) * n);
    ucount++;
  }
  /* Shat = E_1 S: rows 1..p are S, row p+1 is zero */
  for (int a = 0; a < p; ++a)
    for (int b = 0; b < p; ++b) Shat[a * p + b] = S[a * p + b];
  for (int b = 0; b < p; ++b) Shat[p * p + b] = 0.0;

  /* ---- band iterations j = 1, 2, ... (Algorithm 2) ---- */
  int j = 0;
  int converged = 0;
  while (!converged && j < maxit) {
    ++j;
    /* block product every p iterations (reading R3) */
    if ((j - 1) % p == 0)
      for (int l = 0; l < p; ++l)
        csr_matvec(n, A.rowptr, A.colidx, A.vals, USLOT(j + l), Wb + (size_t)l * n);
    int l = (j - 1) % p;
    vcopy(n, Wb + (size_t)l * n, w);
    double normAu = nrm2(n, w);
    for (int t = 0; t < 3 * p + 1; ++t) col[t] = 0.0;
    /* col[t] holds row (j - 2p + t); H column rows j-p..j+p sit at t = p..3p */
    /* known coefficients h_{i,j} = h_{j,i}, i = max(1, j-p) .. j-1 (Sec. 7, C queue) */
    for (int i = (j - p > 1 ? j - p : 1); i <= j - 1; ++i) {
      double h = hsub[(i % p) * p + (j - i - 1)];
      col[i - j + 2 * p] = h;
      axpy(n, -h, USLOT(i), w);
    }
    /* new inner products h_{i,j}, i = j .. j+p-1, modified Gram-Schmidt (Algorithm 1) */
    for (int i = j; i <= j + p - 1; ++i) {
      double h = dot(n, USLOT(i), w);
      col[i - j + 2 * p] = h;
      axpy(n, -h, USLOT(i), w);
    }
    /* removed vectors still in their band (reading R9): coefficient not entered in H */
    for (int g = 0; g < n_ghost; ++g)
      if (ghost_born[g] < j && j <= ghost_born[g] + 2 * p) mgs_step(n, Ghost + (size_t)g * n, w);
    double beta = nrm2(n, w);
    if (!isfinite(beta) || !isfinite(normAu)) { status = OR_ERR_NONFINITE; --j; break; }
    double* unew = USLOT(j + p);
    if (beta <= gamma * normAu) {
      /* dependence (Sec. 5): keep the removed vector, substitute a bench vector */
      if (defl_iters && info->deflations < defl_cap) defl_iters[info->deflations] = j;
      info->deflations++;
      if (bench_next >= nb) { status = OR_ERR_BENCH_EXHAUSTED; --j; break; }
      if (ghost && beta > GHOST_FLOOR * normAu) {
        /* reading R9: the kept vector is the part of w orthogonal to the window (one more MGS pass
         * against u_{j-p+1}..u_{j+p-1} and the removed vectors active at j), normalised; for an
         * exact dependence w is rounding noise with O(1) components along the window */
        double* g = Ghost + (size_t)n_ghost * n;
        vcopy(n, w, g);
        for (int i = (j - p + 1 > 1 ? j - p + 1 : 1); i <= j + p - 1; ++i) mgs_step(n, USLOT(i), g);
        for (int q = 0; q < n_ghost; ++q)
          if (ghost_born[q] < j && j <= ghost_born[q] + 2 * p) mgs_step(n, Ghost + (size_t)q * n, g);
        double ng = nrm2(n, g);
        if (ng > 0.0) {
          scal(n, 1.0 / ng, g);
          ghost_born[n_ghost] = j;
          n_ghost++;
        }
      }
      vcopy(n, Bench + (size_t)bench_next * n, unew);
      bench_next++;
      for (int i = (j - p + 1 > 1 ? j - p + 1 : 1); i <= j + p - 1; ++i) mgs_step(n, USLOT(i), unew);
      for (int g = 0; g < n_ghost; ++g)
        if (ghost_born[g] < j + 1 && j + 1 <= ghost_born[g] + 2 * p)
          mgs_step(n, Ghost + (size_t)g * n, unew);
      double nr = nrm2(n, unew);
      if (!(nr > 0.0)) { status = OR_ERR_BENCH_EXHAUSTED; --j; break; }
      scal(n, 1.0 / nr, unew);
      beta = 0.0;
    } else {
      vcopy(n, w, unew);
      scal(n, 1.0 / beta, unew);
    }
    col[3 * p] = beta; /* h_{j+p,j} */
    for (int k = bench_next; k < nb; ++k) mgs_step(n, unew, Bench + (size_t)k * n);
    if (U_hist && ucount < ucap) memcpy(U_hist + (size_t)ucount * n, unew, sizeof(double) * n);
    ucount++;
    /* C queue: subdiagonal entries of column j, h_{j+k,j}, k = 1..p */
    for (int k = 1; k <= p; ++k) hsub[(j % p) * p + (k - 1)] = col[2 * p + k];
    if (H_band && j <= hist_cap)
      for (int t = 0; t < W2; ++t) H_band[(size_t)(j - 1) * W2 + t] = col[p + t];

    /* ---- progressive band QR (Sec. 4): apply the 2p previous transforms, make the new one ---- */
    for (int i = (j - 2 * p > 1 ? j - 2 * p : 1); i <= j - 1; ++i) {
      int slot = i % (2 * p);
      int t0 = i - j + 2 * p; /* rows i..i+p */
      if (qr_mode == 0) {
        house_apply(P1, hv + (size_t)slot * P1, htau[slot], col + t0, 1);
      } else {
        for (int k = 1; k <= p; ++k) {
          double c = gc[slot * p + k - 1], s = gs[slot * p + k - 1];
          double a = col[t0], b = col[t0 + k];
          col[t0] = c * a + s * b;
          col[t0 + k] = -s * a + c * b;
        }
      }
    }
    int slot = j % (2 * p);
    double rjj;
    if (qr_mode == 0) {
      double tau;
      house_gen(P1, col + 2 * p, hv + (size_t)slot * P1, &tau, &rjj);
      htau[slot] = tau;
      col[2 * p] = rjj;
      for (int k = 1; k <= p; ++k) col[2 * p + k] = 0.0;
      /* reading R5: the same reflector acts on rows j..j+p of Shat (row j+p is the new zero row) */
      for (int b = 0; b < p; ++b) house_apply(P1, hv + (size_t)slot * P1, tau, Shat + b, p);
    } else {
      for (int k = 1; k <= p; ++k) {
        double c, s, r;
        givens_gen(col[2 * p], col[2 * p + k], &c, &s, &r);
        gc[slot * p + k - 1] = c;
        gs[slot * p + k - 1] = s;
        col[2 * p] = r;
        col[2 * p + k] = 0.0;
        for (int b = 0; b < p; ++b) {
          double a0 = Shat[0 * p + b], a1 = Shat[k * p + b];
          Shat[0 * p + b] = c * a0 + s * a1;
          Shat[k * p + b] = -s * a0 + c * a1;
        }
      }
      rjj = col[2 * p];
    }
    if (R_band && j <= hist_cap)
      for (int t = 0; t <= 2 * p; ++t) R_band[(size_t)(j - 1) * W2 + t] = col[t];
    if (!isfinite(rjj)) { status = OR_ERR_NONFINITE; --j; break; }
    if (rjj == 0.0) { status = OR_ERR_BREAKDOWN; --j; break; }

    /* ---- search direction, Eq. (search-dir-comp): m_j = (u_j - sum r_{i,j} m_i) / r_jj ---- */
    double* mj = MSLOT(j);
    vcopy(n, USLOT(j), mj);
    for (int i = (j - 2 * p > 1 ? j - 2 * p : 1); i <= j - 1; ++i)
      axpy(n, -col[i - j + 2 * p], MSLOT(i), mj);
    scal(n, 1.0 / rjj, mj);
    /* ---- progressive update, Eq. (approx-update): X_j = X_{j-1} + m_j z_j^T ---- */
    for (int b = 0; b < p; ++b) z[b] = Shat[0 * p + b];
    OMP_FOR
    for (int64_t r = 0; r < n; ++r) {
      double mr = mj[r];
      for (int b = 0; b < p; ++b) X[r * p + b] += mr * z[b];
    }
    /* ---- recursive residual, Eq. (comp-resid): rho_i = ||Shat(j+1:j+p, i)|| ---- */
    double worst = 0.0;
    for (int b = 0; b < p; ++b) {
      double s2 = 0.0;
      for (int k = 1; k <= p; ++k) s2 += Shat[k * p + b] * Shat[k * p + b];
      double rho = sqrt(s2);
      if (rho_hist && j <= hist_cap) rho_hist[(size_t)(j - 1) * p + b] = rho;
      double rel = f0n[b] > 0.0 ? rho / f0n[b] : 0.0;
      if (rel > worst) worst = rel;
    }
    if (X_hist && j <= xhist_cap) memcpy(X_hist + (size_t)(j - 1) * n * p, X, sizeof(double) * n * p);
    if (worst < tol) converged = 1;
    /* shift the Shat window: rows j+1..j+p become the top rows, append a zero row */
    memmove(Shat, Shat + p, sizeof(double) * p * p);
    for (int b = 0; b < p; ++b) Shat[p * p + b] = 0.0;
  }
  info->iters = j;
  if (status == OR_OK) status = converged ? OR_OK : OR_NOT_CONVERGED;
  info->bench_used = bench_next;

done:
  info->status = status;
  free(F0); free(f0n); free(U); free(M); free(Wb); free(w); free(tmp); free(Bench); free(Ghost);
  free(ghost_born); free(S); free(Shat); free(hsub); free(col); free(hv); free(htau); free(gc);
  free(gs); free(z);
  return status;
}

/* y = A X for a row-major n x p block (test helper: the residual B - A X is formed from it). */
void oracle_csr_spmm(int64_t n, const int32_t* rowptr, const int32_t* colidx, const double* vals,
                     int p, const double* X, double* Y) {
  for (int64_t r = 0; r < n; ++r) {
    for (int b = 0; b < p; ++b) Y[r * p + b] = 0.0;
    for (int32_t k = rowptr[r]; k < rowptr[r + 1]; ++k) {
      double a = vals[k];
      const double* xr = X + (int64_t)colidx[k] * p;
      for (int b = 0; b < p; ++b) Y[r * p + b] += a * xr[b];
    }
  }
}
