// Persistent cooperative kernel running one whole block MINRES solve (band Lanczos version,
// Algorithm 2 of Soodhalter's paper) on the GPU.
//
// Execution model
//   * One cooperative launch per solve.  Every block owns the same contiguous row range in every
//     phase, so row-local updates need no grid synchronisation.
//   * Per band iteration there is ONE streaming pass over the 2p-vector window: the update of
//     iteration j (B step) fused with the known-coefficient subtraction and the inner products of
//     iteration j+1 (A step).  Every p iterations the block product A [u_j .. u_{j+p-1}] runs,
//     fused with the A step of the first iteration of the cycle, and the search directions and the
//     iterate are updated once per cycle (p rank-1 updates of Eq. (approx-update) at once).
//   * The single-pass inner products are classical Gram-Schmidt; they are turned into the
//     modified Gram-Schmidt coefficients of Algorithm 1 exactly, through the Gram entries
//     u_i . u_k of the window recorded when each vector is created (one triangular recurrence of
//     p scalars).  Without it the window's rounding-level non-orthogonality is amplified every
//     iteration.
//   * After each pass every block reduces the per-block partial sums of ALL blocks in the same
//     fixed order, so every block holds bit-identical coefficients and takes identical decisions
//     (dependence test, band QR, convergence) without a broadcast.
//   * Warp 0 of each block is a control warp: between passes it updates the coefficients with
//     all 32 lanes, and DURING the next streaming pass it runs the band QR step of the iteration
//     just finished (the QR only feeds the end-of-cycle direction update and the stopping test,
//     which therefore lags one pass).  The other warps stream the vectors.
//   * The band QR uses Givens rotations (Sec. 4 uses Householder reflectors; R differs only in row
//     signs, X is the same).  The rotations of the last 2p columns are kept accumulated in an
//     orthogonal 3p x 2p window (the accumulation suggested at the end of Sec. 4), so applying
//     them to the new column is one small matrix-vector product; the p rotations of the new column
//     come from prefix norms in closed form.
//   * Lanczos vectors are stored unnormalised with a per-slot scale sigma_i (u_i = sigma_i raw_i).
//   * The streaming passes read their vectors through shared memory: tiles of rows are copied by
//     bulk asynchronous copies (cp.async.bulk, completion on an mbarrier) into two staging buffers,
//     two tiles ahead of the threads that compute on them (Engine::tiles); results go straight to
//     global memory.
//
// Data layout (all vectors have stride `ld` elements, V = double, float or dw (double-word)):
//   U     2p ring slots, u_i in slot i mod 2p        (band Lanczos FIFO, Sec. 7)
//   W     p slots: block product, overwritten in place by the partly orthogonalised w'
//   M     2p ring slots, m_i in slot i mod 2p        (search-direction FIFO, Sec. 7)
//   Bench NB bench vectors; Ghost NB removed vectors (normalised)
//   X     row-major n x p iterate (FP64 mode) or correction D (mixed mode, zeroed on entry)
// U, M and Ghost must be zero on entry.
#pragma once
#include <type_traits>

#include "common.cuh"
#include "dword.cuh"

namespace bmr {

template <typename V>
struct SolveArgs {
  int64_t n;
  int64_t ld;
  int p;
  int nbench;
  int ghost;
  int maxit;
  double tol;
  double gamma;
  uint64_t seed;
  const int32_t* rowptr;
  const int32_t* colidx;
  const V* vals;
  const V* F;  // p vectors: initial block residual F0
  V* X;
  V* U;
  V* W;
  V* M;
  V* Bench;
  V* Ghost;
  double* part;  // [2][NVMAX][nblocks]
  Ctl* ctl;
  double* rho_hist;  // optional: [hist_cap][p] recursive residual norms
  int hist_cap;
  unsigned long long barrier_limit_ns;
  unsigned barrier_extra;  // fault injection: arrivals a grid barrier waits for beyond the grid (0)
};

template <int PM>
struct Layout {
  static constexpr int GR = (PM > 1) ? PM - 1 : 1;  // Gram entries kept per Lanczos vector
  // fused pass (B step of j + A step of j+1)
  static constexpr int BA_NRM = 0, BA_W1 = 1, BA_DOT = 2, BA_GR = 2 + PM, BA_BEN = 2 + PM + GR,
                       BA_GH = 2 + PM + GR + NBMAX;
  static constexpr int BA_N = 2 + PM + GR + 2 * NBMAX;
  // block-product pass
  static constexpr int SP_NRM = 0, SP_DOT = 1, SP_GH = 1 + PM, SP_N = 1 + PM + NBMAX;
  // substitution pass D2
  static constexpr int D2_NRM = 0, D2_BEN = 1, D2_GR = 1 + NBMAX, D2_N = 1 + NBMAX + GR;
  static constexpr int NVMAX = (2 * PM + NBMAX > BA_N) ? 2 * PM + NBMAX : BA_N;
};

constexpr int NSTAGE_MAX = 2;  // staging buffers of the streaming passes (fewer for p > 16)
constexpr int TQMAX = 512;  // tiles per block whose CSR offsets are tabulated for the block product

// Element type of the coefficient copies read by the streaming passes: the vector element type for
// FP32 and double-word vectors (so that the row loops convert nothing), unused for FP64 vectors.
template <typename V> struct CoefCopy { using T = V; };
template <> struct CoefCopy<double> { using T = unsigned char; };
template <typename CT> __device__ __forceinline__ CT to_coef(double d) { return (CT)d; }
template <> __device__ __forceinline__ unsigned char to_coef<unsigned char>(double) { return 0; }

template <int PM, typename CT>
struct __align__(16) Shared {
  unsigned long long tbar[NSTAGE_MAX];  // completion barriers of the staging buffers
  unsigned long long bar_epoch;         // grid barriers this block has passed (thread 0)
  int tq[TQMAX + 1];                // rowptr at the block-product tile boundaries of this block
  int tq_n;                         // tiles tabulated (-1: too many, CSR read directly)
  int csr_nnz;                      // rowptr[n]
  // vectors staged by the current streaming pass: global address of row 0 and byte offset of
  // the slot in a staging buffer (written and read by the issuing warp only)
  const char* cp_src[3 * PM + 8];
  unsigned cp_dst[3 * PM + 8];
  int cp_n, cp_pad;
  int terr, pad_t;                  // a staging wait ran out in this block
  int cycle, status, qstop, qstatus;
  int bench_next, n_ghost, deflations, setup_defl;
  int ghost_born[NBMAX];
  double beta;                  // h_{j+p,j} of the last pass (0 after a substitution)
  double sigq;                  // sigma_j of the column handed to the QR warp
  double f0n[PM];
  double thr2[PM];              // (tol * ||f0_i||)^2
  double inv2[PM];              // 1 / ||f0_i||^2 (0 for a zero column)
  double rho2[PM];              // squared recursive residuals of the last QR step
  double sigma[2 * PM];         // scale of U slots (slot = i mod 2p)
  double hsub[PM][PM];          // C queue: hsub[i mod p][k-1] = h_{i+k,i}
  double hdiag[2];              // h_{i,i} for i = j, j+1 (slot i & 1)
  double normAu2[2];            // ||A u_i||^2, same slots
  double coefB[PM];             // B step of j: h_{j+k,j} sigma_{j+k}
  double coefA[PM];             // A step of j+1: h_{j+1,i} sigma_i, i = j+1-p+k
  double cgB[NBMAX];            // removed-vector coefficients of the B step
  double gram[2 * PM][Layout<PM>::GR];  // gram[i mod 2p][m-1] = u_i . u_{i-m}, m = 1..p-1
  double P[3 * PM][2 * PM];     // accumulated rotations, ring indexed [row mod 3p][col mod 2p]
  double Sh[PM + 1][PM];        // rows j..j+p of Shat, ring indexed by row mod (p+1)
  double colq[2 * PM + 1];      // column j of H-bar (rows j-p..j+p) handed to the QR warp
  double y[3 * PM + 1];         // rotated column, rows j-2p..j+p
  double pref[PM + 1], rinv[PM + 1], gc[PM + 1], gs[PM + 1];
  double rjj[PM];               // r_{j,j} of the iterations of the current cycle
  double Zc[PM][PM];            // z_j of the current cycle
  double bc[NBMAX][2][PM];      // bench maintenance coefficients, by cycle parity
  double dirA[PM];              // direction recurrence coefficients of the cycle:
  union {                       // dirB[l][q] multiplies m_{j0+l-2PM+q}; S only during set-up
    double dirB[PM][2 * PM];
    double S[PM][PM];           // initial QR factor
  };
  double qd[PM], qe[PM];        // set-up Gram-Schmidt coefficients
  // copies of the coefficients read in the row loops, in the vector element type (conversions from
  // double run on the slow FP64 pipe of GB300, so they are done once, by the control warp)
  CT dirAc[PM], dirBc[PM][2 * PM], Zcc[PM][PM], bcc[NBMAX][2][PM];
  CT coefAc[PM], coefBc[PM], cgBc[NBMAX];
  double red[Layout<PM>::NVMAX];   // values of the last grid reduction
  double rba[Layout<PM>::NVMAX];   // saved values of the last fused pass
  double s2[Layout<PM>::NVMAX][32];
  double d4[Layout<PM>::NVMAX][4];
};

// ---- G consecutive elements of a vector in one access (G * sizeof(V) <= 16 bytes, aligned) ----
template <int G>
struct IC {
  static constexpr int value = G;
};

template <int G, typename V>
__device__ __forceinline__ void vld(const V* p, V (&x)[G]) {
  static_assert(G == 1 || G == 2 || G == 4, "group width");
  static_assert(G * sizeof(V) <= 16, "group wider than 16 bytes");
  if constexpr (std::is_same<V, dw>::value) {
    if constexpr (G == 1) {
      const float2 t = *reinterpret_cast<const float2*>(p);
      x[0] = dw::make(t.x, t.y);
    } else {
      const float4 t = *reinterpret_cast<const float4*>(p);
      x[0] = dw::make(t.x, t.y);
      x[1] = dw::make(t.z, t.w);
    }
  } else if constexpr (G == 1) {
    x[0] = *p;
  } else if constexpr (sizeof(V) == 8) {
    const double2 t = *reinterpret_cast<const double2*>(p);
    x[0] = t.x;
    x[1] = t.y;
  } else if constexpr (G == 2) {
    const float2 t = *reinterpret_cast<const float2*>(p);
    x[0] = t.x;
    x[1] = t.y;
  } else {
    const float4 t = *reinterpret_cast<const float4*>(p);
    x[0] = t.x;
    x[1] = t.y;
    x[2] = t.z;
    x[3] = t.w;
  }
}

template <int G, typename V>
__device__ __forceinline__ void vst(V* p, const V (&x)[G]) {
  if constexpr (std::is_same<V, dw>::value) {
    if constexpr (G == 1)
      *reinterpret_cast<float2*>(p) = make_float2(x[0].hi, x[0].lo);
    else
      *reinterpret_cast<float4*>(p) = make_float4(x[0].hi, x[0].lo, x[1].hi, x[1].lo);
  } else if constexpr (G == 1) {
    *p = x[0];
  } else if constexpr (sizeof(V) == 8) {
    *reinterpret_cast<double2*>(p) = make_double2(x[0], x[1]);
  } else if constexpr (G == 2) {
    *reinterpret_cast<float2*>(p) = make_float2(x[0], x[1]);
  } else {
    *reinterpret_cast<float4*>(p) = make_float4(x[0], x[1], x[2], x[3]);
  }
}

// G consecutive elements from shared memory (16/8/4-byte aligned).  Volatile, so that a value the
// code reads twice is re-read from shared memory instead of being held in registers across a row.
template <int G>
__device__ __forceinline__ void sld(const float* p, float (&x)[G]) {
  const unsigned a = smem_u32(p);
  if constexpr (G == 1) {
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(x[0]) : "r"(a));
  } else if constexpr (G == 2) {
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(x[0]), "=f"(x[1]) : "r"(a));
  } else {
    static_assert(G == 4, "group width");
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(x[0]), "=f"(x[1]), "=f"(x[2]), "=f"(x[3]) : "r"(a));
  }
}
template <int G>
__device__ __forceinline__ void sld(const double* p, double (&x)[G]) {
  const unsigned a = smem_u32(p);
  if constexpr (G == 1) {
    asm volatile("ld.shared.f64 %0, [%1];" : "=d"(x[0]) : "r"(a));
  } else {
    static_assert(G == 2, "group width");
    asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(x[0]), "=d"(x[1]) : "r"(a));
  }
}

template <int G>
__device__ __forceinline__ void sld(const dw* p, dw (&x)[G]) {
  const unsigned a = smem_u32(p);
  float h0, l0, h1, l1;
  if constexpr (G == 1) {
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(h0), "=f"(l0) : "r"(a));
    x[0] = dw::make(h0, l0);
  } else {
    static_assert(G == 2, "group width");
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(h0), "=f"(l0), "=f"(h1), "=f"(l1) : "r"(a));
    x[0] = dw::make(h0, l0);
    x[1] = dw::make(h1, l1);
  }
}

// one CSR value through the read-only path
__device__ __forceinline__ double ldg_val(const double* p) { return __ldg(p); }
__device__ __forceinline__ float ldg_val(const float* p) { return __ldg(p); }
__device__ __forceinline__ dw ldg_val(const dw* p) {
  const float2 t = __ldg(reinterpret_cast<const float2*>(p));
  return dw::make(t.x, t.y);
}

// a * b + c in the vector arithmetic (contracted to one FMA for FP64 and FP32 vectors)
__device__ __forceinline__ double madd(double a, double b, double c) { return a * b + c; }
__device__ __forceinline__ float madd(float a, float b, float c) { return a * b + c; }
__device__ __forceinline__ dw madd(dw a, dw b, dw c) { return dw_fma(a, b, c); }

// Per-thread accumulation of inner products (a += x * y), block-level sums (a += b) and the FP64
// value of an accumulator, for every vector element type.
__device__ __forceinline__ void dot_add(double& a, double x, double y) { a = fma(x, y, a); }
__device__ __forceinline__ void dot_add(float& a, float x, float y) { a = fmaf(x, y, a); }
__device__ __forceinline__ void dot_sum(double& a, double b) { a += b; }
__device__ __forceinline__ void dot_sum(float& a, float b) { a += b; }
__device__ __forceinline__ double dot_val(double a) { return a; }
__device__ __forceinline__ double dot_val(float a) { return (double)a; }
__device__ __forceinline__ void dot_add(dw& a, dw x, dw y) { a = dw_fma(x, y, a); }
__device__ __forceinline__ void dot_sum(dw& a, dw b) { a = dw_add(a, b); }
__device__ __forceinline__ double dot_val(dw a) { return to_double(a); }

// Shared-memory staging of the streaming passes: NSTAGE buffers of STG bytes after the Shared block
// (the reduction scratch reuses them).  A pass that streams `nsl` vector slots per row works on
// tiles of rows(nsl) rows; its consumers take groups of group(nsl) consecutive rows.
template <typename V, int PM, int NT>
struct Tiles {
  static constexpr int NS = NT - 32;
  static constexpr int NSTAGE = PM > 16 ? 2 : NSTAGE_MAX;
  static constexpr size_t SH = (sizeof(Shared<PM, typename CoefCopy<V>::T>) + 127) / 128 * 128;
  static constexpr size_t BUDGET = 227 * 1024 - 1024;  // dynamic shared memory of one block
  static constexpr size_t STG_MAX = 80 * 1024;
  static constexpr size_t STG =
      ((BUDGET - SH) / NSTAGE < STG_MAX ? (BUDGET - SH) / NSTAGE : STG_MAX) / 128 * 128;
  __host__ __device__ static constexpr int cap(int nsl) { return (int)(STG / ((size_t)nsl * sizeof(V))); }
  __host__ __device__ static constexpr int group(int nsl) {
    int g = 16 / (int)sizeof(V);
    while (g > 1 && NS * g > cap(nsl)) g /= 2;
    return g;
  }
  __host__ __device__ static constexpr int rows(int nsl) {
    return cap(nsl) >= NS * group(nsl) ? cap(nsl) / (NS * group(nsl)) * (NS * group(nsl)) : cap(nsl) / 32 * 32;
  }
  __host__ __device__ static constexpr size_t smem_bytes() { return SH + NSTAGE * STG; }
  // block product: rows per tile and group width, with the tile's CSR segment staged beside the
  // 2p vector slots (up to 8 nonzeros per row on average)
  __host__ __device__ static constexpr size_t sp_bytes(int t) {
    return ((size_t)2 * PM * t * sizeof(V) + (size_t)(t + 4) * 4 + 15) / 16 * 16 +
           ((size_t)8 * t * 4 + 15) / 16 * 16 + (size_t)8 * t * sizeof(V);
  }
  __host__ __device__ static constexpr int sp_group() {
    int g = 16 / (int)sizeof(V);
    while (g > 1 && sp_bytes(NS * g) > STG) g /= 2;
    return g;
  }
  __host__ __device__ static constexpr int sp_rows() {
    int t = NS * sp_group();
    if (sp_bytes(t) > STG) {
      t = 32;
      while (sp_bytes(t + 32) <= STG) t += 32;
    }
    return t;
  }
};

template <typename V, int PM, int NT>
struct Engine {
  using A = V;  // arithmetic on vector elements
  using R = A;  // per-thread inner-product accumulators
  using LY = Layout<PM>;
  static constexpr int NVMAX = LY::NVMAX;
  static constexpr int NS = NT - 32;  // streaming threads (warps 1..NT/32-1)
  static constexpr int RCH = 16;      // values per chunk of a block reduction
  static constexpr int NBPRE = 4;     // bench vectors held in registers by the fused pass
  const SolveArgs<V>& a;
  using SHT = Shared<PM, typename CoefCopy<V>::T>;
  using CT = typename CoefCopy<V>::T;
  SHT& sh;
  using TL = Tiles<V, PM, NT>;
  A* scr;  // [RCH][NS] scratch for block reductions (inside the staging buffers)
  V* stg;  // staging buffers
  unsigned tseq;  // tiles consumed so far (the same in every streaming thread)
  int64_t rb, re;
  int nblocks;
  int buf;
  int p;
  int lane, warp;
  unsigned long long t_mark;

  __device__ Engine(const SolveArgs<V>& args, SHT& s, V* scratch)
      : a(args), sh(s), scr(reinterpret_cast<A*>(scratch)), stg(scratch), tseq(0), buf(0), p(args.p), t_mark(0) {
    nblocks = gridDim.x;
    int64_t chunk = (a.n + nblocks - 1) / nblocks;
    chunk = (chunk + 31) / 32 * 32;
    rb = (int64_t)blockIdx.x * chunk;
    re = rb + chunk;
    if (re > a.n) re = a.n;
    if (rb > a.n) rb = a.n;
    lane = threadIdx.x & 31;
    warp = threadIdx.x >> 5;
  }

  // first row of this streaming thread (rows advance by NS); control-warp threads get re
  __device__ __forceinline__ int64_t row0() const { return warp == 0 ? re : rb + (threadIdx.x - 32); }

  __device__ __forceinline__ V* stage(int s) const { return stg + (size_t)s * (TL::STG / sizeof(V)); }
  __device__ __forceinline__ static unsigned vbytes(int rows) {  // one vector's tile, whole 16 bytes
    return (unsigned)(((size_t)rows * sizeof(V) + 15) / 16 * 16);
  }

  // (warp 1) entry c of the copy list: vector src into slot `slot` of a tile of T rows
  __device__ __forceinline__ void cp_put(int c, const V* src, int slot, int T) {
    sh.cp_src[c] = reinterpret_cast<const char*>(src);
    sh.cp_dst[c] = (unsigned)((size_t)slot * T * sizeof(V));
  }
  // (warp 1) one tile of every listed vector into buffer sb, plus `extra` bytes that the caller
  // copies itself after this returns; lane 0 announces the bytes before any copy is issued
  __device__ __forceinline__ void cp_issue(int sb, int64_t r0, int rows, unsigned extra) {
    const unsigned by = vbytes(rows);
    unsigned long long* bar = &sh.tbar[sb];
    char* d = reinterpret_cast<char*>(stage(sb));
    const int n = sh.cp_n;
    if (lane == 0) mbar_arrive_expect_tx(bar, (unsigned)n * by + extra);
    __syncwarp();
    const size_t off = (size_t)r0 * sizeof(V);
    for (int c = lane; c < n; c += 32) bulk_g2s(d + sh.cp_dst[c], sh.cp_src[c] + off, by, bar);
  }

  // Staged streaming loop of the streaming warps over rows [rb, re) in tiles of T rows.  Tile i
  // goes to buffer (tseq + i) mod NSTAGE: warp 1 issues its bulk copies with issue(buffer, r0,
  // rows) (one mbarrier arrival announcing the bytes, then the copies), NSTAGE tiles ahead; every streaming
  // thread waits for the buffer's phase (bounded), runs body(IC<G>, tile, o, r0 + o, rows) on
  // groups of G rows (a partial last group row by row), and the streaming warps meet on named
  // barrier 1 before the buffer is refilled.  The writes of the pass are fenced against the bulk
  // (async-proxy) reads of later passes.  Returns false, with ctl->err set, if a wait ran out.
  template <int T, int G, typename ISSUE, typename BODY>
  __device__ __forceinline__ bool tiles(ISSUE&& issue, BODY&& body) {
    static_assert(T >= 32 && T % G == 0 && T % 32 == 0, "tile shape");
    const int st = threadIdx.x - 32;
    const int64_t nrows = re - rb;
    const int nt = nrows > 0 ? (int)((nrows + T - 1) / T) : 0;
    if (warp == 1) {
      fence_proxy_async();
      for (int i = 0; i < TL::NSTAGE && i < nt; ++i)
        issue((int)((tseq + i) % TL::NSTAGE), rb + (int64_t)i * T, (int)min((int64_t)T, nrows - (int64_t)i * T));
    }
    int i = 0;
    for (; i < nt; ++i) {
      const unsigned seq = tseq + i;
      const int s = (int)(seq % TL::NSTAGE);
      const int64_t r0 = rb + (int64_t)i * T;
      const int rows = (int)min((int64_t)T, nrows - (int64_t)i * T);
      if (mbar_wait(&sh.tbar[s], (seq / TL::NSTAGE) & 1u, a.barrier_limit_ns)) {
        const V* tl = stage(s);
#pragma unroll 1
        for (int o = st * G; o < rows; o += NS * G) {
          if (o + G <= rows) {
            body(IC<G>{}, tl, o, r0 + o, rows);
          } else {
            for (int e = o; e < rows; ++e) body(IC<1>{}, tl, e, r0 + e, rows);
          }
        }
      } else {
        sh.terr = 1;
      }
      named_sync(1, NS);
      if (*reinterpret_cast<volatile int*>(&sh.terr)) break;
      if (warp == 1 && i + TL::NSTAGE < nt)
        issue(s, r0 + (int64_t)TL::NSTAGE * T, (int)min((int64_t)T, nrows - (int64_t)(i + TL::NSTAGE) * T));
    }
    fence_proxy_async();
    if (i < nt) {  // a wait ran out: record it, let the copies in flight land (bounded), give up
      if (st == 0) {
        atomicExch(&a.ctl->err, ST_ERR_TIMEOUT);
        for (int k = i; k < nt && k < i + TL::NSTAGE; ++k)
          mbar_wait(&sh.tbar[(tseq + k) % TL::NSTAGE], ((tseq + k) / TL::NSTAGE) & 1u, a.barrier_limit_ns);
      }
      return false;
    }
    tseq += nt;
    return true;
  }

  __device__ __forceinline__ int ring2p(int i) const { return ((i % (2 * p)) + 2 * p) % (2 * p); }
  __device__ __forceinline__ V* uslot(int i) const { return a.U + (int64_t)ring2p(i) * a.ld; }
  __device__ __forceinline__ V* mslot(int i) const { return a.M + (int64_t)ring2p(i) * a.ld; }
  __device__ __forceinline__ double& sig(int i) { return sh.sigma[ring2p(i)]; }
  __device__ __forceinline__ V* wslot(int k) const { return a.W + (int64_t)k * a.ld; }
  __device__ __forceinline__ V* bench(int k) const { return a.Bench + (int64_t)k * a.ld; }
  __device__ __forceinline__ V* ghostv(int g) const { return a.Ghost + (int64_t)g * a.ld; }
  __device__ __forceinline__ bool ghost_active(int g, int jj) const {
    return g < sh.n_ghost && sh.ghost_born[g] < jj && jj <= sh.ghost_born[g] + 2 * p;
  }

  // block 0's timeline, measured by its first streaming thread
  __device__ __forceinline__ void tick(unsigned long long& bucket) {
    if (blockIdx.x == 0 && threadIdx.x == 32) {
      unsigned long long t = gtimer();
      bucket += t - t_mark;
      t_mark = t;
    }
  }
  __device__ __forceinline__ void set_status(int st) {
    if (threadIdx.x == 0 && sh.status == ST_OK) sh.status = st;
    __syncthreads();
  }

  // ---- reduction of nv per-thread values over the whole grid -> sh.red[0..nv) ----------------
  // Inside the block: transpose the streaming threads' values through shared memory and sum in a
  // fixed order; across blocks: every block sums the per-block partials of all blocks in the same
  // fixed order.  Returns false if a grid barrier failed.
  template <typename T, int NVC>
  __device__ bool reduce(const T (&acc)[NVC], int nv) {
    static_assert(sizeof(T) <= 8, "reduction scratch element");
    const int tid = threadIdx.x;
    T* sc = reinterpret_cast<T*>(scr);
    fence_proxy_async();  // this pass's vector writes before later bulk (async-proxy) reads of them
#pragma unroll
    for (int c0 = 0; c0 < NVC; c0 += RCH) {
      if (c0 < nv) {
        if (warp > 0) {
#pragma unroll
          for (int v = 0; v < RCH; ++v)
            if (c0 + v < NVC && c0 + v < nv) sc[v * NS + tid - 32] = acc[c0 + v];
        }
        __syncthreads();
        const int cn = (nv - c0 < RCH) ? nv - c0 : RCH;
        for (int task = tid; task < cn * 32; task += NT) {
          int v = task >> 5, l = task & 31;
          T s = sc[v * NS + l];
#pragma unroll
          for (int q = 1; q < NS / 32; ++q) dot_sum(s, sc[v * NS + l + 32 * q]);
          sh.s2[c0 + v][l] = dot_val(s);
        }
        __syncthreads();
      }
    }
    fold32(nv);
    if (nblocks == 1) {
      for (int v = tid; v < nv; v += NT) sh.red[v] = (sh.d4[v][0] + sh.d4[v][1]) + (sh.d4[v][2] + sh.d4[v][3]);
      __syncthreads();
      return true;
    }
    double* part = a.part + (int64_t)buf * NVMAX * nblocks;
    for (int v = tid; v < nv; v += NT)
      part[(int64_t)v * nblocks + blockIdx.x] = (sh.d4[v][0] + sh.d4[v][1]) + (sh.d4[v][2] + sh.d4[v][3]);
    buf ^= 1;
    if (!grid_barrier(a.ctl, nblocks + a.barrier_extra, sh.bar_epoch, a.barrier_limit_ns)) return false;
    for (int task = tid; task < nv * 32; task += NT) {
      int v = task >> 5, l = task & 31;
      const double* pv = part + (int64_t)v * nblocks;
      double s = 0.0;
      for (int b = l; b < nblocks; b += 32) s += pv[b];
      sh.s2[v][l] = s;
    }
    __syncthreads();
    fold32(nv);
    for (int v = tid; v < nv; v += NT) sh.red[v] = (sh.d4[v][0] + sh.d4[v][1]) + (sh.d4[v][2] + sh.d4[v][3]);
    __syncthreads();
    return true;
  }
  __device__ __forceinline__ void fold32(int nv) {
    for (int task = threadIdx.x; task < nv * 4; task += NT) {
      int v = task >> 2, q = task & 3;
      const double* s = sh.s2[v] + 8 * q;
      sh.d4[v][q] = ((s[0] + s[1]) + (s[2] + s[3])) + ((s[4] + s[5]) + (s[6] + s[7]));
    }
    __syncthreads();
  }

  // ---- set-up ---------------------------------------------------------------------------------
  __device__ bool setup_norms() {
    A acc[PM];
#pragma unroll
    for (int k = 0; k < PM; ++k) acc[k] = 0;
    for (int64_t r = row0(); r < re; r += NS) {
#pragma unroll
      for (int k = 0; k < PM; ++k)
        if (k < p) {
          A f = a.F[(int64_t)k * a.ld + r];
          acc[k] += f * f;
        }
    }
    if (!reduce(acc, p)) return false;
    if (threadIdx.x < p) {
      const int i = threadIdx.x;
      const double f2 = sh.red[i];
      sh.f0n[i] = sqrt(f2);
      sh.thr2[i] = a.tol * a.tol * f2;
      sh.inv2[i] = (f2 > 0.0) ? 1.0 / f2 : 0.0;
    }
    // bench vectors, drawn before the iteration (Sec. 5.1)
    for (int k = 0; k < a.nbench; ++k)
      for (int64_t r = row0(); r < re; r += NS) bench(k)[r] = (V)bench_value(a.seed, k, a.n, r);
    __syncthreads();
    return true;
  }

  // One column of the initial economy QR F0 = U_p S (Eq. (init-QR)): classical Gram-Schmidt with
  // one re-orthogonalisation, from `src` into the slot of u_{i+1}.  Leaves the squared norm in
  // sh.red[0] and the raw inner products with the remaining bench vectors in sh.red[1 + b].
  __device__ bool setup_column(int i, const V* src, bool record_S) {
    const int tid = threadIdx.x;
    if (tid < PM) {
      sh.qd[tid] = 0.0;
      sh.qe[tid] = 0.0;
    }
    __syncthreads();
    if (i > 0) {
      {
        A acc[PM];
#pragma unroll
        for (int k = 0; k < PM; ++k) acc[k] = 0;
        for (int64_t r = row0(); r < re; r += NS) {
          A s = src[r];
#pragma unroll
          for (int k = 0; k < PM; ++k)
            if (k < i) acc[k] += (A)uslot(k + 1)[r] * s;
        }
        if (!reduce(acc, i)) return false;
        if (tid < i) sh.qd[tid] = sig(tid + 1) * sig(tid + 1) * sh.red[tid];
        __syncthreads();
      }
      {
        A cf[PM];
#pragma unroll
        for (int k = 0; k < PM; ++k) cf[k] = (k < i) ? (A)sh.qd[k] : (A)0;
        A acc[PM];
#pragma unroll
        for (int k = 0; k < PM; ++k) acc[k] = 0;
        for (int64_t r = row0(); r < re; r += NS) {
          A v = src[r];
          A uk[PM];
#pragma unroll
          for (int k = 0; k < PM; ++k) {
            uk[k] = (k < i) ? (A)uslot(k + 1)[r] : (A)0;
            v -= cf[k] * uk[k];
          }
#pragma unroll
          for (int k = 0; k < PM; ++k)
            if (k < i) acc[k] += uk[k] * v;
        }
        if (!reduce(acc, i)) return false;
        if (tid < i) sh.qe[tid] = sig(tid + 1) * sig(tid + 1) * sh.red[tid];
        __syncthreads();
      }
    }
    A cf[PM];
#pragma unroll
    for (int k = 0; k < PM; ++k) cf[k] = (k < i) ? (A)(sh.qd[k] + sh.qe[k]) : (A)0;
    constexpr int NVC = 1 + NBMAX;
    A acc[NVC];
#pragma unroll
    for (int k = 0; k < NVC; ++k) acc[k] = 0;
    const int b0 = sh.bench_next, nb = a.nbench;
    V* dst = uslot(i + 1);
    for (int64_t r = row0(); r < re; r += NS) {
      A v = src[r];
#pragma unroll
      for (int k = 0; k < PM; ++k)
        if (k < i) v -= cf[k] * (A)uslot(k + 1)[r];
      dst[r] = (V)v;
      acc[0] += v * v;
#pragma unroll
      for (int b = 0; b < NBMAX; ++b)
        if (b >= b0 && b < nb) acc[1 + b] += (A)bench(b)[r] * v;
    }
    if (!reduce(acc, 1 + nb)) return false;
    if (record_S && tid < i) sh.S[tid][i] = (sh.qd[tid] + sh.qe[tid]) / sig(tid + 1);
    __syncthreads();
    return true;
  }

  // ---- block product fused with the A step of iteration j0 (first pass of a cycle) ------------
  // W_k = A u_{j0+k}; w'_{j0} = W_0 - sum_{i<j0} h_{j0,i} u_i (into W slot 0); inner products
  // u_{j0+k} . w'_{j0}; removed-vector products; ||W_0||^2.  The control warp runs the QR step of
  // iteration qr_j (if > 0) meanwhile.
  // Staged per tile: u_{j0} .. u_{j0+p-1} (own rows; they also serve the gathers that fall in the
  // tile), u_{j0-p} .. u_{j0-1}, and the tile's CSR segment: rowptr, colidx and values, copied in
  // whole 16-byte units inside the arrays (entries outside the copied ranges are read directly).

  // rowptr at this block's block-product tile boundaries (the CSR structure is fixed per solve)
  __device__ void tabulate_csr_tiles() {
    constexpr int T = TL::sp_rows();
    const int64_t nrows = re - rb;
    const int nt = nrows > 0 ? (int)((nrows + T - 1) / T) : 0;
    const bool fit = nt <= TQMAX;
    if (fit)
      for (int i = threadIdx.x; i <= nt; i += NT) sh.tq[i] = __ldg(a.rowptr + min(rb + (int64_t)i * T, re));
    if (threadIdx.x == 0) {
      sh.tq_n = fit ? nt : -1;
      sh.csr_nnz = __ldg(a.rowptr + a.n);
    }
    __syncthreads();
  }

  struct CsrTile {
    bool ok;     // CSR segment staged
    int nrp;     // rowptr entries staged (from r0)
    int64_t qa;  // colidx / values staged for nonzeros [qa, qb)
    int64_t qb;
  };
  // what is staged of the CSR arrays for block-product tile i (rows [r0, r0 + rows))
  __device__ __forceinline__ CsrTile csr_tile(int i, int64_t r0, int rows, bool csr_al) const {
    constexpr int T = TL::sp_rows();
    CsrTile c{false, 0, 0, 0};
    if (!csr_al || sh.tq_n < 0) return c;
    const int64_t end4 = (a.n + 1) / 4 * 4;  // rowptr entries readable in whole 16-byte units
    c.nrp = (int)max((int64_t)0, min((int64_t)((rows + 3) / 4 * 4), end4 - r0));
    const int64_t nnz = sh.csr_nnz;
    c.qa = (int64_t)sh.tq[i] / 4 * 4;
    c.qb = min(((int64_t)sh.tq[i + 1] + 3) / 4 * 4, nnz / 4 * 4);
    if (c.qb < c.qa) c.qb = c.qa;
    c.ok = (c.qb - c.qa) <= (int64_t)8 * T;
    return c;
  }

  __device__ bool pass_spmm(int j0, int qr_j, int qr_l) {
    R acc[LY::SP_N];  // written after the streaming loop
    int ng = 0;
#pragma unroll
    for (int g = 0; g < NBMAX; ++g)
      if (g < sh.n_ghost) ng = g + 1;
    if (warp == 0) {
      if (qr_j > 0) qr_warp(qr_j, qr_l);
#pragma unroll
      for (int k = 0; k < LY::SP_N; ++k) acc[k] = R{};
    } else {
      constexpr int T = TL::sp_rows(), G = TL::sp_group();
      constexpr size_t OUK = (size_t)PM * T * sizeof(V), ORP = 2 * OUK;
      constexpr size_t OCI = ORP + ((size_t)(T + 4) * 4 + 15) / 16 * 16;
      constexpr size_t OCV = OCI + ((size_t)8 * T * 4 + 15) / 16 * 16;
      static_assert(OCV + (size_t)8 * T * sizeof(V) <= TL::STG, "block-product tile");
      const bool csr_al = ((reinterpret_cast<uintptr_t>(a.rowptr) | reinterpret_cast<uintptr_t>(a.colidx) |
                            reinterpret_cast<uintptr_t>(a.vals)) & 15u) == 0;
      // coefficients (negated), scales and slot addresses of u_{j0+k}: registers for p <= 8, computed
      // where used for larger blocks (register budget); the slots of u_{j0} .. u_{j0+p-1} are
      // (s0 + k) mod 2p
      constexpr bool CREG = PM <= 8;
      A cA[CREG ? PM : 1], sg[CREG ? PM : 1];
      const V* usrc[CREG ? PM : 1];
      const int s0 = ring2p(j0);
      if constexpr (CREG) {
#pragma unroll
        for (int k = 0; k < PM; ++k) {
          cA[k] = (k < p) ? -ccoefA(k) : (A)0;
          sg[k] = (k < p) ? (A)sig(j0 + k) : (A)0;
          usrc[k] = uslot(j0 + k);
        }
      }
      auto uk = [&](int k) __attribute__((always_inline)) -> const V* {
        if constexpr (CREG) {
          return usrc[k];
        } else {
          const int sl = s0 + k;
          return a.U + (int64_t)(sl >= 2 * p ? sl - 2 * p : sl) * a.ld;
        }
      };
      auto cAk = [&](int k) __attribute__((always_inline)) -> A {
        if constexpr (CREG) return cA[k]; else return -ccoefA(k);
      };
      auto sgk = [&](int k) __attribute__((always_inline)) -> A {
        if constexpr (CREG) return sg[k]; else return (A)sh.sigma[s0 + k >= 2 * p ? s0 + k - 2 * p : s0 + k];
      };
      const bool has_known = (j0 > 1);
      bool gact[NBMAX];
#pragma unroll
      for (int g = 0; g < NBMAX; ++g) gact[g] = ghost_active(g, j0);
      R an{}, adot[PM], agh[NBMAX];
#pragma unroll
      for (int k = 0; k < PM; ++k) adot[k] = R{};
#pragma unroll
      for (int g = 0; g < NBMAX; ++g) agh[g] = R{};
      if (warp == 1) {  // copy list: u_{j0+k} into slot k, u_{j0-p+k} into slot PM + k
        const int n = has_known ? 2 * p : p;
        for (int c = lane; c < n; c += 32)
          cp_put(c, c < p ? uslot(j0 + c) : uslot(j0 - p + (c - p)), c < p ? c : PM + (c - p), T);
        if (lane == 0) sh.cp_n = n;
        __syncwarp();
      }
      auto issue = [&](int sb, int64_t r0, int rows) __attribute__((always_inline)) {
        const CsrTile c = csr_tile((int)((r0 - rb) / T), r0, rows, csr_al);
        const unsigned bq = c.ok ? (unsigned)(c.qb - c.qa) : 0u;
        const unsigned brp = c.ok ? (unsigned)c.nrp * 4u : 0u;
        cp_issue(sb, r0, rows, brp + bq * (4u + (unsigned)sizeof(V)));
        unsigned long long* bar = &sh.tbar[sb];
        char* d = reinterpret_cast<char*>(stage(sb));
        if (lane == 0 && brp) bulk_g2s(d + ORP, a.rowptr + r0, brp, bar);
        if (lane == 1 && bq) bulk_g2s(d + OCI, a.colidx + c.qa, bq * 4u, bar);
        if (lane == 2 && bq) bulk_g2s(d + OCV, a.vals + c.qa, bq * (unsigned)sizeof(V), bar);
      };
      auto body = [&](auto gt, const V* tl, int o, int64_t r, int rows) __attribute__((always_inline)) {
        constexpr int GG = decltype(gt)::value;
        constexpr int QC = 8;  // nonzeros of every row of the group fetched together
        constexpr int QH = (PM * sizeof(V) <= 32) ? QC : (PM * sizeof(V) <= 64 ? QC / 2 : 1);  // gathers in flight
        const int64_t r0 = r - o;  // first row of the tile
        const CsrTile c = csr_tile((int)((r0 - rb) / T), r0, rows, csr_al);
        const char* tb = reinterpret_cast<const char*>(tl);
        const int32_t* rps = reinterpret_cast<const int32_t*>(tb + ORP);
        const int32_t* cis = reinterpret_cast<const int32_t*>(tb + OCI);
        const V* cvs = reinterpret_cast<const V*>(tb + OCV);
        int32_t kb[GG + 1];
#pragma unroll
        for (int e = 0; e <= GG; ++e) {
          const int lr = o + e;
          kb[e] = (c.ok && lr < c.nrp) ? rps[lr] : __ldg(a.rowptr + r + e);
        }
        A wk[PM][GG];
#pragma unroll
        for (int k = 0; k < PM; ++k)
#pragma unroll
          for (int e = 0; e < GG; ++e) wk[k][e] = 0;
        int32_t mx = 0;
#pragma unroll
        for (int e = 0; e < GG; ++e) mx = max(mx, kb[e + 1] - kb[e]);
        for (int32_t q0 = 0; q0 < mx; q0 += QC) {
          int32_t ci[GG][QC];
          A cv[GG][QC];
#pragma unroll
          for (int e = 0; e < GG; ++e)
#pragma unroll
            for (int qq = 0; qq < QC; ++qq) {
              const int64_t q = (int64_t)kb[e] + q0 + qq;
              ci[e][qq] = -1;
              cv[e][qq] = 0;
              if (q < kb[e + 1]) {
                if (c.ok && q < c.qb) {
                  ci[e][qq] = cis[q - c.qa];
                  cv[e][qq] = cvs[q - c.qa];
                } else {
                  ci[e][qq] = __ldg(a.colidx + q);
                  cv[e][qq] = ldg_val(a.vals + q);
                }
              }
            }
          // columns whose rows lie in the tile come from the staged copy; the others are gathered
          // from global memory by predicated loads, all issued before any is used (one round trip
          // per row of the group)
#pragma unroll
          for (int e = 0; e < GG; ++e) {
            bool out[QC];
#pragma unroll
            for (int qq = 0; qq < QC; ++qq) {
              const int64_t col = ci[e][qq];
              const uint64_t ct = (uint64_t)(col - r0);
              out[qq] = ci[e][qq] >= 0 && ct >= (uint64_t)rows;
              if (ci[e][qq] >= 0 && ct < (uint64_t)rows) {
#pragma unroll
                for (int k = 0; k < PM; ++k)
                  if (k < p) wk[k][e] = madd(cv[e][qq], tl[k * T + ct], wk[k][e]);
              }
            }
#pragma unroll
            for (int h = 0; h < QC; h += QH) {
              A gv[QH][PM];
#pragma unroll
              for (int qq = 0; qq < QH; ++qq)
#pragma unroll
                for (int k = 0; k < PM; ++k)
                  gv[qq][k] = (out[h + qq] && k < p) ? (A)uk(k)[out[h + qq] ? ci[e][h + qq] : 0] : (A)0;
#pragma unroll
              for (int qq = 0; qq < QH; ++qq) {
                // FP64 and double-word: a slot that no lane of the warp gathers (its column lies in
                // the tile for every lane, or it is padding) would add only zeros; the warp skips it
                // (for a stencil the slots are uniform over the 32 consecutive rows of a warp).  FP32
                // keeps the unconditional form, which measured faster for it
                if constexpr (!std::is_same<V, float>::value) {
                  if (!__any_sync(__activemask(), out[h + qq])) continue;
                }
#pragma unroll
                for (int k = 0; k < PM; ++k)
                  if (k < p) wk[k][e] = madd(cv[e][h + qq], gv[qq][k], wk[k][e]);
              }
            }
          }
        }
        A wp[GG], x[GG];
#pragma unroll
        for (int k = 0; k < PM; ++k) {
          const A sk = sgk(k);
#pragma unroll
          for (int e = 0; e < GG; ++e) wk[k][e] *= sk;
        }
#pragma unroll
        for (int e = 0; e < GG; ++e) wp[e] = wk[0][e];
        const V* sp = tl + o;
        if (has_known) {
#pragma unroll
          for (int k = 0; k < PM; ++k)
            if (k < p) {
              sld<GG>(sp + (PM + k) * T, x);
              const A ck = cAk(k);
#pragma unroll
              for (int e = 0; e < GG; ++e) wp[e] = madd(ck, x[e], wp[e]);
            }
        }
#pragma unroll
        for (int k = 0; k < PM; ++k)
          if (k < p) {
            sld<GG>(sp + k * T, x);
#pragma unroll
            for (int e = 0; e < GG; ++e) dot_add(adot[k], x[e], wp[e]);
          }
#pragma unroll
        for (int g = 0; g < NBMAX; ++g)
          if (gact[g]) {
            vld<GG>(ghostv(g) + r, x);
#pragma unroll
            for (int e = 0; e < GG; ++e) dot_add(agh[g], x[e], wp[e]);
          }
#pragma unroll
        for (int e = 0; e < GG; ++e) dot_add(an, wk[0][e], wk[0][e]);
        vst<GG>(wslot(0) + r, wp);
#pragma unroll
        for (int k = 1; k < PM; ++k)
          if (k < p) vst<GG>(wslot(k) + r, wk[k]);
      };
      tiles<T, G>(issue, body);
#pragma unroll
      for (int k = 0; k < LY::SP_N; ++k) acc[k] = R{};
      acc[LY::SP_NRM] = an;
#pragma unroll
      for (int k = 0; k < PM; ++k) acc[LY::SP_DOT + k] = adot[k];
#pragma unroll
      for (int g = 0; g < NBMAX; ++g) acc[LY::SP_GH + g] = agh[g];
    }
    tick(a.ctl->t_sp);
    if (!reduce(acc, ng > 0 ? LY::SP_GH + ng : LY::SP_GH) || sh.terr) return false;
    tick(a.ctl->t_reduce);
    return true;
  }

  // Streaming part of the fused pass (all warps but the control warp).  EXTRA = false is the
  // common case, compiled without removed-vector terms and with every bench vector staged.
  // Staged slots: w'_j, u_j .. u_{j+p-1}, W_{t+1}, u_{j+1-p} .. u_{j-1}, bench vectors.
  template <bool EXTRA>
  __device__ __forceinline__ bool ba_stream(int j, int t, bool hasA, R (&acc)[LY::BA_N]) {
    constexpr int NSL = 1 + 2 * PM + NBPRE;
    constexpr int T = TL::rows(NSL), G = TL::group(NSL);
    constexpr int SW = 0, SUB = 1, SW1 = 1 + PM, SUA = 2 + PM, SBN = 1 + 2 * PM;
    constexpr int NBA = EXTRA ? NBMAX : NBPRE;  // bench accumulators
    const int nb = a.nbench;
    const int b0 = sh.bench_next;
    const int nbp = min(nb - b0, NBPRE);  // bench vectors staged
    const int ka = max(0, p - j);         // u_{j+1-p+k} exists for k >= ka
    // coefficients (negated: the updates are w + (-h) u) held in registers for p <= 8; larger
    // blocks read them from shared memory where they are used (register budget)
    constexpr bool CREG = PM <= 8;
    A cB[CREG ? PM : 1], cA[CREG ? PM : 1], cgb[NBMAX];
    if constexpr (CREG) {
#pragma unroll
      for (int k = 0; k < PM; ++k) {
        cB[k] = (k < p) ? -ccoefB(k) : (A)0;
        cA[k] = (k < p - 1) ? -ccoefA(k) : (A)0;
      }
    }
    auto coefB = [&](int k) __attribute__((always_inline)) -> A {
      if constexpr (CREG) return cB[k]; else return -ccoefB(k);
    };
    auto coefA = [&](int k) __attribute__((always_inline)) -> A {
      if constexpr (CREG) return cA[k]; else return -ccoefA(k);
    };
    const A cA_last = -ccoefA(p - 1);  // multiplies u_j (negated)
    bool gB[NBMAX], gA[NBMAX];
#pragma unroll
    for (int g = 0; g < NBMAX; ++g) {
      gB[g] = EXTRA && ghost_active(g, j);
      gA[g] = EXTRA && ghost_active(g, j + 1);
      cgb[g] = gB[g] ? -ccgB(g) : (A)0;
    }
    V* wout = uslot(j + p);
    const V* wcur = wslot(t);
    V* wnext = wslot(t + 1 < p ? t + 1 : t);
    R an{}, aw1{}, adot[PM], agr[PM], accb[NBA], agh[EXTRA ? NBMAX : 1];
#pragma unroll
    for (int k = 0; k < PM; ++k) adot[k] = agr[k] = R{};
#pragma unroll
    for (int b = 0; b < NBA; ++b) accb[b] = R{};
#pragma unroll
    for (int g = 0; g < (EXTRA ? NBMAX : 1); ++g) agh[g] = R{};
    if (warp == 1) {  // copy list: w'_j, u_j .. u_{j+p-1}, bench, then (A step) W_{t+1}, u_{j+1-p+k}
      const int n = 1 + p + nbp + (hasA ? p - ka : 0);
      for (int c = lane; c < n; c += 32) {
        if (c == 0) {
          cp_put(c, wcur, SW, T);
        } else if (c <= p) {
          cp_put(c, uslot(j + c - 1), SUB + c - 1, T);
        } else if (c <= p + nbp) {
          cp_put(c, bench(b0 + c - p - 1), SBN + c - p - 1, T);
        } else if (c == p + nbp + 1) {
          cp_put(c, wnext, SW1, T);
        } else {
          const int k = ka + c - (p + nbp + 2);
          cp_put(c, uslot(j + 1 - p + k), SUA + k, T);
        }
      }
      if (lane == 0) sh.cp_n = n;
      __syncwarp();
    }
    auto issue = [&](int sb, int64_t r0, int rows) __attribute__((always_inline)) { cp_issue(sb, r0, rows, 0u); };
    auto body = [&](auto gt, const V* tl, int o, int64_t r, int) __attribute__((always_inline)) {
      constexpr int GG = decltype(gt)::value;
      const V* sp = tl + o;
      // the window slots are re-read from shared memory where they are needed (few live registers)
      A w[GG], x[GG];
      sld<GG>(sp + SW * T, w);
      // B step of j
#pragma unroll
      for (int k = 0; k < PM; ++k)
        if (k < p) {
          sld<GG>(sp + (SUB + k) * T, x);
          const A cb = coefB(k);
#pragma unroll
          for (int e = 0; e < GG; ++e) w[e] = madd(cb, x[e], w[e]);
        }
      if constexpr (EXTRA) {
#pragma unroll
        for (int g = 0; g < NBMAX; ++g)
          if (gB[g]) {
            vld<GG>(ghostv(g) + r, x);
#pragma unroll
            for (int e = 0; e < GG; ++e) w[e] = madd(cgb[g], x[e], w[e]);
          }
      }
      vst<GG>(wout + r, w);
#pragma unroll
      for (int e = 0; e < GG; ++e) dot_add(an, w[e], w[e]);
#pragma unroll
      for (int k = 1; k < PM; ++k)
        if (k < p) {
          sld<GG>(sp + (SUB + k) * T, x);
#pragma unroll
          for (int e = 0; e < GG; ++e) dot_add(agr[k - 1], w[e], x[e]);
        }
#pragma unroll
      for (int b = 0; b < NBPRE; ++b)
        if (b < nbp) {
          sld<GG>(sp + (SBN + b) * T, x);
#pragma unroll
          for (int e = 0; e < GG; ++e) dot_add(accb[b], x[e], w[e]);
        }
      if constexpr (EXTRA) {
#pragma unroll
        for (int b = NBPRE; b < NBMAX; ++b)
          if (b0 + b < nb) {
            vld<GG>(bench(b0 + b) + r, x);
#pragma unroll
            for (int e = 0; e < GG; ++e) dot_add(accb[b], x[e], w[e]);
          }
      }
      // A step of j+1
      if (hasA) {
        A w1[GG];
        sld<GG>(sp + SW1 * T, w1);
#pragma unroll
        for (int e = 0; e < GG; ++e) dot_add(aw1, w1[e], w1[e]);
#pragma unroll
        for (int k = 0; k < PM - 1; ++k)
          if (k < p - 1 && k >= ka) {
            sld<GG>(sp + (SUA + k) * T, x);
            const A ca = coefA(k);
#pragma unroll
            for (int e = 0; e < GG; ++e) w1[e] = madd(ca, x[e], w1[e]);
          }
        sld<GG>(sp + SUB * T, x);
#pragma unroll
        for (int e = 0; e < GG; ++e) w1[e] = madd(cA_last, x[e], w1[e]);
#pragma unroll
        for (int k = 0; k < PM - 1; ++k)
          if (k < p - 1) {
            sld<GG>(sp + (SUB + k + 1) * T, x);
#pragma unroll
            for (int e = 0; e < GG; ++e) dot_add(adot[k], x[e], w1[e]);
          }
#pragma unroll
        for (int e = 0; e < GG; ++e) dot_add(adot[PM - 1], w[e], w1[e]);
        if constexpr (EXTRA) {
#pragma unroll
          for (int g = 0; g < NBMAX; ++g)
            if (gA[g]) {
              vld<GG>(ghostv(g) + r, x);
#pragma unroll
              for (int e = 0; e < GG; ++e) dot_add(agh[g], x[e], w1[e]);
            }
        }
        vst<GG>(wnext + r, w1);
      }
    };
    const bool ok = tiles<T, G>(issue, body);
#pragma unroll
    for (int k = 0; k < LY::BA_N; ++k) acc[k] = R{};
    if constexpr (EXTRA) {
#pragma unroll
      for (int g = 0; g < NBMAX; ++g) acc[LY::BA_GH + g] = agh[g];
    }
    acc[LY::BA_NRM] = an;
    acc[LY::BA_W1] = aw1;
#pragma unroll
    for (int k = 0; k < PM; ++k) acc[LY::BA_DOT + k] = adot[k];
#pragma unroll
    for (int k = 0; k < LY::GR; ++k) acc[LY::BA_GR + k] = agr[k];
#pragma unroll
    for (int v = 0; v < NBMAX; ++v)  // static register indices: acc[BA_BEN + b0 + b] = accb[b]
#pragma unroll
      for (int b = 0; b < NBA; ++b)
        if (b0 + b == v) acc[LY::BA_BEN + v] = accb[b];
    return ok;
  }

  // ---- fused pass of iteration j: B step of j (+ A step of j+1 when hasA) ---------------------
  // B:  w_j = w'_j - sum_{k<p} h_{j+k,j} u_{j+k} - sum_g c_g g   -> raw slot of u_{j+p}
  // A:  w'_{j+1} = W_{t+1} - sum_{i=j+1-p}^{j} h_{j+1,i} u_i (in place), and its inner products
  //     with u_{j+1} .. u_{j+p-1}, with w_j (the future u_{j+p}, unnormalised), with the removed
  //     vectors active at j+1.  Also ||w_j||^2, ||W_{t+1}||^2, w_j . u_{j+k} (Gram entries) and
  //     bench . w_j.  The control warp runs the QR step of iteration qr_j (if > 0) meanwhile.
  __device__ bool pass_ba(int j, int t, bool hasA, int qr_j, int qr_l) {
    R acc[LY::BA_N];  // written after the streaming loop (not live across it)
    int ng = 0;
#pragma unroll
    for (int g = 0; g < NBMAX; ++g)
      if (g < sh.n_ghost) ng = g + 1;
    const int nb = a.nbench;
    if (warp == 0) {
      if (qr_j > 0) qr_warp(qr_j, qr_l);
#pragma unroll
      for (int k = 0; k < LY::BA_N; ++k) acc[k] = R{};
    } else if (ng > 0 || nb - sh.bench_next > NBPRE) {
      ba_stream<true>(j, t, hasA, acc);  // removed vectors active, or many bench vectors
    } else {
      ba_stream<false>(j, t, hasA, acc);
    }
    tick(a.ctl->t_stream);
    const int nv = ng > 0 ? LY::BA_GH + ng : LY::BA_BEN + nb;
    if (!reduce(acc, nv) || sh.terr) return false;  // (sh.terr is read after the reduction's block barrier)
    for (int v = threadIdx.x; v < NVMAX; v += NT) sh.rba[v] = (v < nv) ? sh.red[v] : 0.0;
    __syncthreads();
    tick(a.ctl->t_reduce);
    return true;
  }

  // ---- substitution of a dependent vector (Sec. 5.1) at iteration j ---------------------------
  // When new_ghost >= 0 the removed w_j is kept: its part orthogonal to u_{j-p+1} .. u_{j+p-1} and
  // to the removed vectors active at j, normalised (dropped if nothing is left).  Bench vector bk
  // is orthogonalised (one classical Gram-Schmidt pass) against u_{j-p+1} .. u_{j+p-1} and the
  // removed vectors active at j+1, normalised and stored as u_{j+p}.  Patches the saved A-step
  // values.
  __device__ bool substitute(int j, int t, bool hasA, int bk, int new_ghost) {
    const int tid = threadIdx.x;
    const int cyc = sh.cycle;
    const V* bsrc = bench(bk);
    V* dst = uslot(j + p);
    A sg_new = 0;
    if (new_ghost >= 0) {
      bool gB[NBMAX];
      int ngB = 0;
#pragma unroll
      for (int g = 0; g < NBMAX; ++g) {
        gB[g] = ghost_active(g, j);
        if (gB[g]) ngB = g + 1;
      }
      // G1: inner products of w_j with the window and the removed vectors active at j
      {
        constexpr int NVC = 2 * PM + NBMAX;
        A acc[NVC];
#pragma unroll
        for (int k = 0; k < NVC; ++k) acc[k] = 0;
        for (int64_t r = row0(); r < re; r += NS) {
          A wv = dst[r];
#pragma unroll
          for (int k = 0; k < 2 * PM - 1; ++k)
            if (k < 2 * p - 1 && j - p + 1 + k >= 1) acc[k] += (A)uslot(j - p + 1 + k)[r] * wv;
#pragma unroll
          for (int g = 0; g < NBMAX; ++g)
            if (gB[g]) acc[2 * PM + g] += (A)ghostv(g)[r] * wv;
        }
        if (!reduce(acc, 2 * PM + ngB)) return false;
      }
      A cw[2 * PM], cg[NBMAX];
#pragma unroll
      for (int k = 0; k < 2 * PM; ++k) {
        int i = j - p + 1 + k;
        cw[k] = (k < 2 * p - 1 && i >= 1) ? (A)(sig(i) * sig(i) * sh.red[k]) : (A)0;
      }
#pragma unroll
      for (int g = 0; g < NBMAX; ++g) cg[g] = gB[g] ? (A)sh.red[2 * PM + g] : (A)0;
      __syncthreads();
      // G2: the kept vector (unnormalised) and its squared norm
      {
        A acc[1] = {0};
        for (int64_t r = row0(); r < re; r += NS) {
          A v = dst[r];
#pragma unroll
          for (int k = 0; k < 2 * PM - 1; ++k)
            if (k < 2 * p - 1 && j - p + 1 + k >= 1) v -= cw[k] * (A)uslot(j - p + 1 + k)[r];
#pragma unroll
          for (int g = 0; g < NBMAX; ++g)
            if (gB[g]) v -= cg[g] * (A)ghostv(g)[r];
          ghostv(new_ghost)[r] = (V)v;
          acc[0] += v * v;
        }
        if (!reduce(acc, 1)) return false;
      }
      const double g2 = sh.red[0];
      if (g2 > 0.0 && isfinite(g2)) {
        sg_new = (A)rsqrt(g2);
      } else {  // nothing left to keep
        __syncthreads();
        if (tid == 0) sh.n_ghost = new_ghost;
        __syncthreads();
        new_ghost = -1;
      }
    }
    bool gA[NBMAX];
    int ng = 0;
#pragma unroll
    for (int g = 0; g < NBMAX; ++g) {
      gA[g] = ghost_active(g, j + 1);
      if (g < sh.n_ghost) ng = g + 1;
    }
    // D1: normalise the kept vector; inner products of the bench vector with window and ghosts
    {
      constexpr int NVC = 2 * PM + NBMAX;
      A acc[NVC];
#pragma unroll
      for (int k = 0; k < NVC; ++k) acc[k] = 0;
      for (int64_t r = row0(); r < re; r += NS) {
        A bv = bsrc[r];
        if (new_ghost >= 0) ghostv(new_ghost)[r] = (V)((A)ghostv(new_ghost)[r] * sg_new);
#pragma unroll
        for (int k = 0; k < 2 * PM - 1; ++k)
          if (k < 2 * p - 1 && j - p + 1 + k >= 1) acc[k] += (A)uslot(j - p + 1 + k)[r] * bv;
#pragma unroll
        for (int g = 0; g < NBMAX; ++g)
          if (gA[g]) acc[2 * PM + g] += (A)ghostv(g)[r] * bv;
      }
      if (!reduce(acc, 2 * PM + ng)) return false;
    }
    A cw[2 * PM], cg[NBMAX];
#pragma unroll
    for (int k = 0; k < 2 * PM; ++k) {
      int i = j - p + 1 + k;
      cw[k] = (k < 2 * p - 1 && i >= 1) ? (A)(sig(i) * sig(i) * sh.red[k]) : (A)0;
    }
#pragma unroll
    for (int g = 0; g < NBMAX; ++g) cg[g] = gA[g] ? (A)sh.red[2 * PM + g] : (A)0;
    __syncthreads();
    // D2: the substitute, its norm, its inner products with the remaining bench vectors and with
    //     u_{j+1} .. u_{j+p-1} (Gram entries)
    {
      constexpr int NVC = LY::D2_N;
      A acc[NVC];
#pragma unroll
      for (int k = 0; k < NVC; ++k) acc[k] = 0;
      const int nb = a.nbench;
      for (int64_t r = row0(); r < re; r += NS) {
        A v = bsrc[r];
#pragma unroll
        for (int k = 0; k < 2 * PM - 1; ++k)
          if (k < 2 * p - 1 && j - p + 1 + k >= 1) v -= cw[k] * (A)uslot(j - p + 1 + k)[r];
#pragma unroll
        for (int g = 0; g < NBMAX; ++g)
          if (gA[g]) v -= cg[g] * (A)ghostv(g)[r];
        dst[r] = (V)v;
        acc[LY::D2_NRM] += v * v;
#pragma unroll
        for (int b = 0; b < NBMAX; ++b)
          if (b > bk && b < nb) acc[LY::D2_BEN + b] += (A)bench(b)[r] * v;
#pragma unroll
        for (int k = 1; k < PM; ++k)
          if (k < p) acc[LY::D2_GR + k - 1] += v * (A)uslot(j + k)[r];
      }
      if (!reduce(acc, LY::D2_N)) return false;
    }
    if (tid == 0) {
      double nr2 = sh.red[LY::D2_NRM];
      if (!(nr2 > 0.0) || !isfinite(nr2)) {
        sh.status = ST_ERR_BENCH;
      } else {
        double s = rsqrt(nr2);
        sig(j + p) = s;
        for (int b = bk + 1; b < a.nbench; ++b) set_bc(b, (cyc + 1) & 1, t, s * s * sh.red[LY::D2_BEN + b]);
        for (int k = 1; k < p; ++k) sh.gram[ring2p(j + p)][p - k - 1] = s * sig(j + k) * sh.red[LY::D2_GR + k - 1];
      }
    }
    __syncthreads();
    if (sh.status != ST_OK) return true;
    // D3: inner products of w'_{j+1} with the new u_{j+p} and with the new removed vector
    if (hasA) {
      A acc[2] = {0, 0};
      const V* w1 = wslot(t + 1);
      for (int64_t r = row0(); r < re; r += NS) {
        A x = w1[r];
        acc[0] += (A)dst[r] * x;
        if (new_ghost >= 0) acc[1] += (A)ghostv(new_ghost)[r] * x;
      }
      if (!reduce(acc, 2)) return false;
      if (tid == 0) {
        sh.rba[LY::BA_DOT + PM - 1] = sh.red[0];
        if (new_ghost >= 0) sh.rba[LY::BA_GH + new_ghost] = sh.red[1];
      }
      __syncthreads();
    }
    return true;
  }

  // ---- blocked direction and iterate update for the L iterations of a cycle -----------------
  // m_j = (u_j - sum_{i=j-2p}^{j-1} r_{i,j} m_i) / r_{j,j}   (Eq. (search-dir-comp))
  // X  += sum_l m_{j0+l} z_{j0+l}^T                           (Eq. (approx-update), blocked)
  // bench vectors lose their components along u_{j0} .. u_{j0+p-1} (coefficients of parity cyc).
  __device__ __forceinline__ void set_bc(int b, int par, int l, double v) {
    sh.bc[b][par][l] = v;
    sh.bcc[b][par][l] = to_coef<CT>(v);
  }
  static constexpr bool F64 = std::is_same<V, double>::value;
  __device__ __forceinline__ A ccoefA(int k) const {
    if constexpr (F64) return sh.coefA[k]; else return sh.coefAc[k];
  }
  __device__ __forceinline__ A ccoefB(int k) const {
    if constexpr (F64) return sh.coefB[k]; else return sh.coefBc[k];
  }
  __device__ __forceinline__ A ccgB(int g) const {
    if constexpr (F64) return sh.cgB[g]; else return sh.cgBc[g];
  }
  __device__ __forceinline__ A cdirA(int l) const {
    if constexpr (F64) return sh.dirA[l]; else return sh.dirAc[l];
  }
  __device__ __forceinline__ A cdirB(int l, int q) const {
    if constexpr (F64) return sh.dirB[l][q]; else return sh.dirBc[l][q];
  }
  __device__ __forceinline__ A cZ(int l, int c) const {
    if constexpr (F64) return sh.Zc[l][c]; else return sh.Zcc[l][c];
  }
  __device__ __forceinline__ A cbc(int b, int par, int l) const {
    if constexpr (F64) return sh.bc[b][par][l]; else return sh.bcc[b][par][l];
  }

  // Staged slots: m_{j0-2p} .. m_{j0-1}, u_{j0} .. u_{j0+p-1}, the iterate rows (p values per row,
  // when p * sizeof(V) is a whole number of 16-byte units and X is 16-byte aligned), bench vectors.
  __device__ bool pass_dir(int j0, int L, int cyc, bool update_bench) {
    if (warp > 0) {
      constexpr int NSL = 4 * PM + NBPRE;
      constexpr int T = TL::rows(NSL), G = TL::group(NSL);
      constexpr int SMO = 0, SUV = 2 * PM, SX = 3 * PM, SBN = 4 * PM;
      const int nb = a.nbench, b0 = sh.bench_next;
      const int nbp = update_bench ? min(nb - b0, NBPRE) : 0;
      const int q0 = max(2 * PM - 2 * p, 2 * PM + 1 - j0);  // first window position holding some m_i
      V* mout[PM <= 8 ? PM : 1];  // m_{j0+l} (larger blocks: computed where stored)
      if constexpr (PM <= 8) {
#pragma unroll
        for (int l = 0; l < PM; ++l) mout[l] = mslot(j0 + l);
      }
      const bool xst = ((p * (int)sizeof(V)) % 16 == 0) && ((reinterpret_cast<uintptr_t>(a.X) & 15u) == 0);
      const bool xvec = xst && (p == PM);  // whole-vector iterate stores
      if (warp == 1) {  // copy list: m_{j0-2PM+q} (q >= q0), u_{j0+l}, bench
        const int nm = 2 * PM - q0, n = nm + p + nbp;
        for (int c = lane; c < n; c += 32) {
          if (c < nm)
            cp_put(c, mslot(j0 - 2 * PM + q0 + c), SMO + q0 + c, T);
          else if (c < nm + p)
            cp_put(c, uslot(j0 + c - nm), SUV + c - nm, T);
          else
            cp_put(c, bench(b0 + c - nm - p), SBN + c - nm - p, T);
        }
        if (lane == 0) sh.cp_n = n;
        __syncwarp();
      }
      auto issue = [&](int sb, int64_t r0, int rows) __attribute__((always_inline)) {
        const unsigned bx = xst ? (unsigned)((size_t)rows * p * sizeof(V)) : 0u;
        cp_issue(sb, r0, rows, bx);
        if (lane == 0 && bx) bulk_g2s(stage(sb) + SX * T, a.X + r0 * p, bx, &sh.tbar[sb]);
      };
      auto body = [&](auto gt, const V* tl, int o, int64_t r, int) __attribute__((always_inline)) {
        constexpr int GG = decltype(gt)::value;
        const V* sp = tl + o;
        // p <= 8: the 2p old directions and the p Lanczos rows are held in registers (mw positions
        // 0 .. 2PM-1 old, 2PM .. 3PM-1 new); larger blocks re-read them from the staged tile and
        // hold only the new directions (register budget)
        constexpr bool MREG = PM <= 8;
        constexpr int MO = MREG ? 2 * PM : 0;  // position of m_{j0} in mw
        A mw[MREG ? 3 * PM : PM][GG];
        A uv[MREG ? PM : 1][GG];
        if constexpr (MREG) {
#pragma unroll
          for (int q = 0; q < 2 * PM; ++q)
            if (q >= q0) {
              sld<GG>(sp + (SMO + q) * T, mw[q]);
            } else {
#pragma unroll
              for (int e = 0; e < GG; ++e) mw[q][e] = 0;
            }
#pragma unroll
          for (int l = 0; l < PM; ++l)
            if (l < p) {
              sld<GG>(sp + (SUV + l) * T, uv[l]);
            } else {
#pragma unroll
              for (int e = 0; e < GG; ++e) uv[l][e] = 0;
            }
        }
#pragma unroll
        for (int l = 0; l < PM; ++l) {
          if (l < L) {
            const A ca = cdirA(l);
            A nw[GG];
            if constexpr (MREG) {
#pragma unroll
              for (int e = 0; e < GG; ++e) nw[e] = ca * uv[l][e];
            } else {
              A t[GG];
              sld<GG>(sp + (SUV + l) * T, t);
#pragma unroll
              for (int e = 0; e < GG; ++e) nw[e] = ca * t[e];
            }
#pragma unroll
            for (int q = 0; q < 2 * PM; ++q) {
              const A cb = cdirB(l, q);
              const int pos = l + q;  // window position: < 2PM an old direction, else a new one
              if constexpr (MREG) {
#pragma unroll
                for (int e = 0; e < GG; ++e) nw[e] = madd(cb, mw[pos][e], nw[e]);
              } else if (pos < 2 * PM) {
                if (pos >= q0) {
                  A t[GG];
                  sld<GG>(sp + (SMO + pos) * T, t);
#pragma unroll
                  for (int e = 0; e < GG; ++e) nw[e] = madd(cb, t[e], nw[e]);
                }
              } else {
#pragma unroll
                for (int e = 0; e < GG; ++e) nw[e] = madd(cb, mw[pos - 2 * PM][e], nw[e]);
              }
            }
#pragma unroll
            for (int e = 0; e < GG; ++e) mw[MO + l][e] = nw[e];
            vst<GG>((MREG ? mout[l] : mslot(j0 + l)) + r, nw);
          } else {
#pragma unroll
            for (int e = 0; e < GG; ++e) mw[MO + l][e] = 0;
          }
        }
        // iterate rows r .. r+GG-1 (row-major, p per row)
        if constexpr (std::is_same<V, dw>::value) {  // element by element (no row-block array)
          const V* xsrc = xst ? tl + SX * T + (size_t)o * p : a.X + r * p;
          V* xr = a.X + r * (int64_t)p;
#pragma unroll
          for (int e = 0; e < GG; ++e)
#pragma unroll
            for (int c = 0; c < PM; ++c)
              if (c < p) {
                A s = xsrc[e * p + c];
#pragma unroll
                for (int l = 0; l < PM; ++l)
                  if (l < L) s = madd(mw[MO + l][e], cZ(l, c), s);
                xr[e * p + c] = s;
              }
        } else {
        const V* xsrc = xst ? tl + SX * T + (size_t)o * p : a.X + r * p;
        V* xr = a.X + r * (int64_t)p;
        A xs[GG][PM];
#pragma unroll
        for (int e = 0; e < GG; ++e)
#pragma unroll
          for (int c = 0; c < PM; ++c)
            if (c < p) xs[e][c] = xsrc[e * p + c];
#pragma unroll
        for (int e = 0; e < GG; ++e)
#pragma unroll
          for (int c = 0; c < PM; ++c)
            if (c < p) {
              A s = xs[e][c];
#pragma unroll
              for (int l = 0; l < PM; ++l)
                if (l < L) s = madd(mw[MO + l][e], cZ(l, c), s);
              xs[e][c] = s;
            }
        if (xvec) {  // p == PM: 16-byte stores, flat index f = e * PM + c
          constexpr int W = 16 / sizeof(V);
#pragma unroll
          for (int f0 = 0; f0 < GG * PM; f0 += W) {
            if constexpr (GG * PM % W == 0) {
              V tmp[W];
#pragma unroll
              for (int i = 0; i < W; ++i) tmp[i] = xs[(f0 + i) / PM][(f0 + i) % PM];
              vst<W>(xr + f0, tmp);
            }
          }
          if constexpr (GG * PM % W != 0) {
#pragma unroll
            for (int e = 0; e < GG; ++e)
#pragma unroll
              for (int c = 0; c < PM; ++c) xr[e * PM + c] = xs[e][c];
          }
        } else {
#pragma unroll
          for (int e = 0; e < GG; ++e)
#pragma unroll
            for (int c = 0; c < PM; ++c)
              if (c < p) xr[e * p + c] = xs[e][c];
        }
        }
        if (update_bench) {
#pragma unroll
          for (int b = 0; b < NBMAX; ++b)
            if (b0 + b < nb) {
              A v[GG];
              if (b < NBPRE)
                sld<GG>(sp + (SBN + (b < NBPRE ? b : 0)) * T, v);
              else
                vld<GG>(bench(b0 + b) + r, v);
#pragma unroll
              for (int l = 0; l < PM; ++l)
                if (l < p) {
                  const A cc = cbc(b0 + b, cyc & 1, l);
                  A ul[GG];
                  if constexpr (MREG) {
#pragma unroll
                    for (int e = 0; e < GG; ++e) ul[e] = uv[l][e];
                  } else {
                    sld<GG>(sp + (SUV + l) * T, ul);
                  }
#pragma unroll
                  for (int e = 0; e < GG; ++e) v[e] = madd(-cc, ul[e], v[e]);
                }
              vst<GG>(bench(b0 + b) + r, v);
            }
        }
      };
      tiles<T, G>(issue, body);
    }
    __syncthreads();
    tick(a.ctl->t_dir);
    return sh.terr == 0;  // uniform over the block
  }

  // ---- control warp: coefficients between passes --------------------------------------------
  // Modified Gram-Schmidt coefficients (Algorithm 1 order k = 0..p-1) from classical inner
  // products d_k = u_{first+k} . w:  h_k = d_k - sum_{i<k} h_i (u_{first+k} . u_{first+i}).
  // Lane k holds d_k on entry and h_k on exit (lanes >= p hold 0).
  __device__ double mgs_lanes(double d, int first) {
    const double* g = sh.gram[ring2p(first + (lane < p ? lane : 0))];
    for (int i = 0; i < p - 1; ++i) {
      double hi = __shfl_sync(0xffffffffu, d, i);
      if (lane > i && lane < p) d -= hi * g[lane - i - 1];
    }
    return d;
  }

  // known coefficients of the A step of iteration jn: coefA[k] = h_{jn,i} sigma_i, i = jn-p+k
  __device__ void ctl_coefA(int jn) {
    if (lane < p) {
      const int i = jn - p + lane;
      sh.coefA[lane] = (i >= 1) ? sh.hsub[i % p][jn - i - 1] * sig(i) : 0.0;
      sh.coefAc[lane] = to_coef<CT>(sh.coefA[lane]);
    }
  }

  // results of an A step for iteration jn from raw inner products dr (lane k: raw_{jn+k} . w')
  __device__ void ctl_astep(int jn, double dr) {
    double d = (lane < p) ? sig(jn + (lane < p ? lane : 0)) * dr : 0.0;
    const double h = mgs_lanes(d, jn);
    if (lane < p) {
      if (lane == 0)
        sh.hdiag[jn & 1] = h;
      else
        sh.hsub[jn % p][lane - 1] = h;
      sh.coefB[lane] = h * sig(jn + lane);
      sh.coefBc[lane] = to_coef<CT>(sh.coefB[lane]);
    }
  }

  // after the fused pass of iteration jj (all of warp 0; sh.beta = h_{jj+p,jj} already final)
  __device__ void ctl_after_ba(int jj, int t, bool hasA) {
    const double beta = sh.beta;
    // column jj of H-bar, rows jj-p .. jj+p, for the QR warp (known entries from the C queue)
    for (int k = lane; k <= 2 * p; k += 32) {
      double v;
      if (k < p) {
        const int i = jj - p + k;
        v = (i >= 1) ? sh.hsub[i % p][jj - i - 1] : 0.0;
      } else if (k == p) {
        v = sh.hdiag[jj & 1];
      } else if (k < 2 * p) {
        v = sh.hsub[jj % p][k - p - 1];
      } else {
        v = beta;
      }
      sh.colq[k] = v;
    }
    if (lane == 0) sh.sigq = sig(jj);
    __syncwarp();
    if (lane == 0) sh.hsub[jj % p][p - 1] = beta;  // h_{jj,jj-p} was read above
    if (hasA) {
      const double dr =
          (lane < p - 1) ? sh.rba[LY::BA_DOT + lane] : ((lane == p - 1) ? sh.rba[LY::BA_DOT + PM - 1] : 0.0);
      __syncwarp();
      ctl_astep(jj + 1, dr);
      if (lane < NBMAX) {
        sh.cgB[lane] = (lane < sh.n_ghost) ? sh.rba[LY::BA_GH + lane] : 0.0;
        sh.cgBc[lane] = to_coef<CT>(sh.cgB[lane]);
      }
      if (lane == 0) sh.normAu2[(jj + 1) & 1] = sh.rba[LY::BA_W1];
      __syncwarp();
      if (t + 1 < p - 1) ctl_coefA(jj + 2);
    }
    __syncwarp();
  }

  // ---- band QR step of column j (control warp; FP64) -------------------------------------------
  // Input sh.colq (rows j-p..j+p).  Applies the accumulated rotations of the previous 2p columns,
  // generates the p rotations of column j (pivot row j, zeroing rows j+1..j+p), rotates rows
  // j..j+p of Shat and of the window, records the direction coefficients, z_j and the squared
  // residual norms, and sets qstop: 1 = converged at j, 2 = unusable column (error).
  __device__ __forceinline__ double zval(int j, int c, int k) const {
    const int P2 = 2 * p, P3 = 3 * p;
    if (c < P2) {
      int colid = j + 1 - p + c;
      if (colid == j + p) return (k == p) ? 1.0 : 0.0;
      if (k == p) return 0.0;
      int row = j + k;
      return sh.P[((row % P3) + P3) % P3][((colid % P2) + P2) % P2];
    }
    return sh.Sh[(j + k) % (p + 1)][c - P2];
  }
  __device__ __forceinline__ void zput(int j, int c, int k, double v) {
    const int P2 = 2 * p, P3 = 3 * p;
    const int row = j + k;
    if (c < P2)
      sh.P[((row % P3) + P3) % P3][ring2p(j + 1 - p + c)] = v;
    else
      sh.Sh[row % (p + 1)][c - P2] = v;
  }

  __device__ void qr_warp(int j, int l) {
    const unsigned long long tq = (blockIdx.x == 0 && lane == 0) ? gtimer() : 0ull;
    const int P2 = 2 * p, P3 = 3 * p;
    // 1. y = P col (rows j-2p .. j+p-1), y[3p] = h_{j+p,j}
    for (int a_ = lane; a_ < P3; a_ += 32) {
      const int row = j - P2 + a_;
      const double* Pr = sh.P[((row % P3) + P3) % P3];
      double s0 = 0.0, s1 = 0.0;
      int b = 0;
      for (; b + 1 < P2; b += 2) {
        s0 += Pr[ring2p(j - p + b)] * sh.colq[b];
        s1 += Pr[ring2p(j - p + b + 1)] * sh.colq[b + 1];
      }
      if (b < P2) s0 += Pr[ring2p(j - p + b)] * sh.colq[b];
      sh.y[a_] = s0 + s1;
    }
    if (lane == 0) sh.y[P3] = sh.colq[P2];
    __syncwarp();
    // 2. prefix sums of squares of v = y[2p .. 3p] and the rotations of column j
    //    (rotation k acts on rows j and j+k: c_k = x_{k-1}/x_k, s_k = v_k/x_k, x_0 = v_0)
    if (p <= 31) {
      double v = (lane <= p) ? sh.y[P2 + lane] : 0.0;
      double s = v * v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        double u = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += u;
      }
      if (lane <= p) {
        sh.pref[lane] = s;
        sh.rinv[lane] = (s > 0.0) ? rsqrt(s) : 0.0;
      }
    } else if (lane == 0) {
      double s = 0.0;
      for (int k = 0; k <= p; ++k) {
        double v = sh.y[P2 + k];
        s += v * v;
        sh.pref[k] = s;
        sh.rinv[k] = (s > 0.0) ? rsqrt(s) : 0.0;
      }
    }
    __syncwarp();
    for (int k = lane; k <= p; k += 32) {
      if (k == 0) continue;
      const double xprev = (k == 1) ? sh.y[P2] : sh.pref[k - 1] * sh.rinv[k - 1];
      if (sh.pref[k] > 0.0) {
        sh.gc[k] = xprev * sh.rinv[k];
        sh.gs[k] = sh.y[P2 + k] * sh.rinv[k];
      } else {
        sh.gc[k] = 1.0;
        sh.gs[k] = 0.0;
      }
    }
    __syncwarp();
    // 3. rotate the 3p columns (window columns j+1-p .. j+p, then Shat), one lane per column, in
    //    place: the pivot entry after k rotations is q_k / x_k with q_k = sum_{t<=k} v_t z_t and
    //    x_k = sqrt(pref_k); row j+k becomes -s_k * pivot_{k-1} + c_k * z_k.
    for (int a_ = lane; a_ < P2 - 1; a_ += 32) {  // column j+p of the new window: rows j+1-2p..j-1
      const int row = j + 1 - P2 + a_;
      sh.P[((row % P3) + P3) % P3][ring2p(j + p)] = 0.0;
    }
    for (int c = lane; c < P3; c += 32) {
      const double z0 = zval(j, c, 0);
      double q = sh.y[P2] * z0;
      double piv = z0;
      for (int k = 1; k <= p; ++k) {
        const double zk = zval(j, c, k);
        zput(j, c, k, -sh.gs[k] * piv + sh.gc[k] * zk);
        q += sh.y[P2 + k] * zk;
        piv = (sh.pref[k] > 0.0) ? q * sh.rinv[k] : z0;
      }
      zput(j, c, 0, piv);
    }
    __syncwarp();
    // 4. direction coefficients of Eq. (search-dir-comp), r_jj, z_j, squared residual norms
    //    rho_i^2 = ||Shat(j+1:j+p, i)||^2 (Eq. (comp-resid)) and the stopping decision
    const double rinvp = sh.rinv[p];
    for (int q = lane; q < 2 * PM; q += 32) {
      const int qq = q - (2 * PM - P2);  // R row j-2p+qq
      const double dbq = (qq >= 0 && j - P2 + qq >= 1) ? -sh.y[qq] * rinvp : 0.0;
      sh.dirB[l][q] = dbq;
      sh.dirBc[l][q] = to_coef<CT>(dbq);
    }
    if (lane == 0) {
      sh.rjj[l] = sh.pref[p] * rinvp;
      sh.dirA[l] = sh.sigq * rinvp;
      sh.dirAc[l] = to_coef<CT>(sh.dirA[l]);
    }
    bool conv = true, fin = true;
    if (lane < p) {
      sh.Zc[l][lane] = sh.Sh[j % (p + 1)][lane];
      sh.Zcc[l][lane] = to_coef<CT>(sh.Zc[l][lane]);
      double s = 0.0;
      for (int k = 1; k <= p; ++k) {
        const double v = sh.Sh[(j + k) % (p + 1)][lane];
        s += v * v;
      }
      sh.rho2[lane] = s;
      conv = (s < sh.thr2[lane]) || sh.inv2[lane] == 0.0;
      fin = isfinite(s);
      if (a.rho_hist && blockIdx.x == 0 && j <= a.hist_cap) a.rho_hist[(int64_t)(j - 1) * p + lane] = sqrt(s);
    }
    conv = __all_sync(0xffffffffu, conv);
    fin = __all_sync(0xffffffffu, fin);
    __syncwarp();
    if (lane < p) sh.Sh[j % (p + 1)][lane] = 0.0;  // the ring row of j becomes row j+p+1
    if (lane == 0) {
      const double rjj = sh.rjj[l];
      int st = 0;
      if (!fin || !isfinite(rjj)) {
        st = 2;
        sh.qstatus = ST_ERR_NONFINITE;
      } else if (rjj == 0.0) {
        st = 2;
        sh.qstatus = ST_ERR_BREAKDOWN;
      } else if (conv) {
        st = 1;
      }
      sh.qstop = st;
      if (blockIdx.x == 0) a.ctl->t_qr += gtimer() - tq;
    }
    __syncwarp();
  }

  // ---- the whole solve ------------------------------------------------------------------------
  __device__ void run() {
    const int tid = threadIdx.x;
    Ctl* ctl = a.ctl;
    const unsigned long long t_start = gtimer();
    t_mark = t_start;
    for (int i = tid; i < (int)(sizeof(SHT) / 8); i += NT) reinterpret_cast<double*>(&sh)[i] = 0.0;
    __syncthreads();
    if (tid == 0) {
      for (int k = 0; k < TL::NSTAGE; ++k) mbar_init(&sh.tbar[k], 1);
      fence_mbar_init();
    }
    __syncthreads();
    // the rotation window starts as the identity: P[i][i] = 1 for the columns j-p .. j+p-1 of j = 1
    for (int c = tid; c < 2 * p; c += NT) {
      int i = 1 - p + c;
      sh.P[((i % (3 * p)) + 3 * p) % (3 * p)][ring2p(i)] = 1.0;
    }
    __syncthreads();
    if (!setup_norms()) return fail(t_start);
    {
      bool all_zero = true;
      for (int i = 0; i < p; ++i) all_zero &= (sh.f0n[i] == 0.0);
      if (all_zero) {
        if (blockIdx.x == 0 && tid == 0) {
          ctl->status = ST_OK;
          ctl->iters = 0;
          ctl->t_total = gtimer() - t_start;
        }
        return;
      }
    }
    // ---- initial QR F0 = U_p S with the dependence test of each column ----
    for (int i = 0; i < p && sh.status == ST_OK; ++i) {
      if (!setup_column(i, a.F + (int64_t)i * a.ld, true)) return fail(t_start);
      double nv2 = sh.red[0];
      if (!isfinite(nv2)) {
        set_status(ST_ERR_NONFINITE);
        break;
      }
      const bool dep = !(nv2 > a.gamma * a.gamma * sh.f0n[i] * sh.f0n[i]) || sh.f0n[i] == 0.0;
      if (dep) {
        const int bk = sh.bench_next;
        __syncthreads();
        if (bk >= a.nbench) {
          set_status(ST_ERR_BENCH);
          break;
        }
        if (tid == 0) {
          sh.S[i][i] = 0.0;
          sh.setup_defl++;
          sh.bench_next = bk + 1;
        }
        __syncthreads();
        if (!setup_column(i, bench(bk), false)) return fail(t_start);
        nv2 = sh.red[0];
        if (!(nv2 > 0.0) || !isfinite(nv2)) {
          set_status(ST_ERR_BENCH);
          break;
        }
      } else if (tid == 0) {
        sh.S[i][i] = sqrt(nv2);
      }
      __syncthreads();
      if (tid == 0) {
        const double s = rsqrt(nv2);
        sig(i + 1) = s;
        for (int b = sh.bench_next; b < a.nbench; ++b) set_bc(b, 1, i, s * s * sh.red[1 + b]);
      }
      __syncthreads();
    }
    if (sh.status != ST_OK) return finish(t_start, 0, 0);
    if (a.maxit <= 0) return finish(t_start, 0, 3);  // no iteration allowed: X = X0
    // Shat = [S; 0]: rows 1..p, row p+1 zero (ring index row mod (p+1))
    for (int t = tid; t < p * p; t += NT) {
      int r = t / p, c = t % p;
      sh.Sh[(r + 1) % (p + 1)][c] = sh.S[r][c];
    }
    __syncthreads();

    tabulate_csr_tiles();
    // ---- band iterations, one cycle of p iterations at a time ----
    int cycle = 1;
    bool qr_pending = false;  // QR step of the last iteration of the previous cycle not done yet
    for (;;) {
      const int j0 = (cycle - 1) * p + 1;
      if (warp == 0) {
        if (lane == 0) sh.cycle = cycle;
        ctl_coefA(j0);
      }
      __syncthreads();
      tick(ctl->t_scalar);
      if (!pass_spmm(j0, qr_pending ? j0 - 1 : 0, p - 1)) return fail(t_start);
      if (qr_pending && sh.qstop != 0) {  // the previous cycle ended at its last iteration
        const int L = (sh.qstop == 1) ? p : p - 1;
        return end_cycle(t_start, j0 - p, L, cycle - 1, sh.qstop == 1 ? 1 : 2);
      }
      if (warp == 0) {  // results of the A step of j0, known coefficients of j0+1
        const double dr = (lane < p) ? sh.red[LY::SP_DOT + lane] : 0.0;
        ctl_astep(j0, dr);
        if (lane < NBMAX) {
          sh.cgB[lane] = (lane < sh.n_ghost) ? sh.red[LY::SP_GH + lane] : 0.0;
          sh.cgBc[lane] = to_coef<CT>(sh.cgB[lane]);
        }
        if (lane == 0) sh.normAu2[j0 & 1] = sh.red[LY::SP_NRM];
        __syncwarp();
        if (p > 1) ctl_coefA(j0 + 1);
      }
      __syncthreads();
      if (cycle > 1 && !pass_dir(j0 - p, p, cycle - 1, true)) return fail(t_start);  // previous cycle
      tick(ctl->t_scalar);
      for (int t = 0; t < p; ++t) {
        const int jj = j0 + t;
        const bool hasA = (t < p - 1);
        if (!pass_ba(jj, t, hasA, t > 0 ? jj - 1 : 0, t - 1)) return fail(t_start);
        if (t > 0 && sh.qstop != 0)  // iteration jj-1 ended the solve
          return end_cycle(t_start, j0, sh.qstop == 1 ? t : t - 1, cycle, sh.qstop == 1 ? 1 : 2);
        // ---- norm of the new vector and dependence test (Sec. 5) ----
        const double b2 = sh.rba[LY::BA_NRM];
        if (!isfinite(b2)) {
          set_status(ST_ERR_NONFINITE);
          return end_cycle(t_start, j0, t, cycle, 2);
        }
        const bool dep = !(b2 > a.gamma * a.gamma * sh.normAu2[jj & 1]);
        if (dep) {
          const int bk = sh.bench_next;
          const int ng0 = sh.n_ghost;
          __syncthreads();
          if (bk >= a.nbench) {
            set_status(ST_ERR_BENCH);
            return end_cycle(t_start, j0, t, cycle, 2);
          }
          // a removed vector is kept only for a near-dependence (||w|| > 1e-12 ||A u_jj||); at the
          // rounding level of an exact dependence it carries no direction
          const int newg = (a.ghost && b2 > 1e-24 * sh.normAu2[jj & 1]) ? ng0 : -1;
          if (tid == 0) {
            if (newg >= 0) {
              sh.ghost_born[newg] = jj;
              sh.n_ghost = newg + 1;
            }
            sh.bench_next = bk + 1;
            sh.deflations++;
            sh.beta = 0.0;
          }
          __syncthreads();
          if (!substitute(jj, t, hasA, bk, newg)) return fail(t_start);
          if (sh.status != ST_OK) return end_cycle(t_start, j0, t, cycle, 2);
        } else if (warp == 0) {
          if (lane == 0) {
            const double s = rsqrt(b2);
            sig(jj + p) = s;
            sh.beta = b2 * s;
          }
          __syncwarp();
          const double s = sig(jj + p);
          for (int b = sh.bench_next + lane; b < a.nbench; b += 32)
            set_bc(b, (cycle + 1) & 1, t, s * s * sh.rba[LY::BA_BEN + b]);
          for (int k = 1 + lane; k < p; k += 32)
            sh.gram[ring2p(jj + p)][p - k - 1] = s * sig(jj + k) * sh.rba[LY::BA_GR + k - 1];
        }
        __syncthreads();
        if (warp == 0) ctl_after_ba(jj, t, hasA);
        __syncthreads();
        tick(ctl->t_scalar);
        if (jj >= a.maxit) {  // last permitted iteration: finish its QR step now
          if (warp == 0) qr_warp(jj, t);
          __syncthreads();
          const int L = (sh.qstop == 2) ? t : t + 1;
          return end_cycle(t_start, j0, L, cycle, sh.qstop == 2 ? 2 : (sh.qstop == 1 ? 1 : 3));
        }
      }
      qr_pending = true;
      ++cycle;
    }
  }

  // directions and iterate for the L completed iterations of cycle `cyc` starting at j0; stop:
  // 1 converged, 2 error, 3 iteration limit
  __device__ void end_cycle(unsigned long long t_start, int j0, int L, int cyc, int stop) {
    if (L > 0 && !pass_dir(j0, L, cyc, false)) return fail(t_start);
    finish(t_start, j0 + L - 1, stop);
  }

  __device__ void finish(unsigned long long t_start, int iters, int stop) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      Ctl* ctl = a.ctl;
      int st = sh.status;
      if (st == ST_OK && stop == 2) st = sh.qstatus != 0 ? sh.qstatus : ST_ERR_NONFINITE;
      if (st == ST_OK) st = (stop == 1) ? ST_OK : ST_NOT_CONVERGED;
      ctl->status = st;
      ctl->iters = iters;
      ctl->cycles = iters > 0 ? (iters + p - 1) / p : 0;
      ctl->deflations = sh.deflations;
      ctl->setup_deflations = sh.setup_defl;
      ctl->bench_used = sh.bench_next;
      double worst = 0.0;
      for (int i = 0; i < p; ++i) worst = fmax(worst, sh.rho2[i] * sh.inv2[i]);
      ctl->relres_est_max = sqrt(worst);
      ctl->t_total = gtimer() - t_start;
    }
  }
  __device__ void fail(unsigned long long t_start) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      a.ctl->status = ST_ERR_TIMEOUT;
      a.ctl->t_total = gtimer() - t_start;
    }
  }
};

template <typename V, int PM, int NT>
constexpr size_t solve_smem_bytes() {
  static_assert(Tiles<V, PM, NT>::STG * Tiles<V, PM, NT>::NSTAGE >= (size_t)8 * 16 * (NT - 32), "reduction scratch");
  return Tiles<V, PM, NT>::smem_bytes();
}

template <typename V, int PM, int NT>
__global__ void __launch_bounds__(NT, 1) bminres_solve_kernel(SolveArgs<V> args) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  using SHT = Shared<PM, typename CoefCopy<V>::T>;
  SHT& sh = *reinterpret_cast<SHT*>(smem_raw);
  V* stg = reinterpret_cast<V*>(smem_raw + Tiles<V, PM, NT>::SH);
  Engine<V, PM, NT> e(args, sh, stg);
  e.run();
}

}  // namespace bmr
