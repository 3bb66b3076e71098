/*
 * gsi.h -- C ABI of the GB300 (sm_103a) library for gradient-type subspace
 * iteration: Riemannian steepest descent and conjugate gradients with exact
 * line search for the dominant p-dimensional invariant subspace of a real
 * symmetric matrix A (Alimisis, Saad & Vandereycken, arXiv 2306.10379).
 *
 * Problem statement (Sec. 1 and Sec. 2.1): minimise
 * phi(X) = -1/2 tr(X^T A X) over n x p matrices with X^T X = I; the minimiser
 * spans the eigenvectors of the p largest eigenvalues (the smallest ones are
 * obtained from -A). Each iteration runs Alg. 2 (SD) or Alg. 4 (CG) with the
 * exact line search of Alg. 3 and the one-matvec recursion of Eq.
 * (save_matvec).
 *
 * Conventions shared by every entry point:
 *  - Dense n x p blocks are row-major (the p entries of a row contiguous),
 *    float64. p x p matrices are row-major float64.
 *  - "device" pointers are CUDA global-memory addresses on the current
 *    device; "host" pointers are ordinary host memory.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream). Work is stream-ordered; entry points that return results in
 *    host memory synchronise that stream before returning.
 *  - No entry point throws; each returns a gsi_status. On GSI_ERR_ARG nothing
 *    was launched. On GSI_ERR_CUDA the CUDA error string is available from
 *    gsi_last_error().
 *  - Contexts are not thread-safe; distinct contexts are independent.
 */
#ifndef GSI_H
#define GSI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GSI_OK = 0,
  GSI_ERR_ARG = 1,        /* invalid argument (sizes, null pointers, p range) */
  GSI_ERR_CUDA = 2,       /* a CUDA runtime call failed */
  GSI_ERR_OOM = 3,        /* device allocation failed */
  GSI_ERR_NOCONV = 4,     /* max_iters reached before the tolerance */
  GSI_ERR_BREAKDOWN = 5,  /* a p x p factorisation broke down (rank-deficient block) */
  GSI_ERR_NONFINITE = 6,  /* NaN or Inf met in the iteration */
  GSI_ERR_TIMEOUT = 7     /* a bounded device-side wait expired */
} gsi_status;

typedef enum { GSI_CSR = 0, GSI_SELL = 1, GSI_DENSE = 2 } gsi_format;
/* GSI_CHEB: the Chebyshev-filtered subspace iteration the paper compares
 * against (Alg. 1 with the filter of Eq. (optimal_poly)).
 * GSI_LOBCG: the locally optimal block CG method the paper compares against
 * (Sec. 6.4, Eq. (def_Vk_LOBPCG)) in its LOBCG(+) form: every iteration the
 * Rayleigh-Ritz procedure on span(X_k, G_k, P_k), P_k the part of X_k outside
 * span(X_{k-1}) (the better-conditioned block that replaces X_{k-1}), with
 * each block orthonormalised from its Gram matrix (singular values below
 * 1e-7 of the block's largest dropped) and Q^T A Q formed from explicit
 * products with A Q: three block matvecs per iteration. p <= 64 (the
 * 3p x 3p eigenproblem runs in one thread block in float64). */
typedef enum { GSI_SD = 0, GSI_CG = 1, GSI_CHEB = 2, GSI_LOBCG = 3 } gsi_method;
/* Arithmetic of the n x p block work. GSI_PREC_DF64: blocks stored as
 * float32 pairs (48-bit significand), products on the BF16 tensor cores with
 * error-free digit splitting into 7 digits (float64-class results);
 * GSI_PREC_F64: native float64 on the float64 pipe. GSI_PREC_MIXED: as
 * GSI_PREC_DF64, but the operator apply A X of a dense A uses 3 digits per
 * operand (bf16-level products summed exactly in fp32, ~2^-21 relative) until
 * ||R||_F/anorm <= mixed_switch, then a correction phase with 7-digit applies
 * (explicit AX recomputed, CG restarted) until the tolerance; the residual,
 * the Grams and the retraction stay float64-class throughout, so the errors
 * of the cheap apply scale with ||D|| rather than with ||A X||. The p x p
 * step is float64-class in all modes. */
typedef enum { GSI_PREC_DF64 = 0, GSI_PREC_F64 = 1, GSI_PREC_MIXED = 2 } gsi_precision;

/* Symmetric A. fmt = GSI_CSR / GSI_SELL: full CSR storage (both triangles),
 * rowptr: n+1 int64, colidx: nnz int32 (0-based), val: nnz float64.
 * fmt = GSI_DENSE: val holds the n x n matrix row-major (float64), rowptr,
 * colidx and nnz are ignored; the block matvec is then the dense product
 * A X (computed as A^T X, the contraction over n).
 * on_device = 0: the three arrays are host memory; 1: device memory.
 * fmt = GSI_SELL asks the context to convert A to SELL-C-sigma
 * (chunk height sell_C = 32, sorting window sell_sigma) for its SpMM.
 * Symmetry is not checked. */
typedef struct {
  int32_t fmt;
  int64_t n;
  int64_t nnz;
  const int64_t* rowptr;
  const int32_t* colidx;
  const double* val;
  int32_t sell_C;
  int32_t sell_sigma;
  int32_t on_device;
} gsi_matrix;

typedef struct {
  int32_t method;          /* GSI_SD (Alg. 2), GSI_CG (Alg. 4), GSI_CHEB or GSI_LOBCG */
  int32_t which;           /* +1: largest p eigenvalues; -1: smallest (runs on -A) */
  double tol;              /* stop when ||R||_F / anorm <= tol (default 1e-8) */
  double anorm;            /* ||A||_2 or an upper bound; <= 0: ||A||_inf is used */
  int32_t max_iters;       /* default 10000 */
  int32_t k_restart;       /* CG restart period; 0 = never (default) */
  int32_t recompute_every; /* explicit Y = AX every k iterations; 0 = only when the step is tiny */
  int32_t explicit_ax;     /* 1: explicit AX every iteration ("RCG(+)", Sec. 6.4) */
  int32_t precision;       /* gsi_precision, default GSI_PREC_DF64 */
  /* GSI_CHEB only: filter degree d, the unwanted interval [cheb_lo, cheb_hi]
   * (lambda_n and lambda_{p+1}: c = (lo+hi)/2, h = (hi-lo)/2) and the scaling
   * point cheb_scale (an estimate of lambda_1); one iteration = Rayleigh-Ritz,
   * residual test, d filter matvecs and an orthonormalisation. */
  int32_t cheb_degree;
  double cheb_lo, cheb_hi, cheb_scale;
  double mixed_switch;     /* GSI_PREC_MIXED: residual at which the 7-digit phase starts (1e-5) */
  /* 0 (default): stop when ||R||_F / anorm <= tol; 1: when ||R_k||_inf /
   * ||R_0||_inf <= tol (largest row sum of |R|, the criterion of the paper's
   * Table "Comparison of LOBCG and Riemannian CG"; float32 row sums in df64
   * mode, within (p + 1) 2^-24 relative). The final check is taken with an
   * explicit AX either way. */
  int32_t stop_rule;
  /* GSI_CHEB: 1 = the filter's bounds follow each Rayleigh-Ritz step (the
   * practice the paper notes in Sec. 6.2): the unwanted interval is
   * [cheb_lo, theta_min] and the scaling point theta_max, theta the block's
   * Ritz values; cheb_lo must be a lower bound of the spectrum, cheb_hi and
   * cheb_scale are ignored (GSI_ERR_ARG from the step if theta_min <=
   * cheb_lo). 0 (default) = the fixed interval [cheb_lo, cheb_hi] -- any
   * upper end, e.g. lambda_{p+k} (the remark after Eq. (optimal_poly)). */
  int32_t cheb_adaptive;
  /* GSI_CHEB: guard vectors -- the cheb_guard trailing Ritz pairs (smallest
   * Ritz values) are left out of the stopping test, 0 <= cheb_guard < p
   * (default 0). With cheb_adaptive the filter's upper end theta_min then
   * stays below the wanted eigenvalues. */
  int32_t cheb_guard;
} gsi_opts;

typedef struct {
  int32_t iters;           /* iterations done since gsi_create */
  int32_t matvecs;         /* block matvecs A*Z done since gsi_create */
  int32_t restarts;        /* CG restarts to the gradient direction */
  int32_t brent_evals;     /* phi' evaluations in the last line search */
  int32_t converged;       /* 1 once ||R||_F / anorm <= tol with an explicit AX */
  double rel_residual;     /* ||R||_F / anorm at the last check */
  double rel_residual_inf; /* ||R||_inf / ||R_0||_inf (the paper's table criterion) */
  double trace;            /* tr(X^T A X) at the last check (sign as for A, not -A) */
  double last_step;        /* step t of the last line search */
} gsi_info;

typedef struct gsi_ctx gsi_ctx;

/* Fill *o with the defaults listed above. */
gsi_status gsi_default_opts(gsi_opts* o);

/* Create a solver context on the current device.
 * A: the operator (copied into library-owned device memory; the caller keeps
 *    its arrays). p: block size, 1 <= p <= 128 and n >= 2p.
 * X0: n x p start block (need not be orthonormal); X0_on_device selects host
 *    or device memory. It is copied and orthonormalised by the polar factor
 *    X0 (X0^T X0)^{-1/2}, applied twice.
 * stream: the stream all work of this context is ordered on.
 * Returns GSI_ERR_BREAKDOWN if X0 is numerically rank deficient. */
gsi_status gsi_create(const gsi_matrix* A, int32_t p, const double* X0, int32_t X0_on_device,
                      const gsi_opts* o, void* stream, gsi_ctx** out);

/* Run at most nsteps iterations (stops early on convergence); info may be NULL.
 * Returns GSI_OK (also when converged), or an error status. */
gsi_status gsi_step(gsi_ctx* ctx, int32_t nsteps, gsi_info* info);

/* Iterate until the stopping test of opts.stop_rule holds (checked with an
 * explicit AX; by default ||R||_F/anorm <= tol) or
 * max_iters; GSI_ERR_NOCONV in the latter case, with info filled and the
 * basis retrievable. */
gsi_status gsi_solve(gsi_ctx* ctx, gsi_info* info);

/* Current basis. X: n x p (may be NULL); evals: p Ritz values of A (may be
 * NULL; computed by a Rayleigh-Ritz step with an explicit AX, Eq. (rr1),
 * which also rotates the returned X to the Ritz vectors; descending for
 * which = +1, ascending -- smallest first -- for which = -1, in the order of
 * the columns of X). to_device: 1 if X and evals are device pointers, 0 for
 * host. The context's own iterate is not changed. */
gsi_status gsi_get_basis(gsi_ctx* ctx, double* X, double* evals, int32_t to_device);

/* Restart from a new start block with the same operator, p and options,
 * reusing the context's device memory (X0 as in gsi_create). */
gsi_status gsi_reset(gsi_ctx* ctx, const double* X0, int32_t X0_on_device);

/* ---- complex Hermitian A (the footnote to Eq. (phi)) ----------------------
 * minimise -1/2 Re tr(X^H A X) over X^H X = I: the same Alg. 2 / Alg. 4 on
 * the complex Grassmannian. The library runs it as the real method on the
 * realification [[Ar, -Ai], [Ai, Ar]] (2n x 2n) from the realified start
 * block [[X0r, -X0i], [X0i, X0r]] (2n x 2p): the objective is then twice the
 * complex one, and the gradient, the Polak-Ribiere beta, the exact step and
 * the polar factor all commute with the realification, so the real iterates
 * are the realified complex iterates (the first p columns are [Xr; Xi]). */
typedef struct {
  int64_t n;
  int64_t nnz;
  const int64_t* rowptr;   /* n + 1, 0-based, non-decreasing */
  const int32_t* colidx;   /* nnz */
  const double* val;       /* nnz complex values, interleaved (re, im) */
  int32_t on_device;       /* 0: host arrays, 1: device arrays */
} gsi_zmatrix;

/* Context for a complex Hermitian A (full storage, Hermitian not checked),
 * 1 <= p <= 64, n >= 2p; X0 is n x p complex (interleaved re, im, row-major),
 * host or device by X0_on_device. o: method GSI_SD or GSI_CG (others are
 * GSI_ERR_ARG); the stopping test is on the complex residual ||R||_F / anorm
 * when anorm > 0 is given, else ||.||_inf of the realified operator is used.
 * The inputs are read on the host (device arrays are copied there first) to
 * build the realified CSR with exact zeros dropped. gsi_step, gsi_solve,
 * gsi_reset (with a realified 2n x 2p start block), gsi_destroy apply as for
 * a real context; gsi_info's trace is the complex objective's
 * tr(X^H A X), its residuals those of the complex iterate (the infinity norm
 * of the realified rows). */
gsi_status gsi_create_hermitian(const gsi_zmatrix* A, int32_t p, const double* X0, int32_t X0_on_device,
                                const gsi_opts* o, void* stream, gsi_ctx** out);
/* Basis of a Hermitian context: X (n x p complex, interleaved; may be NULL)
 * the current iterate -- orthonormal, not rotated to Ritz vectors -- and
 * evals (p, may be NULL) its Ritz values (explicit AX; descending for
 * which = +1, ascending for -1). to_device: 1 if X and evals are device
 * pointers. GSI_ERR_ARG for a context not made by gsi_create_hermitian. */
gsi_status gsi_get_basis_hermitian(gsi_ctx* ctx, double* X, double* evals, int32_t to_device);

/* Subspace tracking (Sec. 1: eigenspaces of a slowly varying matrix, as in
 * self-consistent-field iterations). Replaces the context's operator by A --
 * same format and n as at gsi_create; nnz may change (the buffers are
 * reallocated) -- and makes the current iterate X the start block of the new
 * problem: X is orthonormalised again, Y = A X is formed, the iteration
 * counters and the CG state (direction, previous residual) start afresh.
 * anorm > 0 sets the bound of the stopping test; otherwise the one given in
 * gsi_create's options is kept, or ||A||_inf of the new A is used if none
 * was given. A is copied as in gsi_create (host or device arrays by
 * A->on_device; the caller keeps them). GSI_ERR_ARG if the format or n
 * differ. */
gsi_status gsi_set_operator(gsi_ctx* ctx, const gsi_matrix* A, double anorm);

/* Device pointers of the context's current iterate X and Y = AX (n x p
 * row-major; float64 for GSI_PREC_F64, df64 pairs for GSI_PREC_DF64), valid
 * until the next call on ctx. For tests and benchmarks. */
gsi_status gsi_state_ptrs(gsi_ctx* ctx, void** X, void** Y);

/* Bounded device waits (no counterpart in the paper). The tensor-core
 * kernels wait on their own products with an iteration limit instead of
 * spinning without end; a wait that runs out drains the tensor core (every
 * product already issued completes before the kernel releases its tensor
 * memory and returns), leaves non-finite outputs and adds one to a
 * process-wide count. gsi_solve, gsi_step, gsi_reset and gsi_create then
 * return GSI_ERR_TIMEOUT instead of the status the non-finite values would
 * cause.
 * gsi_set_wait_limit: polls allowed to each wait on a batch of products,
 *   0 .. 2^24, on the current device; a negative value restores the default
 *   2^24. The drain itself always allows 2^24 polls. A small limit forces
 *   the timeout path (tests); the default is far above any product's
 *   latency.
 * gsi_device_timeouts: the current device's count of waits that ran out
 *   since the library was loaded (synchronises the legacy default stream). */
gsi_status gsi_set_wait_limit(int32_t polls);
gsi_status gsi_device_timeouts(int64_t* count);

/* Kernel classes for gsi_profile_read. */
typedef enum {
  GSI_K_SPMM = 0,      /* block matvec A*Z */
  GSI_K_GRAM = 1,      /* Gram products U^T V */
  GSI_K_BLOCKMUL = 2,  /* n x p blocks times p x p matrices, fused elementwise terms */
  GSI_K_SMALL = 3,     /* p x p step: eigensolver, line search, polar normaliser */
  GSI_K_REDUCE = 4,    /* norms */
  GSI_K_COUNT = 5
} gsi_kernel_class;

/* on != 0: record CUDA events around every kernel group this context launches
 * (on its stream) and accumulate per-class device time; resets the totals. */
gsi_status gsi_profile_enable(gsi_ctx* ctx, int32_t on);
/* Totals since gsi_profile_enable for class k: launch groups, device ms, and
 * the algorithmic bytes / flops of those launches (float64-equivalent:
 * 8 bytes per block entry, 12 bytes per nonzero, 2 flops per multiply-add). */
gsi_status gsi_profile_read(gsi_ctx* ctx, int32_t k, int64_t* launches, double* total_ms,
                            double* alg_bytes, double* alg_flops);
/* Number of kernels this library has launched in this process. */
int64_t gsi_launch_count(void);

gsi_status gsi_destroy(gsi_ctx* ctx);

const char* gsi_status_str(gsi_status s);
/* Text of the last CUDA error seen by this library (thread-local). */
const char* gsi_last_error(void);

/* ------------------------------------------------------------------------
 * Kernel-level entry points. All pointers are device pointers unless noted.
 * They expose the steps of one iteration for parity tests and benchmarks.
 * ---------------------------------------------------------------------- */

/* One block matvec W = A X (Sec. 6.1, "Efficient matvecs"): CSR A (n rows),
 * X and W n x p. */
gsi_status gsi_spmm_csr(int64_t n, const int64_t* rowptr, const int32_t* colidx,
                        const double* val, int32_t p, const double* X, double* W,
                        void* stream);

/* SELL-C-sigma layout of a CSR matrix, built on the host (all pointers host).
 * Rows are sorted by nnz descending (ties: ascending row index) inside each
 * window of sigma rows; chunks of C consecutive permuted rows are stored
 * column-major with the chunk's longest row as width; padding entries have
 * column = own row (0 for padding rows) and value 0.
 * Query sizes with gsi_sell_size(), then fill:
 *   perm[nchunks*C] (original row of each permuted slot, -1 = padding),
 *   chunk_ptr[nchunks+1] (start of each chunk in the entry arrays),
 *   chunk_len[nchunks], sell_col[total], sell_val[total]. */
gsi_status gsi_sell_size(int64_t n, const int64_t* rowptr, int32_t C, int32_t sigma,
                         int64_t* nchunks, int64_t* total);
gsi_status gsi_csr_to_sell(int64_t n, const int64_t* rowptr, const int32_t* colidx,
                           const double* val, int32_t C, int32_t sigma, int64_t* perm,
                           int64_t* chunk_ptr, int64_t* chunk_len, int32_t* sell_col,
                           double* sell_val);

/* Diagonal layout of a CSR matrix whose nonzeros lie on at most max_diags
 * diagonals (finite-difference stencils; host arrays): *ndiag = the number
 * of distinct offsets col - row, or 0 if there are more than max_diags
 * (then nothing else is written). offsets (ndiag int64, ascending) and dia
 * (n x ndiag float64, row-major: dia[r ndiag + d] = A[r, r + offsets[d]], 0
 * where A has no entry) are written if not NULL. Call with NULL arrays to
 * size them. */
gsi_status gsi_csr_to_dia(int64_t n, const int64_t* rowptr, const int32_t* colidx, const double* val,
                          int32_t max_diags, int32_t* ndiag, int64_t* offsets, double* dia);

/* W = A X (Sec. 6.1, one block matvec) for a stencil-shaped A in the
 * diagonal layout of gsi_csr_to_dia: ndiag <= 8 ascending offsets (a host
 * array; at most two of them beyond 64 q rows, q the largest window that
 * fits shared memory for p columns), dia n x ndiag df64 values (2 n ndiag
 * floats, device), X and W n x p df64 (device), even p <= 64, 16-byte
 * aligned. A CTA walks
 * 64-row tiles keeping X's tiles k - q .. k + q in shared memory, filled by
 * cp.async one tile ahead; the far offsets are read from global memory.
 * Diagonals are summed in ascending offset order: for sorted CSR rows the
 * result equals gsi_df_spmm_csr's bit for bit. GSI_ERR_ARG if the shape does
 * not apply. */
gsi_status gsi_df_spmm_dia(int64_t n, int32_t ndiag, const int64_t* offsets, const float* dia, int32_t p,
                           const float* X, float* W, void* stream);

/* W = A X with A in SELL-C-sigma (device arrays from gsi_csr_to_sell).
 * W rows are written at their original (unpermuted) positions. */
gsi_status gsi_spmm_sell(int64_t n, int64_t nchunks, int32_t C, const int64_t* perm,
                         const int64_t* chunk_ptr, const int64_t* chunk_len,
                         const int32_t* sell_col, const double* sell_val, int32_t p,
                         const double* X, double* W, void* stream);

/* Tall-skinny Gram G = U^T V (Eq. (gradPhi) C = X^T A X; Eqs. (diags),
 * (CG_linesearch_D)); U n x p, V n x q (row-major), G p x q.
 * Uses a temporary device buffer for per-block partial sums (stream-ordered
 * allocation on `stream`). */
gsi_status gsi_gram(int64_t n, int32_t p, int32_t q, const double* U, const double* V,
                    double* G, void* stream);

/* Residual R = Y - X C (Eq. (gradPhi), sign flipped: R = -grad phi);
 * X, Y, R n x p, C p x p. R may alias Y. */
gsi_status gsi_residual(int64_t n, int32_t p, const double* X, const double* Y,
                        const double* C, double* R, void* stream);

/* The p x p part of one iteration (Alg. 3 and Eqs. (Gdec)-(xii), (phi_P),
 * (deriv_P), (derv1)-(derv2)): diagonalise B = D^T D = V diag(beta) V^T,
 * form alpha, gamma, zeta = diag(V^T {C, Gamma, Z} V), find the exact step t
 * by Brent on phi'(t), then M = S^{-1/2} with
 * S = XX + t (XD + XD^T) + t^2 B, the measured Gram of X + tD.
 * Inputs (device, p x p): C = X^T Y, B = D^T D, Gam = D^T W, Z = D^T R,
 * XX = X^T X, XD = X^T D. Outputs (device): M (p x p) and out (16 doubles):
 * out[0..4] = {t, phi(t) model value, phi' evaluations, status, max beta_i};
 * status 0 = ok, 5 = S not positive definite; out[5..15] are diagnostics
 * (cycle counts and sweep counts of the phases). precision: GSI_PREC_DF64 finds the eigenbasis
 * with a float32 Jacobi method refined in df64 and forms M by a first-order
 * expansion in that basis; GSI_PREC_F64 runs a float64 Jacobi method for B
 * and for S. */
gsi_status gsi_linesearch(int32_t p, const double* C, const double* B, const double* Gam,
                          const double* Z, const double* XX, const double* XD, double* M,
                          double* out, int32_t precision, void* stream);

/* Retraction with the AX recursion (Eqs. (Ynew), (save_matvec)):
 * X <- (X + t D) M, Y <- (Y + t W) M, in place. */
gsi_status gsi_retract(int64_t n, int32_t p, double t, const double* M, double* X,
                       const double* D, double* Y, const double* W, void* stream);

/* ------------------------------------------------------------------------
 * df64 kernels. A df64 array holds each value as two float32 (hi, lo),
 * interleaved (value i at [2i], [2i+1]), hi + lo exact, |lo| <= ulp(hi)/2:
 * a 48-bit significand. The solver stores every n x p block this way and
 * computes its block products with float64-accurate (error-free split)
 * products on the BF16 tensor cores.
 * ---------------------------------------------------------------------- */

/* W = A X in df64 (Sec. 6.1, one block matvec): CSR A with df64 values
 * (val: 2*nnz floats), X and W n x p df64. */
gsi_status gsi_df_spmm_csr(int64_t n, const int64_t* rowptr, const int32_t* colidx,
                           const float* val, int32_t p, const float* X, float* W, void* stream);

/* OUT = s0 U0 M0 (+ s1 U1 M1 if nk = 2) (+ c0 E0) (+ c1 E1): n x p df64 blocks
 * U*, E*, OUT; M* float64 p x p; c* df64 scalars given as (hi, lo) float
 * pairs (c: 4 floats, c0 then c1). ne = number of E terms (0..2). The
 * products are exact up to the 49-bit digit truncation of the operands
 * (relative error about 2^-45 of sum |U||M|), i.e. float64-class; this is
 * the right multiplication of Eqs. (gradPhi) (R = Y - XC), (Pnew) and
 * (Ynew)/(save_matvec). OUT may alias an E; it may alias a U only if p <= 64.
 * Uses temporary device memory (stream-ordered allocation). */
gsi_status gsi_oz_gemm(int64_t n, int32_t p, int32_t nk, const float* U0, const float* U1,
                       const double* M0, const double* M1, double s0, double s1, int32_t ne,
                       const float* E0, const float* E1, const float* c, float* OUT,
                       void* stream);

/* G = U^T V (float64 p x q) from n x p and n x q df64 blocks, float64-class
 * accurate (the Gram products of Eqs. (gradPhi), (diags), (CG_linesearch_D)).
 * sym = 1 requires U == V and computes only the upper half. Uses temporary
 * device memory (stream-ordered allocation). */
gsi_status gsi_oz_gram(int64_t n, int32_t p, int32_t q, const float* U, const float* V,
                       int32_t sym, double* G, void* stream);

/* Dense block matvec W = A X for a symmetric n x n A (df64, row-major),
 * computed as A^T X with the contraction over n cut into 64-row chunks, each
 * chunk's digit products exact on the tensor cores. nd = 7: float64-class;
 * nd = 3: bf16-level products (the mixed-precision iterations). X and W are
 * n x p df64 (p <= 128). Uses temporary device memory (stream-ordered). */
gsi_status gsi_oz_dense_apply(int64_t n, int32_t p, const float* A, const float* X, float* W,
                              int32_t nd, void* stream);

/* Allocation-free variant of gsi_oz_gram (no counterpart in the paper).
 * For callers that may not allocate device memory when they call in: code
 * recorded into a CUDA graph whose memory pool the caller does not own,
 * real-time or embedded hosts that forbid allocation after start-up, and
 * threads without access to the process's allocator. Arguments and result
 * are those of gsi_oz_gram. The per-block partial sums use one static device
 * array of 8 MiB, which every GPU that loads this library keeps until the
 * process exits; calls whose partials would exceed it (more than 256 SMs)
 * return GSI_ERR_ARG with a message in gsi_last_error(). The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture. The
 * looked-up address is kept for the life of the process, so the device's
 * primary context must not be reset (cudaDeviceReset) between calls. Every
 * call shares the array and overwrites it (it is cleared on each call), so
 * calls whose work overlaps on the GPU -- on different streams, or from
 * different threads -- race; serialise them. No cudaMalloc, cudaFree or
 * allocating library routine is called. */
gsi_status gsi_oz_gram_noalloc(int64_t n, int32_t p, int32_t q, const float* U, const float* V,
                               int32_t sym, double* G, void* stream);

/* Which tensor-core kernels the digit-split products use: 0 (default) and 2
 * the tcgen05 kernels wherever they apply (7-digit Grams of any p, q and
 * the 7-digit dense apply, one CTA per 64 x 64 output block; 3-digit Grams
 * and the 3-digit dense apply on 16-byte aligned blocks of even width;
 * 7-digit block products of any p <= 128, the contraction cut into slices
 * of at most 64 for p > 64), 1 the mma.sync kernels everywhere (they also
 * serve the remaining 3-digit products). Block products with p <= 64 are
 * identical on both (same digits, exact integer digit-pair sums, same
 * combination order); for p > 64 the tcgen05 slices take their own digit
 * exponents and are summed in df64, so the two agree to df64 rounding but
 * not bit for bit. Grams agree to float64-class accuracy but not bit for
 * bit: the tcgen05 Grams take their column exponents over 512-row (U == V)
 * or 384-row chunks (aligned blocks of at most 64 columns, and 3 digits) or
 * over 256-row (U == V) or 160-row chunks (the others), the mma.sync Gram
 * over 64-row chunks. The switch exists to compare them.
 * Process-wide; the environment variable GSI_TENSOR_PATH=mma or =tcgen05
 * selects 1 or 2 before the first product. */
gsi_status gsi_set_tensor_path(int32_t path);
int32_t gsi_tensor_path(void);

/* Measured multiply-add throughput of this GPU (no counterpart in the paper;
 * the denominators behind the choice of df64 and tensor-core digits):
 * out[0] = float64 FMA TFLOP/s, out[1] = float32 FMA TFLOP/s, each the best
 * of three ~50 ms launches of 8 independent FMA chains per thread over
 * 8 blocks per SM (2 flops per FMA). out: 2 host doubles. Allocates and
 * frees a small device buffer on `stream`; synchronises it. */
gsi_status gsi_measure_fma_peaks(double* out, void* stream);

/* ---- batched solver -------------------------------------------------------
 * Many independent problems, each the dominant p_i-dimensional invariant
 * subspace of a symmetric A_i (the problem of Sec. 2.1), iterated together
 * by Alg. 2 (SD) or Alg. 4 (CG) with the exact line search of Alg. 3 and the
 * recursion of Eq. (save_matvec) -- the same iteration as gsi_solve, with
 * every decision taken on the GPU. Block data are df64; operator entries
 * float32; the p x p step float64. The paper solves one problem at a time;
 * batching is a GPU execution form of the same method. */
typedef struct gsi_batch gsi_batch;

/* The tile table of one pass (host-only, no GPU needed): the problems with
 * active[i] != 0 (all when active is NULL), in the order descending p, then
 * descending n, then ascending index, each cut into tiles of
 *   T_i = min(tile_max, max(64, ceil(S / target_tiles)))
 * rows (the last one ragged), S the rows of all selected problems: tiles of
 * tile_max rows while many problems are active, finer ones when few remain.
 * The device builds the same table at the start of every pass from the
 * problems still active. Tile k covers rows [tile_row0[k], tile_row0[k] +
 * tile_rows[k]) of problem tile_prob[k]. order: nprob entries or NULL;
 * ntiles: required; the three tile arrays may be NULL, else hold capacity
 * entries (GSI_ERR_ARG if fewer than ntiles). */
gsi_status gsi_batched_plan(int32_t nprob, const int32_t* n, const int32_t* p, const int32_t* active,
                            int32_t tile_max, int32_t target_tiles, int32_t* order, int32_t* ntiles,
                            int32_t* tile_prob, int32_t* tile_row0, int32_t* tile_rows,
                            int32_t capacity);

/* Create a batch (host inputs, copied; the caller keeps ownership).
 *   n[i], p[i]: size and block width of problem i; p[i] in {2, 4, 8, 16, 32},
 *     n[i] >= 2 p[i].
 *   rowptr, colidx, val: one concatenated CSR: rows of problem i are rows
 *     n[0] + ... + n[i-1] onwards; rowptr has sum(n) + 1 non-decreasing
 *     entries starting at 0 and indexes colidx/val globally; column indices
 *     are local to the problem (0 <= c < n[i], checked); A_i symmetric (not
 *     checked); values float32.
 *   X0: concatenated row-major n[i] x p[i] float64 start blocks (need not
 *     be orthonormal); kept for gsi_batched_reset.
 *   anorm: NULL, or per-problem ||A_i|| for the stopping test (entries <= 0
 *     fall back to o->anorm, then to ||A_i||_inf).
 *   o: method GSI_SD or GSI_CG, which, tol, max_iters, k_restart,
 *     recompute_every, explicit_ax are used; NULL = defaults.
 * The start blocks are orthonormalised and Y = A X formed before return.
 * Errors: GSI_ERR_ARG for invalid sizes or indices, GSI_ERR_OOM / CUDA. */
gsi_status gsi_batched_create(int32_t nprob, const int32_t* n, const int32_t* p,
                              const int64_t* rowptr, const int32_t* colidx, const float* val,
                              const double* X0, const double* anorm, const gsi_opts* o,
                              void* stream, gsi_batch** out);
/* Tile shape: tile_max rows (32..65536), persistent CTAs per SM (1..32) of
 * the tile kernels, tiles aimed at per CTA (1..64; target_tiles = CTAs x
 * tiles_per_cta); restarts the batch from X0. */
gsi_status gsi_batched_set_tiles(gsi_batch* b, int32_t tile_max, int32_t ctas_per_sm,
                                 int32_t tiles_per_cta);
/* Current tile shape and the persistent grid size. Outputs may be NULL. */
gsi_status gsi_batched_get_tiles(gsi_batch* b, int32_t* tile_max, int32_t* ctas_per_sm,
                                 int32_t* tiles_per_cta, int32_t* grid);
/* The tile table the device built for the last pass (copied to host
 * arrays of capacity entries; NULL arrays skipped). */
gsi_status gsi_batched_last_plan(gsi_batch* b, int32_t* ntiles, int32_t* tile_prob,
                                 int32_t* tile_row0, int32_t* tile_rows, int32_t capacity);
/* Autotuner: times npasses passes from the start for every candidate tile
 * shape (tile_max 256..4096, 2/4/8 CTAs per SM, 1/2 tiles per CTA), keeps
 * the fastest and restarts the batch from X0. Outputs may be NULL. */
gsi_status gsi_batched_tune(gsi_batch* b, int32_t npasses, int32_t* tile_max, int32_t* ctas_per_sm,
                            int32_t* tiles_per_cta, double* ms_per_pass);
/* Back to the orthonormalised X0. */
gsi_status gsi_batched_reset(gsi_batch* b);
/* Run npasses passes from the host (a pass is one iteration of every active
 * problem, or the explicit AX of a problem that is about to stop). */
gsi_status gsi_batched_step(gsi_batch* b, int32_t npasses);
/* Run until every problem has stopped. use_graph != 0: one launch of a CUDA
 * graph whose while-node repeats the pass until no problem is active (or
 * 2 max_iters + 4 passes); use_graph == 0: the same passes from a host loop.
 * passes (may be NULL): passes run. GSI_OK if every problem converged, else
 * GSI_ERR_NOCONV (per-problem status from gsi_batched_info). */
gsi_status gsi_batched_solve(gsi_batch* b, int32_t use_graph, int32_t* passes);
/* Per-problem counters as gsi_info (trace = tr(X^T A X)); status: -1 while
 * active, else GSI_OK (converged), GSI_ERR_NOCONV, GSI_ERR_BREAKDOWN or
 * GSI_ERR_NONFINITE. Either output may be NULL. */
gsi_status gsi_batched_info(gsi_batch* b, int32_t i, gsi_info* info, int32_t* status);
/* Problem i's basis into host X (n[i] x p[i] row-major float64) and, if evals
 * is not NULL, its Ritz values (p[i], descending) with X then the Ritz
 * vectors (Eq. (rr1), explicit AX; computed for all problems at once and
 * kept until the next pass). Either output may be NULL. */
gsi_status gsi_batched_get_basis(gsi_batch* b, int32_t i, double* X, double* evals);
gsi_status gsi_batched_destroy(gsi_batch* b);

/* New start blocks (concatenated as in gsi_batched_create; host or device
 * float64 by on_device), kept as the batch's X0; orthonormalised, Y = A X. */
gsi_status gsi_batched_restart(gsi_batch* b, const double* X0, int32_t on_device);

/* ---- learned warm start ----------------------------------------------------
 * A multilayer perceptron din -> hidden -> hidden -> dout (ReLU, ReLU,
 * linear) maps the coefficients of an operator of a family to a coarse basis
 * C (m x p, dout = m p, row-major); the start block is its prolongation
 * P C. The paper motivates warm starts from related problems (Sec. 1) but
 * prints no network: these entry points are the project's. All pointers
 * below are device pointers unless stated; work is ordered on `stream`. */
typedef struct gsi_mlp gsi_mlp;

/* Parameters in one float32 vector: W1 (hidden x din), b1, W2 (hidden x
 * hidden), b2, W3 (dout x hidden), b3, row-major. */
int64_t gsi_mlp_num_params(int32_t din, int32_t hidden, int32_t dout);
/* params: host float32, copied. max_batch: largest batch of later calls. */
gsi_status gsi_mlp_create(int32_t din, int32_t hidden, int32_t dout, int32_t max_batch,
                          const float* params, void* stream, gsi_mlp** out);
/* Current parameters and last gradients into host arrays (either NULL). */
gsi_status gsi_mlp_get_params(gsi_mlp* n, float* params, float* grads);
/* out (batch x dout) = MLP(x (batch x din)); products on the tensor cores
 * with bfloat16 operands and float32 sums; keeps the activations for the
 * next gsi_mlp_backward. */
gsi_status gsi_mlp_forward(gsi_mlp* n, int32_t batch, const float* x, float* out);
/* Gradients of sum(out * dout) for the last forward's batch (same x),
 * stored in the context (overwritten). */
gsi_status gsi_mlp_backward(gsi_mlp* n, int32_t batch, const float* x, const float* dout);
/* One Adam step (Kingma & Ba 2015) with the stored gradients. */
gsi_status gsi_mlp_adam(gsi_mlp* n, double lr, double beta1, double beta2, double eps);
/* Per sample s of a batch: C = C[s], Bt = Bt[s] (m x p float32, consecutive
 * samples m p apart), S = P^T P (m x m CSR, float64 values): N = C^T S C,
 * Q = C^T Bt Bt^T C, loss[s] = p - tr(N^{-1} Q) (the sum of sin^2 of the
 * principal angles between span(P C) and span(U) when Bt = P^T U, U
 * orthonormal), dC[s] = gscale * dloss/dC = -2 gscale [Bt Bt^T C N^{-1} -
 * S C N^{-1} Q N^{-1}]. SC_scratch: batch m p floats. loss float64; NaN
 * (and dC = 0) where N is not positive definite. p <= 64. */
gsi_status gsi_warm_loss_grad(int32_t batch, int32_t m, int32_t p, const int64_t* S_rowptr,
                              const int32_t* S_colidx, const double* S_val, const float* C,
                              const float* Bt, float* SC_scratch, double* loss, float* dC, float gscale,
                              void* stream);
/* forward, mean loss gradient over the batch, backward, Adam (0.9, 0.999,
 * 1e-8); mean_loss (host, may be NULL) is the batch's mean loss before the
 * step. dout of the network must equal m p. */
gsi_status gsi_warm_train_step(gsi_mlp* n, int32_t batch, const float* x, int32_t m, int32_t p,
                               const int64_t* S_rowptr, const int32_t* S_colidx, const double* S_val,
                               const float* Bt, double lr, double* mean_loss);
/* X[s] = P C[s]: bilinear prolongation from nc x nc interior coarse nodes
 * at (a+1)/(nc+1) to nf x nf fine nodes at (i+1)/(nf+1) of the unit square
 * with zero boundary values; node (i, j) is row i + nf j. C float32
 * (batch x nc^2 x p), X float64 (batch x nf^2 x p). */
gsi_status gsi_prolong(int32_t nc, int32_t nf, int32_t p, int32_t batch, const float* C, double* X,
                       void* stream);
/* Bt[s] = P^T U[s] (the transpose of gsi_prolong): U float64, Bt float32. */
gsi_status gsi_restrict(int32_t nc, int32_t nf, int32_t p, int32_t batch, const double* U, float* Bt,
                        void* stream);
/* C = alpha op(A) op(B) + beta C (+ bias[j]), then C = 0 where
 * mask[i][j] <= 0 (mask may be NULL), then ReLU if relu: A(i,k) =
 * A[i sai + k sak], B(k,j) = B[k sbk + j sbj], C[i ldc + j]; float32 in
 * and out, operands rounded to bfloat16, float32 sums (tensor cores). */
gsi_status gsi_gemm_bf16(int32_t M, int32_t N, int32_t K, const float* A, int64_t sai, int64_t sak,
                         const float* B, int64_t sbk, int64_t sbj, float* C, int64_t ldc, float alpha,
                         float beta, const float* bias, const float* mask, int32_t relu, void* stream);
gsi_status gsi_mlp_destroy(gsi_mlp* n);

#ifdef __cplusplus
}
#endif
#endif /* GSI_H */
