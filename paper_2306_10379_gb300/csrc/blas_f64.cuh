// Internal interface of the float64 block kernels (see blas_f64.cu).
#pragma once
#include "common.cuh"

namespace gsi {

struct RowMulArgs {
  int nk;               // number of right-multiplied terms (0..2)
  const double* U[2];   // n x p blocks
  const double* M[2];   // p x p matrices (device)
  double s[2];          // scalars of the product terms
  int ne;               // number of elementwise terms (0..2)
  const double* E[2];   // n x p blocks
  double c[2];          // scalars of the elementwise terms
};

gsi_status spmm_csr(int64_t n, const int64_t* rowptr, const int32_t* colidx, const double* val,
                    int p, const double* X, double* W, cudaStream_t st);
gsi_status spmm_sell(int64_t n, int64_t nchunks, int C, const int64_t* perm,
                     const int64_t* chunk_ptr, const int64_t* chunk_len, const int32_t* scol,
                     const double* sval, int p, const double* X, double* W, cudaStream_t st);
size_t gram_scratch_doubles(int64_t n, int p, int q);
gsi_status gram(int64_t n, int p, int q, const double* U, const double* V, double* G,
                double* scratch, cudaStream_t st);
gsi_status rowmul(int64_t n, int p, const RowMulArgs& a, double* out, cudaStream_t st);
int dots_blocks(int64_t n);
gsi_status dots(int64_t n, int p, int ndots, const double* A0, const double* B0,
                const double* A1, const double* B1, const double* Rnorm, double* out,
                double* scratch, cudaStream_t st);

// dense W = A X (float64), max absolute row sum of a dense A
gsi_status dense_gemm(int64_t n, int p, const double* A, const double* X, double* W, cudaStream_t st);
gsi_status dense_absmax(int64_t n, const double* A, unsigned long long* out, cudaStream_t st);
// out = a W + b Z + e Zp elementwise (Zp may be null)
gsi_status combine3(int64_t count, double a, const double* W, double b, const double* Z, double e,
                    const double* Zp, double* out, cudaStream_t st);
// p x p float64 products over many blocks: out = alpha A B + beta E; out = a X + b Y
gsi_status pp_gemm(int p, double alpha, const double* A, const double* B, double beta,
                   const double* E, double* out, cudaStream_t st);
gsi_status pp_axpby(int p, double a, const double* X, double b, const double* Y, double* out,
                    cudaStream_t st);

// p x p step (small.cu)
size_t small_scratch_doubles(int p);
// mode 0: line search + polar factor (see gsi_linesearch); mode 1: M = S^{-1/2}
// of the symmetric positive definite S given in `B` (start-block orthonormalisation).
gsi_status small_step(int mode, int p, const double* C, const double* B, const double* Gam,
                      const double* Z, const double* XX, const double* XD, double* M,
                      double* out, double* scratch, cudaStream_t st);
// the same step with a float32 Jacobi eigensolver refined in df64 (small_df.cu)
size_t small_df_scratch_bytes(int p);
// modes 3 and 4 split mode 0 in two launches (eigenbasis of B; the rest),
// passing (p + 1) p df64 values through eig_ws
gsi_status small_step_df(int mode, int p, const double* C, const double* B, const double* Gam,
                         const double* Z, const double* XX, const double* XD, double* M,
                         double* out, void* scratch, cudaStream_t st, void* eig_ws = nullptr);
// theta (descending) and U with C = U diag(theta) U^T, C symmetrised first.
gsi_status small_eig(int p, const double* C, double* theta, double* U, double* scratch,
                     cudaStream_t st);

// LOBCG comparator helpers (lobcg.cu)
gsi_status lobcg_coef(int p, const double* theta, const double* U, double tol2, double* M, int* mask,
                      cudaStream_t st);
gsi_status lobcg_mask_gram(int p, double* S, const int* mask, cudaStream_t st);
gsi_status lobcg_assemble(int p, int nb, const double* H11, const double* H12, const double* H13,
                          const double* H22, const double* H23, const double* H33, const int* mask2,
                          const int* mask3, double sentinel, double* H, cudaStream_t st);
gsi_status lobcg_split(int p, int nb, const double* U, double* V1, double* V2, double* V3, cudaStream_t st);

}  // namespace gsi
