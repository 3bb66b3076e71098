// Internal interface of the df64 block kernels: Ozaki-split tensor-core
// products (oz.cu) and the df64 SpMM / conversion / reduction kernels (df_blas.cu).
#pragma once
#include <cuda_bf16.h>

#include "common.cuh"

namespace gsi {

struct OzGemmArgs {
  const float2* U[2];        // n x p df64 blocks; the left operand is U0 (+ a1 U1 if fuse_u1)
  int fuse_u1;
  float2 a1;
  int ne;                    // elementwise terms (0..2)
  const float2* E[2];        // n x p df64 blocks
  float2 ce[2];              // df64 scalars of the elementwise terms
  const __nv_bfloat16* Md;   // digit planes of the right operand
  const int* F;              // column exponents of the right operand
  float2* out;               // n x p df64 (may alias an E; may alias a U only when p <= 64)
  float2* dot_part;          // per-block partials {<out,out>, <out,dot_with>} or null
  const float2* dot_with;
  int dot_self;
  int vec16;                 // every block pointer 16-byte aligned: 16-byte loads and stores
  float* rinf_part;          // per-block max_r sum_j |hi(out[r,j])| (row-wise epilogue only) or null
  int ldu, kofs, kw;         // tcgen05 kernel: the left operand is columns kofs .. kofs+kw-1 of
                             // the row-major n x ldu blocks U (a slice of the contraction)
};

int pad16(int x);
// 0: tcgen05 kernels where they apply; 1: mma.sync kernels only
int tensor_path();
void set_tensor_path(int path);
size_t oz_rhs_bytes(int p, int nk);
// OUT = sum_{k<nk} U_k (s_k M_k) + sum_{e<ne} ce_e E_e; M_k float64 p x p (device).
// With nk = 2 and M_1 == M_0 the left operand U_0 + (s_1/s_0) U_1 is formed in
// df64 on the fly (one product of contraction length p).
// rhs_ws: oz_rhs_bytes(p, nk) bytes of device scratch for the right operand's digits.
// dot_part (optional): 2 * (*nparts) df64 partial sums.
// rinf_part (optional, oz_gemm_max_parts(p) floats): per-block maxima of the
// row sums sum_j |out[r, j]| (float32 sums of the high words), formed in the
// tcgen05 kernel's row-wise epilogue; *rinf_done tells whether they were.
gsi_status oz_gemm(int64_t n, int p, int nk, const float2* const U[2], const double* const M[2],
                   const double s[2], int ne, const float2* const E[2], const float2 ce[2],
                   float2* out, float2* dot_part, const float2* dot_with, bool dot_self,
                   void* rhs_ws, cudaStream_t st, int* nparts, int nd = 7,
                   float* rinf_part = nullptr, bool* rinf_done = nullptr);
int oz_gemm_max_parts(int p);
size_t oz_gram_scratch_bytes(int64_t n, int p, int q, bool sym);
// G = U^T V (float64 p x q); sym: U == V, only the upper half is computed.
// nd: digits per operand (7: float64-class; 3: bf16-level products with exact
// fp32 sums, used by the mixed-precision mode). With Gdf non-null the result
// is written as df64 to Gdf (p x q, any p; q <= 128): for symmetric A this is
// the dense apply A X = A^T X.
// reserve_sms: SMs left free for work running alongside on another stream.
gsi_status oz_gram(int64_t n, int p, int q, const float2* U, const float2* V, bool sym, double* G,
                   float2* scratch, cudaStream_t st, int nd = 7, float2* Gdf = nullptr,
                   int reserve_sms = 0);

// Bounded waits of the tcgen05 kernels: polls allowed to a wait on a batch of
// products (limit < 0: the default, 2^24); a wait that runs out drains the
// tensor core, counts one timeout and leaves non-finite outputs.
gsi_status oz_set_wait_limit(int limit);
// enqueue a copy of the process-wide timeout count into host_dst (pinned)
gsi_status oz_timeouts_async(int* host_dst, cudaStream_t st);

// Stencil-shaped operators: at most DIA_MAXD diagonals (df_blas.cu)
constexpr int DIA_T = 64;            // rows per tile of the shared-memory window
constexpr int DIA_MAXD = 8;          // diagonals stored
constexpr int DIA_MAXFAR = 2;        // diagonals read from global memory
constexpr int DIA_THREADS = 512;
constexpr int DIA_SMEM_MAX = 220 * 1024;
struct DiaArgs {
  int64_t n;
  int p, nd, q;                      // q: the window holds tiles k - q .. k + q
  int off[DIA_MAXD];                 // col - row of each diagonal, ascending
  int near_mask;                     // bit d: diagonal d read from the window
  int far_d[DIA_MAXFAR];             // the other diagonals
  int nfar;
  const float2* val;                 // n x nd df64 values, row-major
  const float2* X;
  float2* W;
  int64_t ntiles, tiles_per_cta;     // set by df_spmm_dia
};
size_t dia_smem_bytes(int p, int q, int nd);
// window geometry for p columns and the diagonals off[0..nd): 1 if the
// staged kernel applies (even p <= 64, at most DIA_MAXFAR far diagonals)
int dia_plan(int p, int nd, const int* off, int* q, int* near_mask, int* far_d, int* nfar);
gsi_status df_spmm_dia(const DiaArgs& a, cudaStream_t st);

// df64 block helpers (df_blas.cu)
gsi_status df_from_f64(int64_t count, const double* x, float2* y, cudaStream_t st);
gsi_status df_to_f64(int64_t count, const float2* x, double* y, cudaStream_t st);
gsi_status df_spmm_csr(int64_t n, const int64_t* rowptr, const int32_t* colidx, const float2* val,
                       int p, const float2* X, float2* W, cudaStream_t st);
gsi_status df_spmm_sell(int64_t nchunks, int C, const int64_t* perm, const int64_t* chunk_ptr,
                        const int64_t* chunk_len, const int32_t* scol, const float2* sval, int p,
                        const float2* X, float2* W, cudaStream_t st);
int df_dots_blocks(int64_t count);
// out[0] = <A0,B0>, out[1] = <A1,B1> (float64), out[2] = max_r sum_j |R[r,j]| (if R)
gsi_status df_dots(int64_t n, int p, const float2* A0, const float2* B0, const float2* A1,
                   const float2* B1, const float2* R, double* out, float2* scratch,
                   cudaStream_t st);
// y = a*x + b*y elementwise (df64 scalars)
gsi_status df_axpby(int64_t count, float2 a, const float2* x, float2 b, float2* y, cudaStream_t st);
// out = a W + b Z + e Zp elementwise (df64 scalars; Zp may be null)
gsi_status df_combine3(int64_t count, float2 a, const float2* W, float2 b, const float2* Z, float2 e,
                       const float2* Zp, float2* out, cudaStream_t st);
// sum of df64 partial pairs into out[0..1] (float64); with rinf_parts, also
// out[2] = max of rinf_parts[0..nparts)
gsi_status df_sum_parts(int nparts, const float2* parts, double* out, cudaStream_t st,
                        const float* rinf_parts = nullptr);

}  // namespace gsi
