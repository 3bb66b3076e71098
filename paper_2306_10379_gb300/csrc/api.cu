// Kernel-level C entry points: the steps of one iteration, exposed for
// parity tests and benchmarks. Temporary buffers are stream-ordered
// allocations on the caller's stream.
#include <algorithm>

#include "blas_f64.cuh"
#include "oz.cuh"

using namespace gsi;

namespace {

struct ScratchGuard {
  void* ptr = nullptr;
  cudaStream_t st;
  explicit ScratchGuard(cudaStream_t s) : st(s) {}
  ~ScratchGuard() {
    if (ptr) cudaFreeAsync(ptr, st);
  }
};

}  // namespace

extern "C" {

gsi_status gsi_spmm_csr(int64_t n, const int64_t* rowptr, const int32_t* colidx,
                        const double* val, int32_t p, const double* X, double* W,
                        void* stream) {
  if (n < 0 || p < 1 || (n > 0 && (!rowptr || !colidx || !val || !X || !W))) return GSI_ERR_ARG;
  return spmm_csr(n, rowptr, colidx, val, p, X, W, (cudaStream_t)stream);
}

gsi_status gsi_spmm_sell(int64_t n, int64_t nchunks, int32_t C, const int64_t* perm,
                         const int64_t* chunk_ptr, const int64_t* chunk_len,
                         const int32_t* sell_col, const double* sell_val, int32_t p,
                         const double* X, double* W, void* stream) {
  if (n < 0 || nchunks < 0 || C <= 0 || p < 1 || nchunks * C < n) return GSI_ERR_ARG;
  if (nchunks > 0 && (!perm || !chunk_ptr || !chunk_len || !sell_col || !sell_val || !X || !W))
    return GSI_ERR_ARG;
  return spmm_sell(n, nchunks, C, perm, chunk_ptr, chunk_len, sell_col, sell_val, p, X, W,
                   (cudaStream_t)stream);
}

gsi_status gsi_gram(int64_t n, int32_t p, int32_t q, const double* U, const double* V,
                    double* G, void* stream) {
  if (n < 0 || p < 1 || q < 1 || p > 128 || q > 128 || !G || (n > 0 && (!U || !V)))
    return GSI_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  ScratchGuard g(st);
  size_t bytes = std::max<size_t>(gram_scratch_doubles(n, p, q), 1) * sizeof(double);
  GSI_CUDA_TRY(cudaMallocAsync(&g.ptr, bytes, st));
  return gram(n, p, q, U, V, G, (double*)g.ptr, st);
}

gsi_status gsi_residual(int64_t n, int32_t p, const double* X, const double* Y,
                        const double* C, double* R, void* stream) {
  if (n < 0 || p < 1 || p > 128 || (n > 0 && (!X || !Y || !C || !R))) return GSI_ERR_ARG;
  RowMulArgs a{};
  a.nk = 1;
  a.U[0] = X;
  a.M[0] = C;
  a.s[0] = -1.0;
  a.ne = 1;
  a.E[0] = Y;
  a.c[0] = 1.0;
  return rowmul(n, p, a, R, (cudaStream_t)stream);
}

gsi_status gsi_linesearch(int32_t p, const double* C, const double* B, const double* Gam,
                          const double* Z, const double* XX, const double* XD, double* M,
                          double* out, int32_t precision, void* stream) {
  if (p < 1 || p > 128 || !C || !B || !Gam || !Z || !XX || !XD || !M || !out) return GSI_ERR_ARG;
  if (precision != GSI_PREC_DF64 && precision != GSI_PREC_F64) return GSI_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  ScratchGuard g(st);
  if (precision == GSI_PREC_DF64) {
    GSI_CUDA_TRY(cudaMallocAsync(&g.ptr, small_df_scratch_bytes(p), st));
    return small_step_df(0, p, C, B, Gam, Z, XX, XD, M, out, g.ptr, st);
  }
  GSI_CUDA_TRY(cudaMallocAsync(&g.ptr, small_scratch_doubles(p) * sizeof(double), st));
  return small_step(0, p, C, B, Gam, Z, XX, XD, M, out, (double*)g.ptr, st);
}

gsi_status gsi_retract(int64_t n, int32_t p, double t, const double* M, double* X,
                       const double* D, double* Y, const double* W, void* stream) {
  if (n < 0 || p < 1 || p > 128 || !M || (n > 0 && (!X || !D || !Y || !W))) return GSI_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  RowMulArgs a{};
  a.nk = 2;
  a.U[0] = X;
  a.M[0] = M;
  a.s[0] = 1.0;
  a.U[1] = D;
  a.M[1] = M;
  a.s[1] = t;
  GSI_TRY(rowmul(n, p, a, X, st));
  a.U[0] = Y;
  a.U[1] = W;
  return rowmul(n, p, a, Y, st);
}

gsi_status gsi_df_spmm_csr(int64_t n, const int64_t* rowptr, const int32_t* colidx,
                           const float* val, int32_t p, const float* X, float* W, void* stream) {
  if (n < 0 || p < 1 || (n > 0 && (!rowptr || !colidx || !val || !X || !W))) return GSI_ERR_ARG;
  return df_spmm_csr(n, rowptr, colidx, reinterpret_cast<const float2*>(val), p,
                     reinterpret_cast<const float2*>(X), reinterpret_cast<float2*>(W),
                     (cudaStream_t)stream);
}

gsi_status gsi_oz_gemm(int64_t n, int32_t p, int32_t nk, const float* U0, const float* U1,
                       const double* M0, const double* M1, double s0, double s1, int32_t ne,
                       const float* E0, const float* E1, const float* c, float* OUT,
                       void* stream) {
  if (n < 0 || p < 1 || p > 128 || nk < 1 || nk > 2 || ne < 0 || ne > 2 || !U0 || !M0 || !OUT ||
      (nk == 2 && (!U1 || !M1)) || (ne > 0 && (!c || !E0)) || (ne > 1 && !E1))
    return GSI_ERR_ARG;
  if (n == 0) return GSI_OK;
  cudaStream_t st = (cudaStream_t)stream;
  ScratchGuard g(st);
  GSI_CUDA_TRY(cudaMallocAsync(&g.ptr, oz_rhs_bytes(p, nk), st));
  const float2* U[2] = {reinterpret_cast<const float2*>(U0), reinterpret_cast<const float2*>(U1)};
  const double* M[2] = {M0, M1};
  double s[2] = {s0, s1};
  const float2* E[2] = {reinterpret_cast<const float2*>(E0), reinterpret_cast<const float2*>(E1)};
  float2 ce[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
  for (int m = 0; m < ne; ++m) ce[m] = make_float2(c[2 * m], c[2 * m + 1]);
  return oz_gemm(n, p, nk, U, M, s, ne, E, ce, reinterpret_cast<float2*>(OUT), nullptr, nullptr,
                 false, g.ptr, st, nullptr);
}

gsi_status gsi_oz_gram(int64_t n, int32_t p, int32_t q, const float* U, const float* V,
                       int32_t sym, double* G, void* stream) {
  if (n < 0 || p < 1 || q < 1 || p > 128 || q > 128 || !G || (n > 0 && (!U || !V)) ||
      (sym && (p != q || U != V)))
    return GSI_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  ScratchGuard g(st);
  GSI_CUDA_TRY(cudaMallocAsync(&g.ptr, std::max<size_t>(oz_gram_scratch_bytes(n, p, q, sym != 0), 16), st));
  return oz_gram(n, p, q, reinterpret_cast<const float2*>(U), reinterpret_cast<const float2*>(V),
                 sym != 0, G, reinterpret_cast<float2*>(g.ptr), st);
}

gsi_status gsi_oz_dense_apply(int64_t n, int32_t p, const float* A, const float* X, float* W,
                              int32_t nd, void* stream) {
  if (n < 1 || p < 1 || p > 128 || !A || !X || !W || (nd != 3 && nd != 7)) return GSI_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  ScratchGuard g(st);
  GSI_CUDA_TRY(cudaMallocAsync(&g.ptr, std::max<size_t>(oz_gram_scratch_bytes(n, (int)n, p, false), 16), st));
  return oz_gram(n, (int)n, p, reinterpret_cast<const float2*>(A), reinterpret_cast<const float2*>(X),
                 false, nullptr, reinterpret_cast<float2*>(g.ptr), st, nd,
                 reinterpret_cast<float2*>(W));
}

gsi_status gsi_set_tensor_path(int32_t path) {
  if (path < 0 || path > 2) return GSI_ERR_ARG;
  set_tensor_path(path);
  return GSI_OK;
}

int32_t gsi_tensor_path(void) { return tensor_path(); }

gsi_status gsi_df_spmm_dia(int64_t n, int32_t ndiag, const int64_t* offsets, const float* dia, int32_t p,
                           const float* X, float* W, void* stream) {
  if (n < 0 || ndiag < 1 || ndiag > DIA_MAXD || !offsets || (n > 0 && (!dia || !X || !W))) return GSI_ERR_ARG;
  if (((uintptr_t)X & 15) || ((uintptr_t)W & 15) || ((uintptr_t)dia & 7)) return GSI_ERR_ARG;
  DiaArgs a{};
  a.n = n;
  a.p = p;
  a.nd = ndiag;
  for (int d = 0; d < ndiag; ++d) {
    if (offsets[d] <= -n || offsets[d] >= n || (d > 0 && offsets[d] <= offsets[d - 1])) return GSI_ERR_ARG;
    a.off[d] = (int)offsets[d];
  }
  if (!dia_plan(p, ndiag, a.off, &a.q, &a.near_mask, a.far_d, &a.nfar)) return GSI_ERR_ARG;
  a.val = reinterpret_cast<const float2*>(dia);
  a.X = reinterpret_cast<const float2*>(X);
  a.W = reinterpret_cast<float2*>(W);
  return df_spmm_dia(a, (cudaStream_t)stream);
}

}  // extern "C"
