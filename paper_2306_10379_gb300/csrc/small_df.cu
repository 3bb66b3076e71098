// The p x p step of one iteration without leaning on the float64 pipe (one
// thread block): the symmetric eigendecomposition B = D^T D = V diag(beta) V^T
// of Eq. (Gdec) is found by a float32 Jacobi method and refined to
// float64-class accuracy in df64 (one Newton-Schulz orthonormalisation of V,
// then Jacobi sweeps on the nearly diagonal V^T B V); the line-search
// coefficients of Eqs. (diags)/(CG_linesearch_D) and Alg. 3 follow in
// float64; the polar normaliser M = S^{-1/2} of the measured Gram S of
// X + tD (Eq. (Ynew)) is taken in the same eigenbasis, where S is diagonal up
// to rounding-level terms F, by the first-order expansion
//   S^{-1/2} = V [diag(s^{-1/2}) + F o Df] V^T,  Df_ij = -1/(r_i r_j (r_i + r_j)),
// r = sqrt(s) (the divided differences of x^{-1/2}).
//
// Jacobi rounds use the round-robin (circle) ordering: p/2 disjoint rotations
// per round, each 2 x 2 block of J^T A J updated by one thread.
#include "small_df_dev.cuh"
#include "blas_f64.cuh"

namespace gsi {

constexpr int SD_THREADS = 1024;

__global__ void __launch_bounds__(SD_THREADS)
small_df_kernel(int mode, int p, const double* C, const double* B, const double* Gam,
                const double* Z, const double* XX, const double* XD, double* M, double* out,
                unsigned char* gws, int use_smem, float2* eig) {
  extern __shared__ __align__(16) unsigned char sm_dyn[];
  __shared__ double red[SD_THREADS / 32];
  __shared__ int flag;
  __shared__ double sh_t;
  // use_smem: 1 = everything in shared memory, 2 = float32 part only
  SdWs w = use_smem == 1 ? sd_carve(sm_dyn, p) : use_smem == 2 ? sd_carve(gws, p, sm_dyn)
                                                                  : sd_carve(gws, p);
  small_df_body(mode, p, C, B, Gam, Z, XX, XD, M, out, w, red, &flag, &sh_t, eig);
}

size_t small_df_scratch_bytes(int p) { return sd_bytes(p); }

gsi_status small_step_df(int mode, int p, const double* C, const double* B, const double* Gam,
                         const double* Z, const double* XX, const double* XD, double* M,
                         double* out, void* scratch, cudaStream_t st, void* eig_ws) {
  if (p < 1 || p > 128 || ((mode == 3 || mode == 4) && !eig_ws)) return GSI_ERR_ARG;
  size_t bytes = sd_bytes(p);
  const size_t dfpart = 4 * (((size_t)p * p * sizeof(float2) + 15) & ~(size_t)15);
  int use_smem = bytes <= 200 * 1024 ? 1 : (bytes - dfpart <= 200 * 1024 ? 2 : 0);
  size_t sm = use_smem == 1 ? bytes : use_smem == 2 ? bytes - dfpart : 0;
  if (use_smem)
    GSI_CUDA_TRY(ensure_dyn_smem((const void*)small_df_kernel, (int)sm));
  small_df_kernel<<<1, SD_THREADS, sm, st>>>(mode, p, C, B, Gam, Z, XX, XD, M, out,
                                             (unsigned char*)scratch, use_smem, (float2*)eig_ws);
  GSI_LAUNCH_CHECK();
  return GSI_OK;
}

}  // namespace gsi
