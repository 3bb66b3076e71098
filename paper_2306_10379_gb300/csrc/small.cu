// The p x p part of one iteration, run by a single thread block in float64:
// the symmetric eigendecomposition D^T D = V diag(beta) V^T (Eq. (Gdec)), the
// line-search coefficients (Eqs. (diags), (CG_linesearch_D)), the exact step
// of Alg. 3 (bracket of Eqs. (derv1)/(derv2), Brent on phi'(t) of Eq.
// (deriv_P)), and the polar normaliser M = S^{-1/2} of Eq. (Ynew).
//
// The eigensolver is a block-parallel cyclic Jacobi method with round-robin
// (circle) ordering: each round applies p/2 disjoint rotations at once.
#include "alg3.cuh"
#include "blas_f64.cuh"
#include "small_dev.cuh"

#include <math.h>

namespace gsi {

constexpr int SMALL_THREADS = 512;
constexpr int SMALL_EIG_MAX = 192;

size_t small_scratch_doubles(int p) { return (size_t)5 * p * p + 5 * (size_t)p + 64; }

__global__ void __launch_bounds__(SMALL_THREADS)
small_step_kernel(int mode, int p, const double* C, const double* B, const double* Gam,
                  const double* Z, const double* XX, const double* XD, double* M, double* out,
                  double* ws) {
  __shared__ double rc[64], rs[64];
  __shared__ int ri[64], rj[64];
  __shared__ double red[64];
  __shared__ int flag;
  __shared__ double sh_t;
  SmallWs w = carve(ws, p);
  const int q = p * p;
  // 1. eigendecomposition of B (symmetrised)
  for (int e = threadIdx.x; e < q; e += blockDim.x) {
    int i = e / p, j = e - i * p;
    w.A[e] = 0.5 * (B[i * p + j] + B[j * p + i]);
    w.V[e] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  block_jacobi(p, w.A, w.V, 60, rc, rs, ri, rj, red);
  if (mode == 1) {
    int st = block_inv_sqrt(p, w.A, w.V, w.sv, M, &flag);
    if (threadIdx.x == 0) {
      out[0] = 0.0;
      out[1] = 0.0;
      out[2] = 0.0;
      out[3] = (double)st;
    }
    return;
  }
  for (int i = threadIdx.x; i < p; i += blockDim.x) w.beta[i] = fmax(w.A[i * p + i], 0.0);
  __syncthreads();
  // 2. alpha, gamma, zeta = diag(V^T {C, Gam, Z} V)
  block_diag_quad(p, C, w.V, w.T, w.alpha);
  block_diag_quad(p, Gam, w.V, w.T, w.gamma);
  block_diag_quad(p, Z, w.V, w.T, w.zeta);
  // 3. the exact step (one thread; O(p) per evaluation)
  if (threadIdx.x == 0) {
    int ev = 0;
    double t = get_mu(p, w.alpha, w.beta, w.gamma, w.zeta, &ev);
    double bmax = 0.0;
    for (int i = 0; i < p; ++i) bmax = fmax(bmax, w.beta[i]);
    sh_t = t;
    out[0] = t;
    out[1] = phi_model(t, p, w.alpha, w.beta, w.gamma, w.zeta);
    out[2] = (double)ev;
    out[4] = bmax;
  }
  __syncthreads();
  const double t = sh_t;
  // 4. S = XX + t (XD + XD^T) + t^2 B, rotated into the eigenbasis of B
  for (int e = threadIdx.x; e < q; e += blockDim.x) {
    int i = e / p, j = e - i * p;
    double sij = 0.5 * (XX[i * p + j] + XX[j * p + i]) + t * (XD[i * p + j] + XD[j * p + i]) +
                 t * t * 0.5 * (B[i * p + j] + B[j * p + i]);
    w.S[e] = sij;
  }
  __syncthreads();
  block_matmul(p, w.S, false, w.V, w.T);  // T = S V
  block_matmul(p, w.V, true, w.T, w.A);   // A = V^T S V (nearly diagonal)
  for (int e = threadIdx.x; e < q; e += blockDim.x) {
    int i = e / p, j = e - i * p;
    w.U[e] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  block_jacobi(p, w.A, w.U, 60, rc, rs, ri, rj, red);
  block_matmul(p, w.V, false, w.U, w.T);  // eigenvectors of S: T = V U
  int st = block_inv_sqrt(p, w.A, w.T, w.sv, M, &flag);
  if (threadIdx.x == 0) out[3] = (double)st;
}

gsi_status small_step(int mode, int p, const double* C, const double* B, const double* Gam,
                      const double* Z, const double* XX, const double* XD, double* M,
                      double* out, double* scratch, cudaStream_t st) {
  if (p < 1 || p > 128) return GSI_ERR_ARG;
  small_step_kernel<<<1, SMALL_THREADS, 0, st>>>(mode, p, C, B, Gam, Z, XX, XD, M, out, scratch);
  GSI_LAUNCH_CHECK();
  return GSI_OK;
}

// Rayleigh-Ritz (Eq. (rr1)): theta descending and U (columns) with
// (C + C^T)/2 = U diag(theta) U^T; p <= SMALL_EIG_MAX (the 3p x 3p
// Rayleigh-Ritz matrix of LOBCG at p <= 64).
__global__ void __launch_bounds__(SMALL_THREADS)
small_eig_kernel(int p, const double* C, double* theta, double* Uout, double* ws) {
  __shared__ double rc[SMALL_EIG_MAX / 2], rs[SMALL_EIG_MAX / 2];
  __shared__ int ri[SMALL_EIG_MAX / 2], rj[SMALL_EIG_MAX / 2];
  __shared__ double red[64];
  __shared__ int order[SMALL_EIG_MAX];
  SmallWs w = carve(ws, p);
  const int q = p * p;
  for (int e = threadIdx.x; e < q; e += blockDim.x) {
    int i = e / p, j = e - i * p;
    w.A[e] = 0.5 * (C[i * p + j] + C[j * p + i]);
    w.V[e] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  block_jacobi(p, w.A, w.V, 60, rc, rs, ri, rj, red);
  if (threadIdx.x == 0) {
    for (int i = 0; i < p; ++i) order[i] = i;
    for (int i = 0; i < p; ++i) {  // selection sort, descending
      int best = i;
      for (int j = i + 1; j < p; ++j)
        if (w.A[order[j] * p + order[j]] > w.A[order[best] * p + order[best]]) best = j;
      int tmp = order[i];
      order[i] = order[best];
      order[best] = tmp;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < p; i += blockDim.x) theta[i] = w.A[order[i] * p + order[i]];
  for (int e = threadIdx.x; e < q; e += blockDim.x) {
    int r = e / p, c = e - r * p;
    Uout[e] = w.V[r * p + order[c]];
  }
}

gsi_status small_eig(int p, const double* C, double* theta, double* U, double* scratch,
                     cudaStream_t st) {
  if (p < 1 || p > SMALL_EIG_MAX) return GSI_ERR_ARG;
  small_eig_kernel<<<1, SMALL_THREADS, 0, st>>>(p, C, theta, U, scratch);
  GSI_LAUNCH_CHECK();
  return GSI_OK;
}

}  // namespace gsi
