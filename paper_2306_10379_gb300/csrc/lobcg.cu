// p x p helpers of the LOBCG comparator (Sec. 6.4, "Comparison to LOBCG"):
// block orthonormalisation coefficients from a Gram's eigendecomposition,
// assembly of the Rayleigh-Ritz matrix Q^T A Q of V_k = span(X_k, G_k, P_k)
// (Eq. (def_Vk_LOBPCG)) and the split of its top eigenvectors into the three
// blocks' coefficients. The n x p work (Grams, block products, SpMMs) runs
// on the solver's kernels.
#include "blas_f64.cuh"

namespace gsi {

// Block orthonormalisation by a Gram S = B^T B = U diag(theta) U^T (theta
// descending): M = U_r diag(theta_r)^(-1/2) over theta_i > tol2 theta_0,
// columns of the dropped eigenvalues zero; mask[j] = 1 for kept columns.
// One block of p threads (p <= 64).
__global__ void lobcg_coef_kernel(int p, const double* theta, const double* U, double tol2, double* M, int* mask) {
  const int j = threadIdx.x;
  if (j >= p) return;
  const double t0 = theta[0];
  const bool keep = t0 > 0.0 && theta[j] > tol2 * t0;
  mask[j] = keep ? 1 : 0;
  const double f = keep ? 1.0 / sqrt(theta[j]) : 0.0;
  for (int i = 0; i < p; ++i) M[i * p + j] = U[i * p + j] * f;
}

gsi_status lobcg_coef(int p, const double* theta, const double* U, double tol2, double* M, int* mask,
                      cudaStream_t st) {
  if (p < 1 || p > 64) return GSI_ERR_ARG;
  lobcg_coef_kernel<<<1, 64, 0, st>>>(p, theta, U, tol2, M, mask);
  GSI_LAUNCH_CHECK();
  return GSI_OK;
}

// Rows and columns of dropped basis columns (mask 0) of a p x p Gram set to
// those of the identity, so that its inverse square root leaves the zero
// columns zero and normalises the rest.
__global__ void lobcg_mask_gram_kernel(int p, double* S, const int* mask) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= p * p) return;
  const int i = e / p, j = e - i * p;
  if (!mask[i] || !mask[j]) S[e] = (i == j) ? 1.0 : 0.0;
}

gsi_status lobcg_mask_gram(int p, double* S, const int* mask, cudaStream_t st) {
  lobcg_mask_gram_kernel<<<ceil_div(p * p, 256), 256, 0, st>>>(p, S, mask);
  GSI_LAUNCH_CHECK();
  return GSI_OK;
}

// H (nb p x nb p, nb = 2 or 3) from its blocks H_ab = Q_a^T A Q_b (a <= b),
// the diagonal blocks symmetrised; rows and columns of dropped basis columns
// (mask2 / mask3 = 0 for blocks 2 / 3) zero with `sentinel` on the diagonal
// (below every Ritz value, so that no such column is selected).
__global__ void lobcg_assemble_kernel(int p, int nb, const double* H11, const double* H12, const double* H13,
                                      const double* H22, const double* H23, const double* H33, const int* mask2,
                                      const int* mask3, double sentinel, double* H) {
  const int m = nb * p;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m * m) return;
  const int r = e / m, c = e - r * m;
  const int br = r / p, bc = c / p, i = r - br * p, j = c - bc * p;
  auto live = [&](int b, int k) { return b == 0 || (b == 1 ? mask2[k] : mask3[k]) != 0; };
  if (!live(br, i) || !live(bc, j)) {
    H[e] = (r == c) ? sentinel : 0.0;
    return;
  }
  const double* blk[3][3] = {{H11, H12, H13}, {nullptr, H22, H23}, {nullptr, nullptr, H33}};
  double v;
  if (br == bc) v = 0.5 * (blk[br][br][i * p + j] + blk[br][br][j * p + i]);
  else if (br < bc) v = blk[br][bc][i * p + j];
  else v = blk[bc][br][j * p + i];
  H[e] = v;
}

gsi_status lobcg_assemble(int p, int nb, const double* H11, const double* H12, const double* H13,
                          const double* H22, const double* H23, const double* H33, const int* mask2,
                          const int* mask3, double sentinel, double* H, cudaStream_t st) {
  const int m = nb * p;
  lobcg_assemble_kernel<<<ceil_div(m * m, 256), 256, 0, st>>>(p, nb, H11, H12, H13, H22, H23, H33, mask2,
                                                              mask3, sentinel, H);
  GSI_LAUNCH_CHECK();
  return GSI_OK;
}

// The top p eigenvectors (the first p columns of U, nb p x nb p, eigenvalues
// descending) cut into the blocks' coefficients V_b (p x p): X_{k+1} =
// sum_b Q_b V_b.
__global__ void lobcg_split_kernel(int p, int nb, const double* U, double* V1, double* V2, double* V3) {
  const int m = nb * p;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nb * p * p) return;
  const int b = e / (p * p), r = e - b * p * p, i = r / p, j = r - i * p;
  double* V = b == 0 ? V1 : (b == 1 ? V2 : V3);
  V[i * p + j] = U[(b * p + i) * m + j];
}

gsi_status lobcg_split(int p, int nb, const double* U, double* V1, double* V2, double* V3, cudaStream_t st) {
  lobcg_split_kernel<<<ceil_div(nb * p * p, 256), 256, 0, st>>>(p, nb, U, V1, V2, V3);
  GSI_LAUNCH_CHECK();
  return GSI_OK;
}

}  // namespace gsi
