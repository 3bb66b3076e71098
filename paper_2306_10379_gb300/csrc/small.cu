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

#include <math.h>

namespace gsi {

constexpr int SMALL_THREADS = 512;
constexpr double DEPS = 2.220446049250313e-16;

struct SmallWs {
  double *A, *V, *T, *U, *S;   // p x p each
  double *alpha, *beta, *gamma, *zeta, *sv;  // p each
};

__device__ SmallWs carve(double* ws, int p) {
  SmallWs w;
  size_t q = (size_t)p * p;
  w.A = ws;
  w.V = ws + q;
  w.T = ws + 2 * q;
  w.U = ws + 3 * q;
  w.S = ws + 4 * q;
  w.alpha = ws + 5 * q;
  w.beta = w.alpha + p;
  w.gamma = w.beta + p;
  w.zeta = w.gamma + p;
  w.sv = w.zeta + p;
  return w;
}

size_t small_scratch_doubles(int p) { return (size_t)5 * p * p + 5 * (size_t)p + 64; }

__device__ void block_reduce2(double& a, double& b, double* red) {
  // sum of a and b over the block; result broadcast to all threads
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) {
    red[2 * w] = a;
    red[2 * w + 1] = b;
  }
  __syncthreads();
  a = 0.0;
  b = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
    a += red[2 * i];
    b += red[2 * i + 1];
  }
  __syncthreads();
}

// Eigendecomposition of the symmetric A (p x p, row-major, overwritten by a
// nearly diagonal matrix whose diagonal holds the eigenvalues); V is
// multiplied on the right by the rotations (initialise it to I, or to a
// previous eigenbasis for a warm start with A = V^T A0 V).
__device__ void block_jacobi(int p, double* A, double* V, int max_sweeps, double* rc, double* rs,
                             int* ri, int* rj, double* red) {
  const int m = (p + 1) & ~1;  // even number of players; index p is a dummy when p is odd
  const int half = m / 2;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
      double a = A[e];
      tot += a * a;
      if (e / p != e % p) off += a * a;
    }
    block_reduce2(off, tot, red);
    if (!(off > 1e-4 * DEPS * DEPS * tot) || tot == 0.0) break;
    for (int r = 0; r < m - 1; ++r) {
      for (int k = threadIdx.x; k < half; k += blockDim.x) {
        int a, b;
        if (k == 0) {
          a = r;
          b = m - 1;
        } else {
          a = (r + k) % (m - 1);
          b = (r + (m - 1) - k) % (m - 1);
        }
        int i = min(a, b), j = max(a, b);
        double c = 1.0, s = 0.0;
        if (j < p) {
          double aij = A[i * p + j];
          double aii = A[i * p + i], ajj = A[j * p + j];
          if (aij != 0.0 && fabs(aij) > 1e-3 * DEPS * sqrt(fabs(aii)) * sqrt(fabs(ajj))) {
            double th = (ajj - aii) / (2.0 * aij);
            double t;
            if (fabs(th) > 1e150) {
              t = 0.5 / th;
            } else {
              t = copysign(1.0, th) / (fabs(th) + sqrt(th * th + 1.0));
            }
            c = 1.0 / sqrt(t * t + 1.0);
            s = t * c;
          }
        } else {
          i = j = -1;
        }
        rc[k] = c;
        rs[k] = s;
        ri[k] = i;
        rj[k] = j;
      }
      __syncthreads();
      // rows i, j of J^T A
      for (int e = threadIdx.x; e < half * p; e += blockDim.x) {
        int k = e / p, col = e - k * p;
        int i = ri[k], j = rj[k];
        if (i < 0 || rs[k] == 0.0) continue;
        double c = rc[k], s = rs[k];
        double ai = A[i * p + col], aj = A[j * p + col];
        A[i * p + col] = c * ai - s * aj;
        A[j * p + col] = s * ai + c * aj;
      }
      __syncthreads();
      // columns i, j of (J^T A) J, and of V J
      for (int e = threadIdx.x; e < half * p; e += blockDim.x) {
        int k = e / p, row = e - k * p;
        int i = ri[k], j = rj[k];
        if (i < 0 || rs[k] == 0.0) continue;
        double c = rc[k], s = rs[k];
        double ai = A[row * p + i], aj = A[row * p + j];
        A[row * p + i] = c * ai - s * aj;
        A[row * p + j] = s * ai + c * aj;
        double vi = V[row * p + i], vj = V[row * p + j];
        V[row * p + i] = c * vi - s * vj;
        V[row * p + j] = s * vi + c * vj;
      }
      __syncthreads();
      for (int k = threadIdx.x; k < half; k += blockDim.x) {
        int i = ri[k], j = rj[k];
        if (i >= 0 && rs[k] != 0.0) {
          A[i * p + j] = 0.0;
          A[j * p + i] = 0.0;
        }
      }
      __syncthreads();
    }
  }
}

// Out = X^T Y (transX) or X Y, all p x p row-major, block-parallel.
__device__ void block_matmul(int p, const double* X, bool transX, const double* Y, double* Out) {
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
    int i = e / p, j = e - i * p;
    double s = 0.0;
    if (transX) {
      for (int k = 0; k < p; ++k) s = fma(X[k * p + i], Y[k * p + j], s);
    } else {
      for (int k = 0; k < p; ++k) s = fma(X[i * p + k], Y[k * p + j], s);
    }
    Out[e] = s;
  }
  __syncthreads();
}

// diag(V^T G V), G symmetrised as (G + G^T)/2 (the diagonal does not change).
__device__ void block_diag_quad(int p, const double* G, const double* V, double* T, double* d) {
  block_matmul(p, G, false, V, T);  // T = G V
  for (int i = threadIdx.x; i < p; i += blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < p; ++k) s = fma(V[k * p + i], T[k * p + i], s);
    d[i] = s;
  }
  __syncthreads();
}

// M = U diag(s^{-1/2}) U^T for S = U diag(s) U^T held as (A diagonal, U).
// Returns 0, or 5 if some s_i <= 0 or is not finite.
__device__ int block_inv_sqrt(int p, const double* Adiag, const double* U, double* sv, double* M,
                              int* flag) {
  if (threadIdx.x == 0) *flag = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < p; i += blockDim.x) {
    double s = Adiag[i * p + i];
    if (!(s > 0.0) || !isfinite(s)) {
      *flag = 5;
      sv[i] = 0.0;
    } else {
      sv[i] = 1.0 / sqrt(s);
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
    int i = e / p, j = e - i * p;
    double s = 0.0;
    for (int k = 0; k < p; ++k) s = fma(U[i * p + k] * sv[k], U[j * p + k], s);
    M[e] = s;
  }
  __syncthreads();
  return *flag;
}

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
// (C + C^T)/2 = U diag(theta) U^T.
__global__ void __launch_bounds__(SMALL_THREADS)
small_eig_kernel(int p, const double* C, double* theta, double* Uout, double* ws) {
  __shared__ double rc[64], rs[64];
  __shared__ int ri[64], rj[64];
  __shared__ double red[64];
  __shared__ int order[128];
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
  if (p < 1 || p > 128) return GSI_ERR_ARG;
  small_eig_kernel<<<1, SMALL_THREADS, 0, st>>>(p, C, theta, U, scratch);
  GSI_LAUNCH_CHECK();
  return GSI_OK;
}

}  // namespace gsi
