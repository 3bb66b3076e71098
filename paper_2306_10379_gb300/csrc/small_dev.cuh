// Block-parallel float64 building blocks of the p x p step: one thread
// block works on p x p row-major matrices (global or shared memory) with
// blockDim-strided loops. Used by the single-problem step and by the batched
// solver, which runs one block per problem.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace gsi {

constexpr double DEPS = 2.220446049250313e-16;

struct SmallWs {
  double *A, *V, *T, *U, *S;   // p x p each
  double *alpha, *beta, *gamma, *zeta, *sv;  // p each
};

static __device__ SmallWs carve(double* ws, int p) {
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

static __device__ void block_reduce2(double& a, double& b, double* red) {
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
static __device__ void block_jacobi(int p, double* A, double* V, int max_sweeps, double* rc, double* rs,
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
static __device__ void block_matmul(int p, const double* X, bool transX, const double* Y, double* Out) {
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
static __device__ void block_diag_quad(int p, const double* G, const double* V, double* T, double* d) {
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
static __device__ int block_inv_sqrt(int p, const double* Adiag, const double* U, double* sv, double* M,
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

}  // namespace gsi
