// Block kernels of one iteration in float64: the block matvec (CSR and
// SELL-C-sigma SpMM), tall-skinny Gram products, right multiplication of
// n x p blocks by p x p matrices, and Frobenius inner products.
//
// Layout: every n x p block is row-major with leading dimension p.
#include "blas_f64.cuh"

#include <algorithm>

namespace gsi {

// ---------------------------------------------------------------------------
// SpMM W = A X, CSR (Sec. 6.1 "Efficient matvecs": one block matvec per
// iteration). Thread <-> (row, pair of columns); the threads of one row are
// adjacent, so the gathered X rows are read as contiguous 16-byte vectors and
// the row's (col, val) stream is a broadcast.
// ---------------------------------------------------------------------------
template <bool VEC2>
__global__ void spmm_csr_kernel(int64_t n, const int64_t* __restrict__ rowptr,
                                const int32_t* __restrict__ colidx,
                                const double* __restrict__ val, int p, int cpr,
                                const double* __restrict__ X, double* __restrict__ W) {
  int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t row = gid / cpr;
  int c = (int)(gid - row * cpr);
  if (row >= n) return;
  int64_t b = __ldg(rowptr + row), e = __ldg(rowptr + row + 1);
  if (VEC2) {
    double ax = 0.0, ay = 0.0;
    for (int64_t k = b; k < e; ++k) {
      double a = __ldg(val + k);
      int64_t col = __ldg(colidx + k);
      double2 x = __ldg(reinterpret_cast<const double2*>(X + col * p) + c);
      ax = fma(a, x.x, ax);
      ay = fma(a, x.y, ay);
    }
    reinterpret_cast<double2*>(W + row * p)[c] = make_double2(ax, ay);
  } else {
    double acc = 0.0;
    for (int64_t k = b; k < e; ++k) {
      double a = __ldg(val + k);
      int64_t col = __ldg(colidx + k);
      acc = fma(a, __ldg(X + col * p + c), acc);
    }
    W[row * p + c] = acc;
  }
}

gsi_status spmm_csr(int64_t n, const int64_t* rowptr, const int32_t* colidx, const double* val,
                    int p, const double* X, double* W, cudaStream_t st) {
  if (n <= 0) return GSI_OK;
  const int threads = 256;
  if ((p & 1) == 0) {
    int cpr = p / 2;
    int64_t total = n * cpr;
    spmm_csr_kernel<true><<<ceil_div(total, threads), threads, 0, st>>>(n, rowptr, colidx, val, p,
                                                                         cpr, X, W);
  } else {
    int64_t total = n * p;
    spmm_csr_kernel<false><<<ceil_div(total, threads), threads, 0, st>>>(n, rowptr, colidx, val, p,
                                                                          p, X, W);
  }
  GSI_LAUNCH_CHECK();
  return GSI_OK;
}

// ---------------------------------------------------------------------------
// SpMM W = A X, SELL-C-sigma. Thread <-> (permuted slot, column); chunk
// entries are read column-major (entry j of the C rows of a chunk adjacent).
// ---------------------------------------------------------------------------
__global__ void spmm_sell_kernel(int64_t nslots, int C, const int64_t* __restrict__ perm,
                                 const int64_t* __restrict__ chunk_ptr,
                                 const int64_t* __restrict__ chunk_len,
                                 const int32_t* __restrict__ scol,
                                 const double* __restrict__ sval, int p,
                                 const double* __restrict__ X, double* __restrict__ W) {
  int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t slot = gid / p;
  int c = (int)(gid - slot * p);
  if (slot >= nslots) return;
  int64_t row = __ldg(perm + slot);
  if (row < 0) return;
  int64_t ch = slot / C;
  int lane = (int)(slot - ch * C);
  int64_t base = __ldg(chunk_ptr + ch) + lane;
  int64_t len = __ldg(chunk_len + ch);
  double acc = 0.0;
  for (int64_t j = 0; j < len; ++j) {
    int64_t s = base + j * C;
    acc = fma(__ldg(sval + s), __ldg(X + (int64_t)__ldg(scol + s) * p + c), acc);
  }
  W[row * p + c] = acc;
}

gsi_status spmm_sell(int64_t n, int64_t nchunks, int C, const int64_t* perm,
                     const int64_t* chunk_ptr, const int64_t* chunk_len, const int32_t* scol,
                     const double* sval, int p, const double* X, double* W, cudaStream_t st) {
  (void)n;
  int64_t nslots = nchunks * C;
  if (nslots <= 0) return GSI_OK;
  int64_t total = nslots * p;
  spmm_sell_kernel<<<ceil_div(total, 256), 256, 0, st>>>(nslots, C, perm, chunk_ptr, chunk_len,
                                                         scol, sval, p, X, W);
  GSI_LAUNCH_CHECK();
  return GSI_OK;
}

// ---------------------------------------------------------------------------
// Gram G = U^T V. Stage 1: block b sums rows [b*rpb, (b+1)*rpb) into a p x q
// partial; each thread owns a 4 x 4 tile of outputs, rows are staged through
// shared memory 16 at a time. Stage 2: a fixed-order sum of the partials, so
// the result is deterministic for given (n, p, q).
// ---------------------------------------------------------------------------
constexpr int GRAM_RB = 16;

__global__ void gram_partial_kernel(int64_t n, int p, int q, int64_t rpb,
                                    const double* __restrict__ U, const double* __restrict__ V,
                                    double* __restrict__ part) {
  extern __shared__ double sm[];
  double* Us = sm;                  // GRAM_RB x p
  double* Vs = sm + GRAM_RB * p;    // GRAM_RB x q
  const int tq = (q + 3) / 4;
  const int ti = threadIdx.x / tq, tj = threadIdx.x % tq;
  const int tp = (p + 3) / 4;
  const bool active = ti < tp;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
  int64_t r0 = (int64_t)blockIdx.x * rpb;
  int64_t r1 = min(n, r0 + rpb);
  for (int64_t rb = r0; rb < r1; rb += GRAM_RB) {
    int nr = (int)min((int64_t)GRAM_RB, r1 - rb);
    for (int e = threadIdx.x; e < GRAM_RB * p; e += blockDim.x) {
      int rr = e / p;
      Us[e] = rr < nr ? U[(rb + rr) * p + (e - rr * p)] : 0.0;
    }
    for (int e = threadIdx.x; e < GRAM_RB * q; e += blockDim.x) {
      int rr = e / q;
      Vs[e] = rr < nr ? V[(rb + rr) * q + (e - rr * q)] : 0.0;
    }
    __syncthreads();
    if (active) {
      for (int rr = 0; rr < nr; ++rr) {
        double u[4], v[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          int i = 4 * ti + a;
          u[a] = i < p ? Us[rr * p + i] : 0.0;
        }
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          int j = 4 * tj + b;
          v[b] = j < q ? Vs[rr * q + j] : 0.0;
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = fma(u[a], v[b], acc[a][b]);
      }
    }
    __syncthreads();
  }
  if (active) {
    double* out = part + (int64_t)blockIdx.x * p * q;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        int i = 4 * ti + a, j = 4 * tj + b;
        if (i < p && j < q) out[i * q + j] = acc[a][b];
      }
  }
}

__global__ void sum_partials_kernel(int nb, int pq, const double* __restrict__ part,
                                    double* __restrict__ G) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= pq) return;
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += part[(int64_t)b * pq + e];
  G[e] = s;
}

int gram_blocks(int64_t n) {
  int64_t want = (int64_t)sm_count() * 4;
  int64_t by_rows = (n + 255) / 256;  // at least 256 rows per block
  return (int)std::max<int64_t>(1, std::min(want, by_rows));
}

size_t gram_scratch_doubles(int64_t n, int p, int q) {
  return (size_t)gram_blocks(n) * p * q;
}

gsi_status gram(int64_t n, int p, int q, const double* U, const double* V, double* G,
                double* scratch, cudaStream_t st) {
  int nb = gram_blocks(n);
  int64_t rpb = (n + nb - 1) / nb;
  rpb = (rpb + GRAM_RB - 1) / GRAM_RB * GRAM_RB;
  nb = (int)((n + rpb - 1) / rpb);
  if (n <= 0) nb = 0;
  int threads = ((p + 3) / 4) * ((q + 3) / 4);
  threads = (threads + 31) / 32 * 32;
  size_t smem = (size_t)GRAM_RB * (p + q) * sizeof(double);
  if (nb > 0) {
    gram_partial_kernel<<<nb, threads, smem, st>>>(n, p, q, rpb, U, V, scratch);
    GSI_LAUNCH_CHECK();
  }
  int pq = p * q;
  sum_partials_kernel<<<ceil_div(pq, 256), 256, 0, st>>>(nb, pq, scratch, G);
  GSI_LAUNCH_CHECK();
  return GSI_OK;
}

// ---------------------------------------------------------------------------
// Right multiplication with elementwise terms:
//   out[r, :] = sum_k s_k * U_k[r, :] M_k  +  sum_e c_e * E_e[r, :]
// (k < 2, e < 2). Residual R = Y - X C, CG direction R + b P - X (b K), and
// the retraction X M + D (t M) are all of this form. A block stages its rows
// of the U_k in shared memory before writing, so out may alias any input.
// ---------------------------------------------------------------------------
constexpr int RM_RB = 8;

__global__ void rowmul_kernel(int64_t n, int p, RowMulArgs a, double* out) {
  extern __shared__ double sm[];  // a.nk * RM_RB * p
  int64_t r0 = (int64_t)blockIdx.x * RM_RB;
  int nr = (int)min((int64_t)RM_RB, n - r0);
  for (int k = 0; k < a.nk; ++k)
    for (int e = threadIdx.x; e < nr * p; e += blockDim.x)
      sm[k * RM_RB * p + e] = a.U[k][r0 * p + e];
  double ev[RM_RB * 128 / 64];  // elementwise values read before the barrier
  int cnt = 0;
  for (int e = threadIdx.x; e < nr * p; e += blockDim.x, ++cnt) {
    double s = 0.0;
    for (int m = 0; m < a.ne; ++m) s = fma(a.c[m], a.E[m][r0 * p + e], s);
    ev[cnt] = s;
  }
  __syncthreads();
  cnt = 0;
  for (int e = threadIdx.x; e < nr * p; e += blockDim.x, ++cnt) {
    int rr = e / p, j = e - rr * p;
    double s = ev[cnt];
    for (int k = 0; k < a.nk; ++k) {
      const double* u = sm + k * RM_RB * p + rr * p;
      const double* M = a.M[k];
      double t = 0.0;
      for (int l = 0; l < p; ++l) t = fma(u[l], __ldg(M + l * p + j), t);
      s = fma(a.s[k], t, s);
    }
    out[r0 * p + e] = s;
  }
}

gsi_status rowmul(int64_t n, int p, const RowMulArgs& a, double* out, cudaStream_t st) {
  if (n <= 0) return GSI_OK;
  const int threads = 64;  // RM_RB * p / threads <= 16 values per thread for p <= 128
  size_t smem = (size_t)std::max(1, a.nk) * RM_RB * p * sizeof(double);
  rowmul_kernel<<<ceil_div(n, RM_RB), threads, smem, st>>>(n, p, a, out);
  GSI_LAUNCH_CHECK();
  return GSI_OK;
}

// ---------------------------------------------------------------------------
// Frobenius inner products <A0, B0>, <A1, B1> and the matrix infinity norm
// max_r sum_j |R[r, j]| in one pass; results in out[0..2]. Deterministic
// two-stage reduction (per-block partials, then a fixed-order sum).
// ---------------------------------------------------------------------------
__global__ void dots_partial_kernel(int64_t n, int p, int ndots, const double* A0,
                                    const double* B0, const double* A1, const double* B1,
                                    const double* Rn, int64_t rpb, double* part) {
  __shared__ double red[3][256];
  double s0 = 0.0, s1 = 0.0, mx = 0.0;
  int64_t r0 = (int64_t)blockIdx.x * rpb, r1 = min(n, r0 + rpb);
  for (int64_t e = r0 * p + threadIdx.x; e < r1 * p; e += blockDim.x) {
    if (ndots > 0) s0 = fma(A0[e], B0[e], s0);
    if (ndots > 1) s1 = fma(A1[e], B1[e], s1);
  }
  if (Rn) {
    for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
      double rs = 0.0;
      for (int j = 0; j < p; ++j) rs += fabs(Rn[r * p + j]);
      mx = fmax(mx, rs);
    }
  }
  red[0][threadIdx.x] = s0;
  red[1][threadIdx.x] = s1;
  red[2][threadIdx.x] = mx;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      red[0][threadIdx.x] += red[0][threadIdx.x + w];
      red[1][threadIdx.x] += red[1][threadIdx.x + w];
      red[2][threadIdx.x] = fmax(red[2][threadIdx.x], red[2][threadIdx.x + w]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[blockIdx.x * 3 + 0] = red[0][0];
    part[blockIdx.x * 3 + 1] = red[1][0];
    part[blockIdx.x * 3 + 2] = red[2][0];
  }
}

__global__ void dots_final_kernel(int nb, const double* part, double* out) {
  if (threadIdx.x != 0) return;
  double s0 = 0.0, s1 = 0.0, mx = 0.0;
  for (int b = 0; b < nb; ++b) {
    s0 += part[b * 3 + 0];
    s1 += part[b * 3 + 1];
    mx = fmax(mx, part[b * 3 + 2]);
  }
  out[0] = s0;
  out[1] = s1;
  out[2] = mx;
}

int dots_blocks(int64_t n) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sm_count() * 4, (n + 63) / 64));
}

gsi_status dots(int64_t n, int p, int ndots, const double* A0, const double* B0,
                const double* A1, const double* B1, const double* Rnorm, double* out,
                double* scratch, cudaStream_t st) {
  int nb = dots_blocks(n);
  int64_t rpb = (n + nb - 1) / nb;
  dots_partial_kernel<<<nb, 256, 0, st>>>(n, p, ndots, A0, B0, A1, B1, Rnorm, rpb, scratch);
  GSI_LAUNCH_CHECK();
  dots_final_kernel<<<1, 32, 0, st>>>(nb, scratch, out);
  GSI_LAUNCH_CHECK();
  return GSI_OK;
}

// ---------------------------------------------------------------------------
// p x p float64 helpers spread over many blocks (one thread per output):
//   out = alpha * A B + beta * E      (pp_gemm; E may be null)
//   out = a * X + b * Y               (pp_axpby)
// ---------------------------------------------------------------------------
__global__ void pp_gemm_kernel(int p, double alpha, const double* A, const double* B, double beta,
                               const double* E, double* out) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= p * p) return;
  int i = e / p, j = e - i * p;
  double s = 0.0;
  for (int k = 0; k < p; ++k) s = fma(A[i * p + k], B[k * p + j], s);
  double v = alpha * s;
  if (E) v = fma(beta, E[e], v);
  out[e] = v;
}

__global__ void pp_axpby_kernel(int p, double a, const double* X, double b, const double* Y,
                                double* out) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= p * p) return;
  out[e] = a * X[e] + (Y ? b * Y[e] : 0.0);
}

// Dense W = A X (A n x n row-major, X n x p): 64 x 64 output tiles, K staged
// through shared memory 32 at a time, a 4 x 4 register tile per thread.
__global__ void dense_gemm_kernel(int64_t n, int p, const double* __restrict__ A,
                                  const double* __restrict__ X, double* __restrict__ W) {
  __shared__ double As[64][33];
  __shared__ double Xs[32][65];
  const int64_t r0 = (int64_t)blockIdx.x * 64;
  const int c0 = blockIdx.y * 64;
  const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
  double acc[4][4] = {};
  for (int64_t k0 = 0; k0 < n; k0 += 32) {
    for (int e = threadIdx.x; e < 64 * 32; e += 256) {
      int r = e / 32, k = e % 32;
      As[r][k] = (r0 + r < n && k0 + k < n) ? A[(r0 + r) * n + k0 + k] : 0.0;
      int kk = e / 64, cc = e % 64;
      Xs[kk][cc] = (k0 + kk < n && c0 + cc < p) ? X[(k0 + kk) * p + c0 + cc] : 0.0;
    }
    __syncthreads();
    for (int k = 0; k < 32; ++k) {
      double a[4], x[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[ty * 4 + i][k];
#pragma unroll
      for (int j = 0; j < 4; ++j) x[j] = Xs[k][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], x[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int64_t r = r0 + ty * 4 + i;
      int c = c0 + tx * 4 + j;
      if (r < n && c < p) W[r * p + c] = acc[i][j];
    }
}

gsi_status dense_gemm(int64_t n, int p, const double* A, const double* X, double* W, cudaStream_t st) {
  if (n <= 0) return GSI_OK;
  dim3 grid(ceil_div(n, 64), ceil_div(p, 64));
  dense_gemm_kernel<<<grid, 256, 0, st>>>(n, p, A, X, W);
  GSI_LAUNCH_CHECK();
  return GSI_OK;
}

__global__ void dense_absmax_kernel(int64_t n, const double* A, unsigned long long* out) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  double s = 0.0;
  for (int64_t k = 0; k < n; ++k) s += fabs(A[r * n + k]);
  atomicMax(out, (unsigned long long)__double_as_longlong(s));
}

gsi_status dense_absmax(int64_t n, const double* A, unsigned long long* out, cudaStream_t st) {
  dense_absmax_kernel<<<ceil_div(n, 128), 128, 0, st>>>(n, A, out);
  GSI_LAUNCH_CHECK();
  return GSI_OK;
}

__global__ void combine3_kernel(int64_t count, double a, const double* W, double b, const double* Z,
                                double e, const double* Zp, double* out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  double v = a * W[i] + b * Z[i];
  if (Zp) v += e * Zp[i];
  out[i] = v;
}

gsi_status combine3(int64_t count, double a, const double* W, double b, const double* Z, double e,
                    const double* Zp, double* out, cudaStream_t st) {
  if (count <= 0) return GSI_OK;
  combine3_kernel<<<ceil_div(count, 256), 256, 0, st>>>(count, a, W, b, Z, e, Zp, out);
  GSI_LAUNCH_CHECK();
  return GSI_OK;
}

gsi_status pp_gemm(int p, double alpha, const double* A, const double* B, double beta,
                   const double* E, double* out, cudaStream_t st) {
  pp_gemm_kernel<<<ceil_div(p * p, 64), 64, 0, st>>>(p, alpha, A, B, beta, E, out);
  GSI_LAUNCH_CHECK();
  return GSI_OK;
}

gsi_status pp_axpby(int p, double a, const double* X, double b, const double* Y, double* out,
                    cudaStream_t st) {
  pp_axpby_kernel<<<ceil_div(p * p, 256), 256, 0, st>>>(p, a, X, b, Y, out);
  GSI_LAUNCH_CHECK();
  return GSI_OK;
}

}  // namespace gsi
