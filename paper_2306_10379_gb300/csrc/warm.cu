// Learned warm start: a multilayer perceptron maps the 16 coefficients of a
// diffusion operator to a coarse basis C (m = nc^2 rows, p columns); the
// start block is its bilinear prolongation P C to the fine grid. Training
// minimises the subspace loss L = p - tr(N^{-1} Q), N = C^T S C, S = P^T P,
// Q = C^T Bt Bt^T C, Bt = P^T U against the plain method's converged bases U.
// The paper motivates starting subspace iterations from related problems but
// gives no network; everything here is the project's own.
//
// Kernels: a bfloat16 tensor-core GEMM (mma.sync m16n8k16, float32
// accumulation) with bias / ReLU / ReLU-mask epilogues for the three layers
// forward and backward; column sums for the bias gradients; the per-sample
// loss and its analytic gradient; Adam; prolongation and restriction.
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "common.cuh"

namespace gsi {
namespace {

constexpr int GBM = 64, GBN = 64, GBK = 32, GPAD = 8;

__device__ __forceinline__ void mma_bf16_16816(float c[4], const uint32_t a[4], const uint32_t b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// C[i][j] = alpha sum_k A(i,k) B(k,j) + beta C[i][j] (+ bias[j]); then, if
// mask: C = 0 where mask[i][j] <= 0; if relu: C = max(C, 0). A(i,k) =
// A[i*sai + k*sak], B(k,j) = B[k*sbk + j*sbj]; operands rounded to
// bfloat16 (nearest even) when staged, products summed in float32.
// Block 64 x 64, 4 warps of 32 x 32, K steps of 32.
__global__ void __launch_bounds__(128) gemm_bf16_kernel(int M, int N, int K, const float* __restrict__ A,
                                                        int64_t sai, int64_t sak, const float* __restrict__ B,
                                                        int64_t sbk, int64_t sbj, float* __restrict__ C,
                                                        int64_t ldc, float alpha, float beta,
                                                        const float* __restrict__ bias,
                                                        const float* __restrict__ mask, int relu) {
  __shared__ __align__(16) __nv_bfloat16 As[GBM][GBK + GPAD];
  __shared__ __align__(16) __nv_bfloat16 Bs[GBN][GBK + GPAD];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp >> 1, wn = warp & 1, g = lane >> 2, t = lane & 3;
  const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
  float acc[2][4][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
  for (int k0 = 0; k0 < K; k0 += GBK) {
    // stage 64 x 32 of A (rows i, columns k) and 32 x 64 of B as [j][k]
    // consecutive threads walk the operand's contiguous index
    for (int e = tid; e < GBM * GBK; e += 128) {
      int i, k;
      if (sai == 1) {
        i = e % GBM;
        k = e / GBM;
      } else {
        i = e / GBK;
        k = e - i * GBK;
      }
      const int gi = m0 + i, gk = k0 + k;
      const float v = (gi < M && gk < K) ? A[gi * sai + gk * sak] : 0.f;
      As[i][k] = __float2bfloat16_rn(v);
    }
    for (int e = tid; e < GBN * GBK; e += 128) {
      int j, k;
      if (sbj == 1) {
        j = e % GBN;
        k = e / GBN;
      } else {
        j = e / GBK;
        k = e - j * GBK;
      }
      const int gj = n0 + j, gk = k0 + k;
      const float v = (gj < N && gk < K) ? B[gk * sbk + gj * sbj] : 0.f;
      Bs[j][k] = __float2bfloat16_rn(v);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GBK; kk += 16) {
      uint32_t af[2][4], bfr[4][2];
#pragma unroll
      for (int mi = 0; mi < 2; ++mi) {
        const int r = wm * 32 + mi * 16 + g;
        af[mi][0] = *reinterpret_cast<const uint32_t*>(&As[r][kk + 2 * t]);
        af[mi][1] = *reinterpret_cast<const uint32_t*>(&As[r + 8][kk + 2 * t]);
        af[mi][2] = *reinterpret_cast<const uint32_t*>(&As[r][kk + 2 * t + 8]);
        af[mi][3] = *reinterpret_cast<const uint32_t*>(&As[r + 8][kk + 2 * t + 8]);
      }
#pragma unroll
      for (int ni = 0; ni < 4; ++ni) {
        const int c = wn * 32 + ni * 8 + g;
        bfr[ni][0] = *reinterpret_cast<const uint32_t*>(&Bs[c][kk + 2 * t]);
        bfr[ni][1] = *reinterpret_cast<const uint32_t*>(&Bs[c][kk + 2 * t + 8]);
      }
#pragma unroll
      for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni) mma_bf16_16816(acc[mi][ni], af[mi], bfr[ni]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int mi = 0; mi < 2; ++mi) {
#pragma unroll
    for (int ni = 0; ni < 4; ++ni) {
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int i = m0 + wm * 32 + mi * 16 + g + (r >= 2 ? 8 : 0);
        const int j = n0 + wn * 32 + ni * 8 + 2 * t + (r & 1);
        if (i >= M || j >= N) continue;
        const int64_t o = (int64_t)i * ldc + j;
        float v = alpha * acc[mi][ni][r];
        if (beta != 0.f) v += beta * C[o];
        if (bias) v += bias[j];
        if (mask && !(mask[o] > 0.f)) v = 0.f;
        if (relu) v = fmaxf(v, 0.f);
        C[o] = v;
      }
    }
  }
}

// out[j] = sum_i G[i][j] (rows in order)
__global__ void colsum_kernel(int rows, int cols, const float* __restrict__ G, float* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= cols) return;
  float s = 0.f;
  for (int i = 0; i < rows; ++i) s += G[(int64_t)i * cols + j];
  out[j] = s;
}

// Adam (Kingma & Ba 2015): c1 = 1 / (1 - b1^t), c2 = 1 / (1 - b2^t)
__global__ void adam_kernel(int64_t count, float* __restrict__ w, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  w[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
}

// hat-function weights of fine node f (0-based) against coarse nodes: the
// two neighbours a0, a0 + 1 with weights w0, w1 (absent ones get weight 0)
__device__ __forceinline__ void hat(int f, int nc, int nf, int& a0, double& w0, double& w1) {
  const double tx = (double)(f + 1) * (nc + 1) / (nf + 1) - 1.0;
  a0 = (int)floor(tx);
  w1 = tx - a0;
  w0 = 1.0 - w1;
}

// X[s] (nf^2 x p, float64) = P C[s] (C: nc^2 x p, float32), P = P1 (x) P1
__global__ void prolong_kernel(int nc, int nf, int p, int batch, const float* __restrict__ C,
                               double* __restrict__ X) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t per = (int64_t)nf * nf * p;
  if (idx >= per * batch) return;
  const int s = (int)(idx / per);
  const int64_t e = idx - s * per;
  const int r = (int)(e / p), c = (int)(e - (int64_t)r * p);
  const int i = r % nf, j = r / nf;
  int ax, ay;
  double wx[2], wy[2];
  hat(i, nc, nf, ax, wx[0], wx[1]);
  hat(j, nc, nf, ay, wy[0], wy[1]);
  const float* Cs = C + (int64_t)s * nc * nc * p;
  double v = 0.0;
  for (int db = 0; db < 2; ++db) {
    const int b = ay + db;
    if (b < 0 || b >= nc) continue;
    for (int da = 0; da < 2; ++da) {
      const int a = ax + da;
      if (a < 0 || a >= nc) continue;
      v += wy[db] * wx[da] * (double)Cs[(a + nc * b) * p + c];
    }
  }
  X[idx] = v;
}

// Bt[s] (nc^2 x p, float32) = P^T U[s] (U: nf^2 x p, float64): coarse node
// a gathers the fine nodes inside its hat's support
__global__ void restrict_kernel(int nc, int nf, int p, int batch, const double* __restrict__ U,
                                float* __restrict__ Bt) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t per = (int64_t)nc * nc * p;
  if (idx >= per * batch) return;
  const int s = (int)(idx / per);
  const int64_t e = idx - s * per;
  const int rc = (int)(e / p), c = (int)(e - (int64_t)rc * p);
  const int a = rc % nc, b = rc / nc;
  // fine nodes with |x_f - x_c| < 1/(nc+1): (i+1)/(nf+1) in (a/(nc+1), (a+2)/(nc+1))
  const int lo_a = max(0, (int)floor((double)a * (nf + 1) / (nc + 1)) - 1);
  const int hi_a = min(nf - 1, (int)ceil((double)(a + 2) * (nf + 1) / (nc + 1)));
  const int lo_b = max(0, (int)floor((double)b * (nf + 1) / (nc + 1)) - 1);
  const int hi_b = min(nf - 1, (int)ceil((double)(b + 2) * (nf + 1) / (nc + 1)));
  const double* Us = U + (int64_t)s * nf * nf * p;
  double v = 0.0;
  for (int j = lo_b; j <= hi_b; ++j) {
    const double wy = fmax(0.0, 1.0 - fabs((double)(j + 1) * (nc + 1) / (nf + 1) - (b + 1)));
    if (wy == 0.0) continue;
    for (int i = lo_a; i <= hi_a; ++i) {
      const double wx = fmax(0.0, 1.0 - fabs((double)(i + 1) * (nc + 1) / (nf + 1) - (a + 1)));
      if (wx == 0.0) continue;
      v += wx * wy * Us[(int64_t)(i + nf * j) * p + c];
    }
  }
  Bt[idx] = (float)v;
}

// One block per sample s: with C = C[s] (m x p), Bt = Bt[s] (m x p),
//   SC = S C; N = C^T SC (symmetrised); G = Bt^T C; Q = G^T G;
//   loss[s] = p - tr(N^{-1} Q);
//   dC[s] = gscale * (-2) [Bt (G N^{-1}) - SC (N^{-1} Q N^{-1})].
// Long sums in float32 over 32-row chunks, chunk sums and the p x p algebra
// in float64 (N^{-1} from its Cholesky factor). A non-positive pivot gives
// loss = NaN and dC = 0. Dynamic shared memory: 5 p^2 doubles + 2 p^2 floats.
constexpr int WT = 256;

__global__ void __launch_bounds__(WT) warm_loss_kernel(int m, int p, const int64_t* __restrict__ Srp,
                                                       const int32_t* __restrict__ Sci,
                                                       const double* __restrict__ Sv,
                                                       const float* __restrict__ Call,
                                                       const float* __restrict__ Btall,
                                                       float* __restrict__ SCall, double* __restrict__ loss,
                                                       float* __restrict__ dCall, float gscale) {
  extern __shared__ __align__(16) double wsm[];
  __shared__ int bad;
  __shared__ double trace;
  const int s = blockIdx.x, tid = threadIdx.x, q = p * p;
  const int64_t off = (int64_t)s * m * p;
  const float* C = Call + off;
  const float* Bt = Btall + off;
  float* SC = SCall + off;
  float* dC = dCall + off;
  double* Nm = wsm;       // N, then its Cholesky factor L (lower)
  double* Gm = Nm + q;    // G, then G N^{-1}
  double* Qm = Gm + q;    // Q
  double* Ni = Qm + q;    // L^{-1}, then N^{-1}
  double* Tm = Ni + q;    // scratch
  float* A1 = reinterpret_cast<float*>(Tm + q);  // G N^{-1}
  float* A2 = A1 + q;                            // N^{-1} Q N^{-1}
  if (tid == 0) bad = 0;
  // SC = S C
  for (int e = tid; e < m * p; e += WT) {
    const int r = e / p, c = e - r * p;
    double a = 0.0;
    for (int64_t k = Srp[r]; k < Srp[r + 1]; ++k) a += Sv[k] * (double)C[(int64_t)Sci[k] * p + c];
    SC[e] = (float)a;
  }
  __syncthreads();
  // N = C^T SC and G = Bt^T C
  for (int e = tid; e < 2 * q; e += WT) {
    const int which = e / q, rem = e - which * q, i = rem / p, j = rem - i * p;
    const float* U = which == 0 ? C : Bt;
    const float* V = which == 0 ? SC : C;
    double tot = 0.0;
    for (int r0 = 0; r0 < m; r0 += 32) {
      float a = 0.f;
      const int r1 = min(m, r0 + 32);
      for (int r = r0; r < r1; ++r) a = fmaf(U[(int64_t)r * p + i], V[(int64_t)r * p + j], a);
      tot += (double)a;
    }
    (which == 0 ? Nm : Gm)[rem] = tot;
  }
  __syncthreads();
  for (int e = tid; e < q; e += WT) {  // symmetrise N; Q = G^T G
    const int i = e / p, j = e - i * p;
    double a = 0.0;
    for (int k = 0; k < p; ++k) a = fma(Gm[k * p + i], Gm[k * p + j], a);
    Qm[e] = a;
    Tm[e] = 0.5 * (Nm[e] + Nm[j * p + i]);
  }
  __syncthreads();
  for (int e = tid; e < q; e += WT) Nm[e] = Tm[e];
  __syncthreads();
  // Cholesky N = L L^T (right-looking, column k by the block)
  for (int k = 0; k < p; ++k) {
    if (tid == 0) {
      const double d = Nm[k * p + k];
      if (!(d > 0.0) || !isfinite(d)) bad = 1;
      Nm[k * p + k] = d > 0.0 ? sqrt(d) : 1.0;
    }
    __syncthreads();
    const double lkk = Nm[k * p + k];
    for (int i = k + 1 + tid; i < p; i += WT) Nm[i * p + k] /= lkk;
    __syncthreads();
    for (int e = tid; e < (p - k - 1) * (p - k - 1); e += WT) {
      const int i = k + 1 + e / (p - k - 1), j = k + 1 + e % (p - k - 1);
      if (j <= i) Nm[i * p + j] -= Nm[i * p + k] * Nm[j * p + k];
    }
    __syncthreads();
  }
  // L^{-1} by forward substitution, one column per thread
  for (int c = tid; c < p; c += WT) {
    for (int i = 0; i < p; ++i) {
      double v = (i == c) ? 1.0 : 0.0;
      for (int k = c; k < i; ++k) v -= Nm[i * p + k] * Ni[k * p + c];
      Ni[i * p + c] = i < c ? 0.0 : v / Nm[i * p + i];
    }
  }
  __syncthreads();
  // N^{-1} = L^{-T} L^{-1}
  for (int e = tid; e < q; e += WT) {
    const int i = e / p, j = e - i * p;
    double a = 0.0;
    for (int k = max(i, j); k < p; ++k) a = fma(Ni[k * p + i], Ni[k * p + j], a);
    Tm[e] = a;
  }
  __syncthreads();
  for (int e = tid; e < q; e += WT) Ni[e] = Tm[e];
  __syncthreads();
  // T = N^{-1} Q; G <- G N^{-1} (into A1 as float)
  for (int e = tid; e < q; e += WT) {
    const int i = e / p, j = e - i * p;
    double a = 0.0, b = 0.0;
    for (int k = 0; k < p; ++k) {
      a = fma(Ni[i * p + k], Qm[k * p + j], a);
      b = fma(Gm[i * p + k], Ni[k * p + j], b);
    }
    Tm[e] = a;
    A1[e] = (float)b;
  }
  __syncthreads();
  if (tid == 0) {
    double tr = 0.0;
    for (int k = 0; k < p; ++k) tr += Tm[k * p + k];
    trace = tr;
  }
  // A2 = T N^{-1}
  for (int e = tid; e < q; e += WT) {
    const int i = e / p, j = e - i * p;
    double a = 0.0;
    for (int k = 0; k < p; ++k) a = fma(Tm[i * p + k], Ni[k * p + j], a);
    A2[e] = (float)a;
  }
  __syncthreads();
  const bool ok = !bad;
  if (tid == 0) loss[s] = ok ? (double)p - trace : NAN;
  const float sc = -2.f * gscale;
  for (int e = tid; e < m * p; e += WT) {
    const int r = e / p, c = e - r * p;
    float a = 0.f;
    for (int k = 0; k < p; ++k) a = fmaf(Bt[(int64_t)r * p + k], A1[k * p + c], a);
    for (int k = 0; k < p; ++k) a = fmaf(-SC[(int64_t)r * p + k], A2[k * p + c], a);
    dC[e] = ok ? sc * a : 0.f;
  }
}

size_t warm_smem(int p) { return (size_t)5 * p * p * sizeof(double) + (size_t)2 * p * p * sizeof(float); }

}  // namespace
}  // namespace gsi

using namespace gsi;

// parameters, flat: W1 (hid x din), b1, W2 (hid x hid), b2, W3 (dout x hid), b3
struct gsi_mlp {
  int din = 0, hid = 0, dout = 0, max_batch = 0;
  int64_t np = 0, step = 0;
  cudaStream_t st = nullptr;
  float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  float *h1 = nullptr, *h2 = nullptr, *out = nullptr, *d1 = nullptr, *d2 = nullptr, *dout_buf = nullptr;
  float* sc_buf = nullptr;
  double* loss = nullptr;
  double* hloss = nullptr;  // pinned
  std::vector<void*> allocs;
  float* W1() const { return w; }
  float* b1() const { return w + (int64_t)hid * din; }
  float* W2() const { return b1() + hid; }
  float* b2() const { return W2() + (int64_t)hid * hid; }
  float* W3() const { return b2() + hid; }
  float* b3() const { return W3() + (int64_t)dout * hid; }
  // the same offsets into the gradient
  float* gof(const float* p) const { return g + (p - w); }
};

namespace {

gsi_status gemm(cudaStream_t st, int M, int N, int K, const float* A, int64_t sai, int64_t sak,
                const float* B, int64_t sbk, int64_t sbj, float* C, int64_t ldc, float alpha, float beta,
                const float* bias, const float* mask, int relu) {
  if (M <= 0 || N <= 0) return GSI_OK;
  dim3 grid((unsigned)((N + GBN - 1) / GBN), (unsigned)((M + GBM - 1) / GBM));
  gemm_bf16_kernel<<<grid, 128, 0, st>>>(M, N, K, A, sai, sak, B, sbk, sbj, C, ldc, alpha, beta, bias,
                                         mask, relu);
  GSI_LAUNCH_CHECK();
  return GSI_OK;
}

gsi_status malloc_t(gsi_mlp* n, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 256));
  if (e != cudaSuccess) return cuda_status(e);
  n->allocs.push_back(*p);
  return GSI_OK;
}

// forward with the activations kept for backward
gsi_status mlp_forward(gsi_mlp* n, int batch, const float* x, float* out) {
  const int H = n->hid;
  GSI_TRY(gemm(n->st, batch, H, n->din, x, n->din, 1, n->W1(), 1, n->din, n->h1, H, 1.f, 0.f, n->b1(),
               nullptr, 1));
  GSI_TRY(gemm(n->st, batch, H, H, n->h1, H, 1, n->W2(), 1, H, n->h2, H, 1.f, 0.f, n->b2(), nullptr, 1));
  GSI_TRY(gemm(n->st, batch, n->dout, H, n->h2, H, 1, n->W3(), 1, H, out, n->dout, 1.f, 0.f, n->b3(),
               nullptr, 0));
  return GSI_OK;
}

// gradients of sum(out * dout) for the batch of the last forward
gsi_status mlp_backward(gsi_mlp* n, int batch, const float* x, const float* dout) {
  const int H = n->hid, D = n->dout;
  cudaStream_t st = n->st;
  // W3: dout^T h2; b3: column sums of dout
  GSI_TRY(gemm(st, D, H, batch, dout, 1, D, n->h2, H, 1, n->gof(n->W3()), H, 1.f, 0.f, nullptr, nullptr, 0));
  colsum_kernel<<<ceil_div(D, 256), 256, 0, st>>>(batch, D, dout, n->gof(n->b3()));
  GSI_LAUNCH_CHECK();
  // d2 = (dout W3) o [h2 > 0]
  GSI_TRY(gemm(st, batch, H, D, dout, D, 1, n->W3(), H, 1, n->d2, H, 1.f, 0.f, nullptr, n->h2, 0));
  GSI_TRY(gemm(st, H, H, batch, n->d2, 1, H, n->h1, H, 1, n->gof(n->W2()), H, 1.f, 0.f, nullptr, nullptr, 0));
  colsum_kernel<<<ceil_div(H, 256), 256, 0, st>>>(batch, H, n->d2, n->gof(n->b2()));
  GSI_LAUNCH_CHECK();
  // d1 = (d2 W2) o [h1 > 0]
  GSI_TRY(gemm(st, batch, H, H, n->d2, H, 1, n->W2(), H, 1, n->d1, H, 1.f, 0.f, nullptr, n->h1, 0));
  GSI_TRY(gemm(st, H, n->din, batch, n->d1, 1, H, x, n->din, 1, n->gof(n->W1()), n->din, 1.f, 0.f, nullptr,
               nullptr, 0));
  colsum_kernel<<<ceil_div(H, 256), 256, 0, st>>>(batch, H, n->d1, n->gof(n->b1()));
  GSI_LAUNCH_CHECK();
  return GSI_OK;
}

gsi_status mlp_adam(gsi_mlp* n, double lr, double b1, double b2, double eps) {
  n->step++;
  const double c1 = 1.0 / (1.0 - pow(b1, (double)n->step));
  const double c2 = 1.0 / (1.0 - pow(b2, (double)n->step));
  adam_kernel<<<ceil_div(n->np, 256), 256, 0, n->st>>>(n->np, n->w, n->g, n->m, n->v, (float)lr, (float)b1,
                                                       (float)b2, (float)eps, (float)c1, (float)c2);
  GSI_LAUNCH_CHECK();
  return GSI_OK;
}

gsi_status loss_grad(int batch, int m, int p, const int64_t* Srp, const int32_t* Sci, const double* Sv,
                     const float* C, const float* Bt, float* SC, double* loss, float* dC, float gscale,
                     cudaStream_t st) {
  if (batch <= 0) return GSI_OK;
  const size_t sm = warm_smem(p);  // <= 196 KB for p <= 64; with the static part above 48 KB from p = 32
  if (sm >= 32 * 1024)
    GSI_CUDA_TRY(cudaFuncSetAttribute(warm_loss_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  warm_loss_kernel<<<batch, WT, sm, st>>>(m, p, Srp, Sci, Sv, C, Bt, SC, loss, dC, gscale);
  GSI_LAUNCH_CHECK();
  return GSI_OK;
}

}  // namespace

extern "C" {

int64_t gsi_mlp_num_params(int32_t din, int32_t hidden, int32_t dout) {
  return (int64_t)hidden * din + hidden + (int64_t)hidden * hidden + hidden + (int64_t)dout * hidden + dout;
}

gsi_status gsi_mlp_destroy(gsi_mlp* n) {
  if (!n) return GSI_ERR_ARG;
  if (n->st) cudaStreamSynchronize(n->st);
  for (void* p : n->allocs) cudaFree(p);
  if (n->hloss) cudaFreeHost(n->hloss);
  delete n;
  return GSI_OK;
}

gsi_status gsi_mlp_create(int32_t din, int32_t hidden, int32_t dout, int32_t max_batch, const float* params,
                          void* stream, gsi_mlp** out) {
  if (!out || !params || din < 1 || hidden < 1 || dout < 1 || max_batch < 1) return GSI_ERR_ARG;
  *out = nullptr;
  gsi_mlp* n = new gsi_mlp();
  n->din = din;
  n->hid = hidden;
  n->dout = dout;
  n->max_batch = max_batch;
  n->st = (cudaStream_t)stream;
  n->np = gsi_mlp_num_params(din, hidden, dout);
  const size_t pb = (size_t)n->np * sizeof(float);
  const size_t hb = (size_t)max_batch * hidden * sizeof(float);
  const size_t ob = (size_t)max_batch * dout * sizeof(float);
  gsi_status s = GSI_OK;
#define CK(expr)                \
  do {                          \
    s = (expr);                 \
    if (s != GSI_OK) goto fail; \
  } while (0)
  CK(malloc_t(n, (void**)&n->w, pb));
  CK(malloc_t(n, (void**)&n->g, pb));
  CK(malloc_t(n, (void**)&n->m, pb));
  CK(malloc_t(n, (void**)&n->v, pb));
  CK(malloc_t(n, (void**)&n->h1, hb));
  CK(malloc_t(n, (void**)&n->h2, hb));
  CK(malloc_t(n, (void**)&n->d1, hb));
  CK(malloc_t(n, (void**)&n->d2, hb));
  CK(malloc_t(n, (void**)&n->out, ob));
  CK(malloc_t(n, (void**)&n->dout_buf, ob));
  CK(malloc_t(n, (void**)&n->sc_buf, ob));
  CK(malloc_t(n, (void**)&n->loss, (size_t)max_batch * sizeof(double)));
  CK(cuda_status_ok(cudaMallocHost((void**)&n->hloss, (size_t)max_batch * sizeof(double))));
  CK(cuda_status_ok(cudaMemcpy(n->w, params, pb, cudaMemcpyHostToDevice)));
  CK(cuda_status_ok(cudaMemset(n->g, 0, pb)));
  CK(cuda_status_ok(cudaMemset(n->m, 0, pb)));
  CK(cuda_status_ok(cudaMemset(n->v, 0, pb)));
#undef CK
  *out = n;
  return GSI_OK;
fail:
  gsi_mlp_destroy(n);
  return s;
}

gsi_status gsi_mlp_get_params(gsi_mlp* n, float* params, float* grads) {
  if (!n) return GSI_ERR_ARG;
  GSI_CUDA_TRY(cudaStreamSynchronize(n->st));
  if (params) GSI_CUDA_TRY(cudaMemcpy(params, n->w, (size_t)n->np * sizeof(float), cudaMemcpyDeviceToHost));
  if (grads) GSI_CUDA_TRY(cudaMemcpy(grads, n->g, (size_t)n->np * sizeof(float), cudaMemcpyDeviceToHost));
  return GSI_OK;
}

gsi_status gsi_mlp_forward(gsi_mlp* n, int32_t batch, const float* x, float* out) {
  if (!n || !x || !out || batch < 1 || batch > n->max_batch) return GSI_ERR_ARG;
  return mlp_forward(n, batch, x, out);
}

gsi_status gsi_mlp_backward(gsi_mlp* n, int32_t batch, const float* x, const float* dout) {
  if (!n || !x || !dout || batch < 1 || batch > n->max_batch) return GSI_ERR_ARG;
  return mlp_backward(n, batch, x, dout);
}

gsi_status gsi_mlp_adam(gsi_mlp* n, double lr, double beta1, double beta2, double eps) {
  if (!n || !(lr > 0.0)) return GSI_ERR_ARG;
  return mlp_adam(n, lr, beta1, beta2, eps);
}

gsi_status gsi_warm_loss_grad(int32_t batch, int32_t m, int32_t p, const int64_t* S_rowptr,
                              const int32_t* S_colidx, const double* S_val, const float* C, const float* Bt,
                              float* SC_scratch, double* loss, float* dC, float gscale, void* stream) {
  if (batch < 1 || m < 1 || p < 1 || p > 64 || !S_rowptr || !S_colidx || !S_val || !C || !Bt ||
      !SC_scratch || !loss || !dC)
    return GSI_ERR_ARG;
  return loss_grad(batch, m, p, S_rowptr, S_colidx, S_val, C, Bt, SC_scratch, loss, dC, gscale,
                   (cudaStream_t)stream);
}

gsi_status gsi_warm_train_step(gsi_mlp* n, int32_t batch, const float* x, int32_t m, int32_t p,
                               const int64_t* S_rowptr, const int32_t* S_colidx, const double* S_val,
                               const float* Bt, double lr, double* mean_loss) {
  if (!n || !x || !Bt || batch < 1 || batch > n->max_batch || p < 1 || p > 64 || (int64_t)m * p != n->dout)
    return GSI_ERR_ARG;
  GSI_TRY(mlp_forward(n, batch, x, n->out));
  GSI_TRY(loss_grad(batch, m, p, S_rowptr, S_colidx, S_val, n->out, Bt, n->sc_buf, n->loss, n->dout_buf,
                    1.f / batch, n->st));
  GSI_TRY(mlp_backward(n, batch, x, n->dout_buf));
  GSI_TRY(mlp_adam(n, lr, 0.9, 0.999, 1e-8));
  if (mean_loss) {
    GSI_CUDA_TRY(cudaMemcpyAsync(n->hloss, n->loss, (size_t)batch * sizeof(double), cudaMemcpyDeviceToHost,
                                 n->st));
    GSI_CUDA_TRY(cudaStreamSynchronize(n->st));
    double s = 0.0;
    for (int i = 0; i < batch; ++i) s += n->hloss[i];
    *mean_loss = s / batch;
  }
  return GSI_OK;
}

gsi_status gsi_prolong(int32_t nc, int32_t nf, int32_t p, int32_t batch, const float* C, double* X,
                       void* stream) {
  if (nc < 1 || nf < 1 || p < 1 || batch < 1 || !C || !X) return GSI_ERR_ARG;
  const int64_t total = (int64_t)batch * nf * nf * p;
  prolong_kernel<<<ceil_div(total, 256), 256, 0, (cudaStream_t)stream>>>(nc, nf, p, batch, C, X);
  GSI_LAUNCH_CHECK();
  return GSI_OK;
}

gsi_status gsi_restrict(int32_t nc, int32_t nf, int32_t p, int32_t batch, const double* U, float* Bt,
                        void* stream) {
  if (nc < 1 || nf < 1 || p < 1 || batch < 1 || !U || !Bt) return GSI_ERR_ARG;
  const int64_t total = (int64_t)batch * nc * nc * p;
  restrict_kernel<<<ceil_div(total, 256), 256, 0, (cudaStream_t)stream>>>(nc, nf, p, batch, U, Bt);
  GSI_LAUNCH_CHECK();
  return GSI_OK;
}

gsi_status gsi_gemm_bf16(int32_t M, int32_t N, int32_t K, const float* A, int64_t sai, int64_t sak,
                         const float* B, int64_t sbk, int64_t sbj, float* C, int64_t ldc, float alpha,
                         float beta, const float* bias, const float* mask, int32_t relu, void* stream) {
  if (M < 0 || N < 0 || K < 0 || !A || !B || !C) return GSI_ERR_ARG;
  return gemm((cudaStream_t)stream, M, N, K, A, sai, sak, B, sbk, sbj, C, ldc, alpha, beta, bias, mask, relu);
}

}  // extern "C"
