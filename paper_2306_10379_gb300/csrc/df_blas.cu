// df64 block kernels run on the float32 pipes: the block matvec (CSR and
// SELL-C-sigma SpMM, the one operator apply per iteration of Sec. 6.1),
// Frobenius inner products, axpby and the float64 <-> df64 conversions used
// at the API boundary.
#include <algorithm>

#include "df.cuh"
#include "oz.cuh"

namespace gsi {

__global__ void f64_to_df_kernel(int64_t count, const double* __restrict__ x, float2* __restrict__ y) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) y[i] = df_from_double(x[i]);
}

__global__ void df_to_f64_kernel(int64_t count, const float2* __restrict__ x, double* __restrict__ y) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) y[i] = df_to_double(x[i]);
}

gsi_status df_from_f64(int64_t count, const double* x, float2* y, cudaStream_t st) {
  if (count <= 0) return GSI_OK;
  f64_to_df_kernel<<<ceil_div(count, 256), 256, 0, st>>>(count, x, y);
  GSI_LAUNCH_CHECK();
  return GSI_OK;
}

gsi_status df_to_f64(int64_t count, const float2* x, double* y, cudaStream_t st) {
  if (count <= 0) return GSI_OK;
  df_to_f64_kernel<<<ceil_div(count, 256), 256, 0, st>>>(count, x, y);
  GSI_LAUNCH_CHECK();
  return GSI_OK;
}

// acc (sh + se) += a * x with a, x df64: the leading product is split exactly
// (TwoProd) and added exactly (TwoSum); all second-order terms go to se.
__device__ __forceinline__ void df_mac(float& sh, float& se, float2 a, float2 x) {
  float p = __fmul_rn(a.x, x.x);
  float pe = __fmaf_rn(a.x, x.x, -p);
  float2 t = two_sum(sh, p);
  sh = t.x;
  se = __fadd_rn(se, __fadd_rn(t.y, __fmaf_rn(a.x, x.y, __fmaf_rn(a.y, x.x, pe))));
}

// W = A X, CSR; thread <-> (row, pair of columns) with 16-byte loads of two
// df64 entries of the gathered X row.
template <bool VEC2>
__global__ void df_spmm_csr_kernel(int64_t n, const int64_t* __restrict__ rowptr,
                                   const int32_t* __restrict__ colidx,
                                   const float2* __restrict__ val, int p, int cpr,
                                   const float2* __restrict__ X, float2* __restrict__ W) {
  int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t row = gid / cpr;
  int c = (int)(gid - row * cpr);
  if (row >= n) return;
  int64_t b = __ldg(rowptr + row), e = __ldg(rowptr + row + 1);
  if (VEC2) {
    float h0 = 0.f, e0 = 0.f, h1 = 0.f, e1 = 0.f;
    for (int64_t k = b; k < e; ++k) {
      float2 a = __ldg(val + k);
      int64_t col = __ldg(colidx + k);
      float4 x = __ldg(reinterpret_cast<const float4*>(X + col * p) + c);
      df_mac(h0, e0, a, make_float2(x.x, x.y));
      df_mac(h1, e1, a, make_float2(x.z, x.w));
    }
    float2 r0 = fast_two_sum(h0, e0), r1 = fast_two_sum(h1, e1);
    reinterpret_cast<float4*>(W + row * p)[c] = make_float4(r0.x, r0.y, r1.x, r1.y);
  } else {
    float h0 = 0.f, e0 = 0.f;
    for (int64_t k = b; k < e; ++k) {
      float2 a = __ldg(val + k);
      int64_t col = __ldg(colidx + k);
      df_mac(h0, e0, a, __ldg(X + col * p + c));
    }
    W[row * p + c] = fast_two_sum(h0, e0);
  }
}

// W = A X for even p <= 128 and 16-byte aligned blocks: a group of lpr lanes
// (a power of two, 2 lpr >= min(p, 64)) per row, lane l holding columns 2l,
// 2l + 1 (and 64 + 2l, 65 + 2l when CPL = 2). The row's nonzeros go in
// batches of 8: their column indices and values are loaded first, then the 8
// gathered X rows (16-byte loads), then the 8 multiply-adds, so that a group
// has up to 8 gathers in flight instead of one (4 rows of 2 x 16 B when
// CPL = 2). Same summation order as df_spmm_csr_kernel (k ascending), so the
// results are identical.
// SELL: rows are the slots of the SELL-C-sigma layout (entry j of slot s of
// chunk c at chunk_ptr[c] + j C + s; padding entries add exact zeros); W is
// written at the original row perm[slot].
template <int CPL, bool SELL>
__global__ void __launch_bounds__(256)
df_spmm_rows_kernel(int64_t nrows, int lpr_log2, int p, const int64_t* __restrict__ rowptr,
                    const int32_t* __restrict__ colidx, const float2* __restrict__ val, int C,
                    const int64_t* __restrict__ perm, const int64_t* __restrict__ chunk_len,
                    const float2* __restrict__ X, float2* __restrict__ W) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t r = gid >> lpr_log2;
  const int cl = (int)(gid & ((1 << lpr_log2) - 1));
  if (r >= nrows) return;
  int64_t b, orow;
  int cnt, stride;
  if (SELL) {
    orow = __ldg(perm + r);
    if (orow < 0) return;
    const int64_t ch = r / C;
    b = __ldg(rowptr + ch) + (r - ch * C);  // rowptr = chunk_ptr
    cnt = (int)__ldg(chunk_len + ch);
    stride = C;
  } else {
    orow = r;
    b = __ldg(rowptr + r);
    cnt = (int)(__ldg(rowptr + r + 1) - b);
    stride = 1;
  }
  const int32_t* ci_row = colidx + b;
  const float2* v_row = val + b;
  constexpr int NB = 8 / CPL;  // nonzeros per batch
  bool act[CPL];
#pragma unroll
  for (int c = 0; c < CPL; ++c) act[c] = 64 * c + 2 * cl < p;
  float h[2 * CPL], e[2 * CPL];
#pragma unroll
  for (int c = 0; c < 2 * CPL; ++c) h[c] = e[c] = 0.f;
  for (int k = 0; k < cnt; k += NB) {
    int ci[NB];
    float2 vv[NB];
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      ci[u] = 0;
      vv[u] = make_float2(0.f, 0.f);
      if (k + u < cnt) {
        const int idx = (k + u) * stride;
        ci[u] = __ldg(ci_row + idx);
        vv[u] = __ldg(v_row + idx);
      }
    }
    float4 xx[NB][CPL];
#pragma unroll
    for (int u = 0; u < NB; ++u)
#pragma unroll
      for (int c = 0; c < CPL; ++c) {
        xx[u][c] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (k + u < cnt && act[c])
          xx[u][c] = __ldg(reinterpret_cast<const float4*>(X + (int64_t)ci[u] * p + 64 * c) + cl);
      }
#pragma unroll
    for (int u = 0; u < NB; ++u)
      if (k + u < cnt)
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
          df_mac(h[2 * c], e[2 * c], vv[u], make_float2(xx[u][c].x, xx[u][c].y));
          df_mac(h[2 * c + 1], e[2 * c + 1], vv[u], make_float2(xx[u][c].z, xx[u][c].w));
        }
  }
#pragma unroll
  for (int c = 0; c < CPL; ++c)
    if (act[c]) {
      const float2 r0 = fast_two_sum(h[2 * c], e[2 * c]), r1 = fast_two_sum(h[2 * c + 1], e[2 * c + 1]);
      reinterpret_cast<float4*>(W + orow * p + 64 * c)[cl] = make_float4(r0.x, r0.y, r1.x, r1.y);
    }
}

// The row-group kernel serves even 64 < p <= 128 with 16-byte aligned X and W
// (a warp per row, two float4 columns per lane). Measured at 128^3: p = 128
// 1.65 ms against 1.99 ms for the column-pair kernel; for p <= 64 the column-
// pair kernel is faster (p = 64: 1.00 against 1.53 ms; p = 32: 0.52 against
// 0.79 ms), its 40 registers against ~72 keeping twice the warps resident.
static bool rows_shape(int p, const void* X, const void* W, int* lpr_log2, int* cpl) {
  if ((p & 1) || p <= 64 || p > 128 || ((uintptr_t)X & 15) || ((uintptr_t)W & 15)) return false;
  *lpr_log2 = 5;
  *cpl = 2;
  return true;
}

gsi_status df_spmm_csr(int64_t n, const int64_t* rowptr, const int32_t* colidx, const float2* val,
                       int p, const float2* X, float2* W, cudaStream_t st) {
  if (n <= 0) return GSI_OK;
  int lg = 0, cpl = 1;
  if (rows_shape(p, X, W, &lg, &cpl)) {
    const int64_t threads = n << lg;
    if (cpl == 1)
      df_spmm_rows_kernel<1, false><<<ceil_div(threads, 256), 256, 0, st>>>(n, lg, p, rowptr, colidx, val, 0,
                                                                           nullptr, nullptr, X, W);
    else
      df_spmm_rows_kernel<2, false><<<ceil_div(threads, 256), 256, 0, st>>>(n, lg, p, rowptr, colidx, val, 0,
                                                                           nullptr, nullptr, X, W);
    GSI_LAUNCH_CHECK();
    return GSI_OK;
  }
  // 16-byte loads of column pairs only from 16-byte aligned blocks
  if ((p & 1) == 0 && ((uintptr_t)X & 15) == 0 && ((uintptr_t)W & 15) == 0) {
    int cpr = p / 2;
    df_spmm_csr_kernel<true><<<ceil_div(n * cpr, 256), 256, 0, st>>>(n, rowptr, colidx, val, p,
                                                                      cpr, X, W);
  } else {
    df_spmm_csr_kernel<false><<<ceil_div(n * p, 256), 256, 0, st>>>(n, rowptr, colidx, val, p, p,
                                                                     X, W);
  }
  GSI_LAUNCH_CHECK();
  return GSI_OK;
}

__global__ void df_spmm_sell_kernel(int64_t nslots, int C, const int64_t* __restrict__ perm,
                                    const int64_t* __restrict__ chunk_ptr,
                                    const int64_t* __restrict__ chunk_len,
                                    const int32_t* __restrict__ scol,
                                    const float2* __restrict__ sval, int p,
                                    const float2* __restrict__ X, float2* __restrict__ W) {
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
  float h0 = 0.f, e0 = 0.f;
  for (int64_t j = 0; j < len; ++j) {
    int64_t s = base + j * C;
    df_mac(h0, e0, __ldg(sval + s), __ldg(X + (int64_t)__ldg(scol + s) * p + c));
  }
  W[row * p + c] = fast_two_sum(h0, e0);
}

gsi_status df_spmm_sell(int64_t nchunks, int C, const int64_t* perm, const int64_t* chunk_ptr,
                        const int64_t* chunk_len, const int32_t* scol, const float2* sval, int p,
                        const float2* X, float2* W, cudaStream_t st) {
  int64_t nslots = nchunks * C;
  if (nslots <= 0) return GSI_OK;
  int lg = 0, cpl = 1;
  if (rows_shape(p, X, W, &lg, &cpl)) {
    const int64_t threads = nslots << lg;
    if (cpl == 1)
      df_spmm_rows_kernel<1, true><<<ceil_div(threads, 256), 256, 0, st>>>(nslots, lg, p, chunk_ptr, scol, sval, C,
                                                                          perm, chunk_len, X, W);
    else
      df_spmm_rows_kernel<2, true><<<ceil_div(threads, 256), 256, 0, st>>>(nslots, lg, p, chunk_ptr, scol, sval, C,
                                                                          perm, chunk_len, X, W);
    GSI_LAUNCH_CHECK();
    return GSI_OK;
  }
  df_spmm_sell_kernel<<<ceil_div(nslots * p, 256), 256, 0, st>>>(nslots, C, perm, chunk_ptr,
                                                                  chunk_len, scol, sval, p, X, W);
  GSI_LAUNCH_CHECK();
  return GSI_OK;
}

// Frobenius products <A0,B0>, <A1,B1> and max_r sum_j |R[r,j]|, df64
// accumulation, deterministic two-stage reduction.
constexpr int DOT_THREADS = 256;

int df_dots_blocks(int64_t count) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sm_count() * 4, (count + 1023) / 1024));
}

__device__ __forceinline__ float2 shfl_df(float2 v, int o) {
  return make_float2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o));
}

__global__ void df_dots_kernel(int64_t n, int p, const float2* A0, const float2* B0,
                               const float2* A1, const float2* B1, const float2* R, float2* part) {
  __shared__ float2 red[2][DOT_THREADS / 32];
  __shared__ float redm[DOT_THREADS / 32];
  const int64_t count = n * p;
  int64_t per = (count + gridDim.x - 1) / gridDim.x;
  int64_t e0 = blockIdx.x * per, e1 = min(count, e0 + per);
  float2 s0 = make_float2(0.f, 0.f), s1 = make_float2(0.f, 0.f);
  for (int64_t e = e0 + threadIdx.x; e < e1; e += DOT_THREADS) {
    if (A0) s0 = df_add(s0, df_mul(A0[e], B0[e]));
    if (A1) s1 = df_add(s1, df_mul(A1[e], B1[e]));
  }
  float mx = 0.f;
  if (R) {
    int64_t r0 = (e0 + p - 1) / p, r1 = (e1 + p - 1) / p;
    for (int64_t r = r0 + threadIdx.x; r < r1; r += DOT_THREADS) {
      float s = 0.f;
      for (int j = 0; j < p; ++j) s += fabsf(R[r * p + j].x);
      mx = fmaxf(mx, s);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    s0 = df_add(s0, shfl_df(s0, o));
    s1 = df_add(s1, shfl_df(s1, o));
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    red[0][w] = s0;
    red[1][w] = s1;
    redm[w] = mx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float2 t0 = make_float2(0.f, 0.f), t1 = make_float2(0.f, 0.f);
    float m = 0.f;
    for (int i = 0; i < DOT_THREADS / 32; ++i) {
      t0 = df_add(t0, red[0][i]);
      t1 = df_add(t1, red[1][i]);
      m = fmaxf(m, redm[i]);
    }
    part[3 * blockIdx.x] = t0;
    part[3 * blockIdx.x + 1] = t1;
    part[3 * blockIdx.x + 2] = make_float2(m, 0.f);
  }
}

__global__ void df_dots_final_kernel(int nb, const float2* part, double* out) {
  if (threadIdx.x != 0) return;
  float2 t0 = make_float2(0.f, 0.f), t1 = make_float2(0.f, 0.f);
  float m = 0.f;
  for (int b = 0; b < nb; ++b) {
    t0 = df_add(t0, part[3 * b]);
    t1 = df_add(t1, part[3 * b + 1]);
    m = fmaxf(m, part[3 * b + 2].x);
  }
  out[0] = df_to_double(t0);
  out[1] = df_to_double(t1);
  out[2] = (double)m;
}

gsi_status df_dots(int64_t n, int p, const float2* A0, const float2* B0, const float2* A1,
                   const float2* B1, const float2* R, double* out, float2* scratch,
                   cudaStream_t st) {
  int nb = df_dots_blocks(n * p);
  df_dots_kernel<<<nb, DOT_THREADS, 0, st>>>(n, p, A0, B0, A1, B1, R, scratch);
  GSI_LAUNCH_CHECK();
  df_dots_final_kernel<<<1, 32, 0, st>>>(nb, scratch, out);
  GSI_LAUNCH_CHECK();
  return GSI_OK;
}

__global__ void df_axpby_kernel(int64_t count, float2 a, const float2* x, float2 b, float2* y) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) y[i] = df_add(df_mul(a, x[i]), df_mul(b, y[i]));
}

gsi_status df_axpby(int64_t count, float2 a, const float2* x, float2 b, float2* y, cudaStream_t st) {
  if (count <= 0) return GSI_OK;
  df_axpby_kernel<<<ceil_div(count, 256), 256, 0, st>>>(count, a, x, b, y);
  GSI_LAUNCH_CHECK();
  return GSI_OK;
}

// out = a W + b Z + e Zp (df64 scalars; Zp may be null) -- one step of the
// Chebyshev three-term recurrence after the matvec W = A Z
__global__ void df_combine3_kernel(int64_t count, float2 a, const float2* W, float2 b,
                                   const float2* Z, float2 e, const float2* Zp, float2* out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  float2 v = df_add(df_mul(a, W[i]), df_mul(b, Z[i]));
  if (Zp) v = df_add(v, df_mul(e, Zp[i]));
  out[i] = v;
}

gsi_status df_combine3(int64_t count, float2 a, const float2* W, float2 b, const float2* Z, float2 e,
                       const float2* Zp, float2* out, cudaStream_t st) {
  if (count <= 0) return GSI_OK;
  df_combine3_kernel<<<ceil_div(count, 256), 256, 0, st>>>(count, a, W, b, Z, e, Zp, out);
  GSI_LAUNCH_CHECK();
  return GSI_OK;
}

__global__ void df_sum_parts_kernel(int nparts, const float2* parts, double* out, const float* rinf) {
  if (threadIdx.x != 0) return;
  float2 t0 = make_float2(0.f, 0.f), t1 = make_float2(0.f, 0.f);
  float m = 0.f;
  // unrolled so that several partials are in flight at once (same order)
#pragma unroll 8
  for (int b = 0; b < nparts; ++b) {
    t0 = df_add(t0, parts[2 * b]);
    t1 = df_add(t1, parts[2 * b + 1]);
    if (rinf) m = fmaxf(m, rinf[b]);
  }
  out[0] = df_to_double(t0);
  out[1] = df_to_double(t1);
  if (rinf) out[2] = (double)m;
}

gsi_status df_sum_parts(int nparts, const float2* parts, double* out, cudaStream_t st,
                        const float* rinf_parts) {
  df_sum_parts_kernel<<<1, 32, 0, st>>>(nparts, parts, out, rinf_parts);
  GSI_LAUNCH_CHECK();
  return GSI_OK;
}

}  // namespace gsi
