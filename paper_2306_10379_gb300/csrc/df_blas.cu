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


// ---------------------------------------------------------------------------
// Stencil-shaped operators (every nonzero on one of at most DIA_MAXD
// diagonals col - row = off[d]): the diagonals' values are stored row-major
// as df64 (n x nd, zero where A has no entry), and W = A X runs through a
// shared-memory window. A CTA walks a contiguous range of 64-row tiles; tiles
// k - q .. k + q of X (and the diagonal values of tile k) sit in a ring of
// 2q + 2 slots filled by cp.async one tile ahead, so the offsets with
// |off| <= 64 q are read from shared memory and only the others ("far",
// at most two) from global memory. For the 3D 7-point stencil on a 128^3
// grid (offsets 0, +-1, +-128, +-16384, q = 2) an X row is read from L2
// three times instead of seven. The diagonals are summed in ascending offset
// order -- the column order of a sorted CSR row -- and the zeros of absent
// entries add exactly nothing, so the result equals the CSR kernel's bit for
// bit when the CSR rows are sorted. Measured at 128^3 it is slower than the
// CSR kernel (p = 64: 1.59 against 1.02 ms; p = 8: 1.35 against 0.14 ms):
// one CTA per SM with serial per-row accumulation leaves a per-tile latency
// floor, and with contiguous tile ranges per CTA the far-diagonal rows are
// not in L2 when they are read. The solver uses it only on request.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16_dia(void* smem, const void* gmem, bool valid) {
  uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
  int sz = valid ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(sz));
}
__device__ __forceinline__ void cp_async8_dia(void* smem, const void* gmem, bool valid) {
  uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
  int sz = valid ? 8 : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(sa), "l"(gmem), "r"(sz));
}

template <int NFAR>
__global__ void __launch_bounds__(DIA_THREADS, 1) df_spmm_dia_kernel(DiaArgs a) {
  extern __shared__ __align__(16) unsigned char dia_sm[];
  const int p = a.p, nd = a.nd, q = a.q, NS = 2 * q + 2;
  const int hp = p / 2;                       // column pairs
  float2* win = reinterpret_cast<float2*>(dia_sm);                       // NS x DIA_T x p
  float2* dv = win + (size_t)NS * DIA_T * p;                             // NS x DIA_T x nd
  const int64_t k0 = (int64_t)blockIdx.x * a.tiles_per_cta;
  const int64_t k1 = min(a.ntiles, k0 + a.tiles_per_cta);
  if (k0 >= k1) return;
  auto slot = [&](int64_t k) { return (int)(((k % NS) + NS) % NS); };
  // tile k's X rows and (for k in range) its diagonal values into slot(k);
  // rows outside [0, n) are zero-filled
  auto load = [&](int64_t k) {
    float2* xd = win + (size_t)slot(k) * DIA_T * p;
    const int64_t r0 = k * DIA_T;
    for (int e = threadIdx.x; e < DIA_T * hp; e += DIA_THREADS) {
      const int row = e / hp, c2 = e - row * hp;
      const int64_t R = r0 + row;
      const bool ok = R >= 0 && R < a.n;
      cp_async16_dia(xd + row * p + 2 * c2, a.X + (ok ? R * p + 2 * c2 : 0), ok);
    }
    float2* vd = dv + (size_t)slot(k) * DIA_T * nd;
    for (int e = threadIdx.x; e < DIA_T * nd; e += DIA_THREADS) {
      const int64_t R = r0 + e / nd;
      const bool ok = R >= 0 && R < a.n;
      cp_async8_dia(vd + e, a.val + (ok ? r0 * nd + e : 0), ok);
    }
    asm volatile("cp.async.commit_group;\n" ::);
  };
  for (int64_t k = k0 - q; k <= k0 + q; ++k) load(k);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool act = lane < hp;
  constexpr int RPW = DIA_T / (DIA_THREADS / 32);  // rows per warp and tile
  for (int64_t k = k0; k < k1; ++k) {
    load(k + q + 1);  // into the slot of tile k - q - 1, free since the last iteration
    asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    __syncthreads();
    const int s0 = slot(k);  // the window's tiles k + kt sit in slots s0 + kt (mod NS), |kt| <= q < NS
    const float2* vk = dv + (size_t)s0 * DIA_T * nd;
    // far diagonals: X rows from global memory, loaded two rows ahead
    int foff0 = 0, foff1 = 0;
#pragma unroll
    for (int d = 0; d < DIA_MAXD; ++d) {
      if (NFAR > 0 && d == a.far_d[0]) foff0 = a.off[d];
      if (NFAR > 1 && d == a.far_d[1]) foff1 = a.off[d];
    }
    const int64_t nrow = a.n;
    const float2* Xg = a.X;
    const int64_t rbase = k * DIA_T + warp;
    auto far1 = [=](int j, int o) {
      const int64_t R = rbase + j * (DIA_THREADS / 32);
      const int64_t col = R + o;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (act && j < RPW && R < nrow && col >= 0 && col < nrow)
        v = __ldg(reinterpret_cast<const float4*>(Xg + col * p) + lane);
      return v;
    };
    float4 fa0 = make_float4(0.f, 0.f, 0.f, 0.f), fa1 = fa0, fb0 = fa0, fb1 = fa0;
    if (NFAR > 0) {
      fa0 = far1(0, foff0);
      fb0 = far1(1, foff0);
    }
    if (NFAR > 1) {
      fa1 = far1(0, foff1);
      fb1 = far1(1, foff1);
    }
#pragma unroll 1
    for (int j = 0; j < RPW; ++j) {
      const float4 fc0 = fa0, fc1 = fa1;
      fa0 = fb0;
      fa1 = fb1;
      if (NFAR > 0) fb0 = far1(j + 2, foff0);
      if (NFAR > 1) fb1 = far1(j + 2, foff1);
      const int rr = warp + j * (DIA_THREADS / 32);
      const int64_t R = k * DIA_T + rr;
      if (R >= a.n || !act) continue;
      float h0 = 0.f, e0 = 0.f, h1 = 0.f, e1 = 0.f;
#pragma unroll
      for (int d = 0; d < DIA_MAXD; ++d) {  // constant indices keep a.off in parameter space
        if (d < nd) {
          const float2 v = vk[rr * nd + d];
          float4 x;
          if ((a.near_mask >> d) & 1) {
            const int src = rr + a.off[d];  // row relative to tile k's first row
            const int kt = src >= 0 ? src / DIA_T : -((-src + DIA_T - 1) / DIA_T);
            const int rin = src - kt * DIA_T;
            int sk = s0 + kt;
            sk += sk < 0 ? NS : 0;
            sk -= sk >= NS ? NS : 0;
            x = *reinterpret_cast<const float4*>(win + ((size_t)sk * DIA_T + rin) * p + 2 * lane);
          } else {
            x = (NFAR > 1 && a.far_d[1] == d) ? fc1 : fc0;
          }
          df_mac(h0, e0, v, make_float2(x.x, x.y));
          df_mac(h1, e1, v, make_float2(x.z, x.w));
        }
      }
      const float2 r0v = fast_two_sum(h0, e0), r1v = fast_two_sum(h1, e1);
      reinterpret_cast<float4*>(a.W + R * p)[lane] = make_float4(r0v.x, r0v.y, r1v.x, r1v.y);
    }
    __syncthreads();
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

size_t dia_smem_bytes(int p, int q, int nd) {
  return (size_t)(2 * q + 2) * DIA_T * ((size_t)p + nd) * sizeof(float2);
}

int dia_plan(int p, int nd, const int* off, int* q_out, int* near_mask, int* far_d, int* nfar) {
  if ((p & 1) || p > 64 || nd < 1 || nd > DIA_MAXD) return 0;
  // the largest window that fits: 2q + 2 slots of DIA_T rows of X and values
  int qmax = 0;
  while (dia_smem_bytes(p, qmax + 1, nd) <= (size_t)DIA_SMEM_MAX) ++qmax;
  if (qmax < 1) return 0;
  int q = 1, nf = 0, mask = 0;
  for (int d = 0; d < nd; ++d) {
    const int ao = off[d] < 0 ? -off[d] : off[d];
    if (ao <= DIA_T * qmax) {
      mask |= 1 << d;
      q = std::max(q, (ao + DIA_T - 1) / DIA_T);
    } else {
      if (nf == DIA_MAXFAR) return 0;
      far_d[nf++] = d;
    }
  }
  *q_out = q;
  *near_mask = mask;
  *nfar = nf;
  return 1;
}

gsi_status df_spmm_dia(const DiaArgs& a0, cudaStream_t st) {
  DiaArgs a = a0;
  if (a.n <= 0) return GSI_OK;
  a.ntiles = (a.n + DIA_T - 1) / DIA_T;
  const int grid = (int)std::min<int64_t>(a.ntiles, sm_count());
  a.tiles_per_cta = (a.ntiles + grid - 1) / grid;
  const size_t sm = dia_smem_bytes(a.p, a.q, a.nd);
  if (a.nfar == 0) {
    GSI_CUDA_TRY(cudaFuncSetAttribute(df_spmm_dia_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    df_spmm_dia_kernel<0><<<grid, DIA_THREADS, sm, st>>>(a);
  } else if (a.nfar == 1) {
    GSI_CUDA_TRY(cudaFuncSetAttribute(df_spmm_dia_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    df_spmm_dia_kernel<1><<<grid, DIA_THREADS, sm, st>>>(a);
  } else {
    GSI_CUDA_TRY(cudaFuncSetAttribute(df_spmm_dia_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    df_spmm_dia_kernel<2><<<grid, DIA_THREADS, sm, st>>>(a);
  }
  GSI_LAUNCH_CHECK();
  return GSI_OK;
}

}  // namespace gsi
