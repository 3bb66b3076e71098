// Float64-accurate block products on the BF16 tensor cores (error-free
// splitting after Ozaki, Ogita, Oishi & Rump, "Error-free transformations of
// matrix multiplication by using fast routines of matrix multiplication and
// its applications", Numer. Algorithms 59, 2012), for the two contraction
// shapes of one iteration:
//   oz_gemm : OUT = sum_k U_k M_k + sum_e c_e E_e   (n x p blocks times p x p)
//   oz_gram : G   = U^T V                          (contraction over the n rows)
// Block data is df64 (float2 = hi, lo). Every operand is cut into ND = 7
// signed "digits" d_i in [-128, 128] on a fixed-point grid set by a power of
// two per row (gemm, left operand), per column (p x p right operand) or per
// column and row chunk (gram: 64 rows in the mma.sync kernel, 256 or 160 in
// the tcgen05 kernel):
//   x = 2^(E-7) * sum_{i<7} d_i 2^(-7 i) + r,  |r| <= 2^(E-46) + 2^(E-50)
// (the remainder below the last digit, and one rounding where the low word
// of x joins the remainder after digit 2).
// Digits are exact in bf16 and are stored with their weights, d_i 2^(-7 i);
// products of two digits are exact in fp32, and the 28 digit pairs
// (i + i' <= 6) are summed per "group" g = i + i' in fp32 accumulators whose
// partial sums stay below 2^24 times the group's weight 2^(-7 g) for
// contraction lengths up to 256, so the tensor-core accumulation is exact.
// The 7 group sums S_g are then combined in df64:
// OUT = 2^(E_r + F_j - 14) sum_g S_g.
#include <cuda_bf16.h>
#include <stdlib.h>
#include <string.h>

#include "df.cuh"
#include "oz.cuh"

namespace gsi {

constexpr int ND = 7;

// 0 and 2: tcgen05 kernels wherever they apply (7-digit block products and
// Grams of any p, q <= 128), 1: mma.sync kernels
// only (set by gsi_set_tensor_path, or by GSI_TENSOR_PATH=mma / =tcgen05 at
// the first product)
static int g_tensor_path = -1;
int tensor_path() {
  if (g_tensor_path < 0) {
    const char* e = getenv("GSI_TENSOR_PATH");
    g_tensor_path = (e && strcmp(e, "mma") == 0) ? 1 : (e && strcmp(e, "tcgen05") == 0) ? 2 : 0;
  }
  return g_tensor_path;
}
void set_tensor_path(int path) { g_tensor_path = (path == 1 || path == 2) ? path : 0; }
constexpr float MAGIC = 12582912.0f;  // 1.5 * 2^23: x + MAGIC - MAGIC rounds x to an integer

__device__ __forceinline__ int exponent_above(float maxabs) {
  // smallest E with maxabs < 2^E, clamped to keep 2^(7-E) finite in fp32
  if (!(maxabs > 0.0f)) return 0;
  int e = ((__float_as_int(maxabs) >> 23) & 255) - 127;
  return max(e + 1, -100);
}

// The 7 digits of (h + l) on the grid of 2^(E-7), each returned with its
// weight: d[i] = d_i 2^(-7 i) (exact in bf16 like d_i itself, so a product of
// digits i and j already carries the 2^(-7 (i + j)) of its group). In the
// frame a = (h + l) 2^(7-E), |a| < 128: adding 1.5 * 2^(23 - 7i) rounds a to
// a multiple of 2^(-7i), and a <- a - d[i] is exact. Digits 0..2 come from h
// alone, then l is folded in (at that point h's remainder is a multiple of
// 2^-17 and |l 2^(7-E)| <= 2^-17 * 8, so one rounding of at most 2^-45 of the
// scale can occur), digits 3..6 follow.
template <int N>
__device__ __forceinline__ void digitsN(float h, float l, int E, float d[N]) {
  const float s = exp2i(7 - E);
  float a = __fmul_rn(h, s);
  const float b = __fmul_rn(l, s);
#pragma unroll
  for (int i = 0; i < N; ++i) {
    if (i == 3) a = __fadd_rn(a, b);
    const float m = MAGIC * exp2i(-7 * i);  // exact power of two, constant per i
    float t = __fadd_rn(a, m);
    float di = __fsub_rn(t, m);
    d[i] = di;
    a = __fsub_rn(a, di);
  }
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

// sum_g S_g as df64, where S_g is the group sum of weighted digit products
// (an integer times 2^(-7 g)): from the smallest group up, TwoSum per step
template <int N>
__device__ __forceinline__ float2 combine_groups(const float S[N]) {
  float h = S[N - 1], l = 0.0f;
#pragma unroll
  for (int g = N - 2; g >= 0; --g) {
    float2 t = two_sum(S[g], h);
    h = t.x;
    l = __fadd_rn(l, t.y);
  }
  return fast_two_sum(h, l);
}

// sum_g S_g as df64 like combine_groups, with the groups NEXACT .. N - 1 (of
// weight 2^-28 and below when NEXACT = 4 and g0 = 0) added in float32: their
// rounding stays below 2^-52 of the product's scale, far under the 2^-49 of
// the digit cut; the others by TwoSum from the smallest up. S_g is an exact
// integer times 2^(-7 (g + g0)), g0 = 0 or 1. NEXACT = N - 1 is combine_groups.
template <int N, int NEXACT>
__device__ __forceinline__ float2 combine_groups_fast(const float S[N]) {
  static_assert(NEXACT >= 1 && NEXACT < N, "S[N - 1] starts the sum");
  float h = S[N - 1];
#pragma unroll
  for (int g = N - 2; g >= NEXACT; --g) h = __fadd_rn(S[g], h);
  float l = 0.0f;
#pragma unroll
  for (int g = NEXACT - 1; g >= 0; --g) {
    const float2 t = two_sum(S[g], h);
    h = t.x;
    l = __fadd_rn(l, t.y);
  }
  return fast_two_sum(h, l);
}

__device__ __forceinline__ void ldsm_x4(uint32_t r[4], const void* p) {
  uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t r[4], const void* p) {
  uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}
__device__ __forceinline__ void ldsm_x2(uint32_t r[2], const void* p) {
  uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n"
               : "=r"(r[0]), "=r"(r[1])
               : "r"(a));
}
__device__ __forceinline__ void ldsm_x2_t(uint32_t r[2], const void* p) {
  uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n"
               : "=r"(r[0]), "=r"(r[1])
               : "r"(a));
}
__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], const uint32_t b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// ---------------------------------------------------------------------------
// Right operand: B = [s_0 M_0; s_1 M_1] restricted to the rows k0 .. k0+kw-1
// of each M_k (K = nk*kw rows, p columns, float64), cut into digits with one
// power of two per column. Layout for the tensor cores: Md[plane][n][k]
// (k contiguous, K16 = K rounded up to 16), F[n]. One block per column n.
// ---------------------------------------------------------------------------
__global__ void oz_prep_rhs_kernel(int p, int p16, int nk, int K16, const double* M0,
                                   const double* M1, double s0, double s1,
                                   __nv_bfloat16* Md, int* F, int k0, int kw) {
  const int n = blockIdx.x;
  __shared__ float red[32];
  __shared__ int sE;
  const int K = nk * kw;
  float mx = 0.0f;
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    int kk = k / kw, l = k0 + k - kk * kw;
    double v = (n < p) ? (kk == 0 ? s0 * M0[l * p + n] : s1 * M1[l * p + n]) : 0.0;
    mx = fmaxf(mx, fabsf((float)v));
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    float m = 0.0f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
    sE = exponent_above(m);
    F[n] = sE;
  }
  __syncthreads();
  const int E = sE;
  for (int k = threadIdx.x; k < K16; k += blockDim.x) {
    double v = 0.0;
    if (k < K && n < p) {
      int kk = k / kw, l = k0 + k - kk * kw;
      v = (kk == 0 ? s0 * M0[l * p + n] : s1 * M1[l * p + n]);
    }
    float2 x = df_from_double(v);
    float d[ND];
    digitsN<ND>(x.x, x.y, E, d);
#pragma unroll
    for (int i = 0; i < ND; ++i)
      Md[((size_t)i * p16 + n) * K16 + k] = __float2bfloat16_rn(d[i]);
  }
}

// cp.async staging (8-byte granularity, zero fill for out-of-range elements)
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem, bool valid) {
  uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
  int sz = valid ? 8 : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(sa), "l"(gmem), "r"(sz));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// ---------------------------------------------------------------------------
// oz_gemm: OUT = (U0 + a1 U1) M + sum_e c_e E_e, M already scaled and cut
// into digits (oz_prep_rhs). Rows in tiles of RT = 32, output columns in
// slices of up to 64 (blockIdx.y). 8 warps: 2 row groups of 16 x 4 column
// groups; each warp owns up to 2 n-tiles of 8 columns. The raw df64 rows of
// the next tile are fetched with cp.async while the current tile is on the
// tensor cores.
// ---------------------------------------------------------------------------
constexpr int GM_RT = 32;
constexpr int GM_THREADS = 256;

__host__ __device__ inline int gm_ud_stride(int K16) { return K16 + 8; }   // bf16 elements per row
__host__ __device__ inline int gm_md_stride(int K16) { return K16 + 8; }

size_t oz_gemm_smem(int K16, int NC, int nraw, int nd = ND) {
  return (size_t)nd * GM_RT * gm_ud_stride(K16) * 2 + (size_t)nd * NC * gm_md_stride(K16) * 2 +
         (size_t)nraw * GM_RT * K16 * sizeof(float2) + (GM_RT + NC) * sizeof(int) + 64;
}

__device__ __forceinline__ void gm_stage(const OzGemmArgs& a, int64_t n, int p, int K16, int64_t r0,
                                         float2* raw0, float2* raw1) {
  for (int e = threadIdx.x; e < GM_RT * K16; e += GM_THREADS) {
    int rr = e / K16, k = e - rr * K16;
    int64_t R = r0 + rr;
    bool ok = R < n && k < p;
    int64_t idx = ok ? R * p + k : 0;
    cp_async8(raw0 + e, a.U[0] + idx, ok);
    if (raw1) cp_async8(raw1 + e, a.U[1] + idx, ok);
  }
  cp_async_commit();
}

template <int NDT>
__global__ void __launch_bounds__(GM_THREADS, 2)
oz_gemm_kernel(int64_t n, int p, int p16, int K16, OzGemmArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int col0 = blockIdx.y * 64;
  const int NC = min(64, p16 - col0);
  const int uds = gm_ud_stride(K16), mds = gm_md_stride(K16);
  const bool two = a.fuse_u1 != 0;
  __nv_bfloat16* Ud = reinterpret_cast<__nv_bfloat16*>(smem);
  __nv_bfloat16* Ms = Ud + (size_t)NDT * GM_RT * uds;
  float2* raw0 = reinterpret_cast<float2*>(Ms + (size_t)NDT * NC * mds);
  float2* raw1 = two ? raw0 + GM_RT * K16 : nullptr;
  int* Er = reinterpret_cast<int*>(raw0 + (two ? 2 : 1) * GM_RT * K16);
  int* Fs = Er + GM_RT;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t ntiles = (n + GM_RT - 1) / GM_RT;
  if ((int64_t)blockIdx.x < ntiles) gm_stage(a, n, p, K16, (int64_t)blockIdx.x * GM_RT, raw0, raw1);

  // right operand digits for this column slice
  for (int e = tid; e < NDT * NC * (K16 / 8); e += GM_THREADS) {
    int chunk = e % (K16 / 8);
    int rowi = e / (K16 / 8);
    int plane = rowi / NC, nn = rowi - plane * NC;
    const uint4* src = reinterpret_cast<const uint4*>(a.Md + ((size_t)plane * p16 + col0 + nn) * K16) + chunk;
    *reinterpret_cast<uint4*>(Ms + ((size_t)plane * NC + nn) * mds + chunk * 8) = *src;
  }
  for (int e = tid; e < NC; e += GM_THREADS) Fs[e] = a.F[col0 + e];

  float2 dacc0 = make_float2(0.f, 0.f), dacc1 = make_float2(0.f, 0.f);
  const int wr = warp >> 2, wc = warp & 3;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t r0 = tile * GM_RT;
    cp_async_wait_all();
    __syncthreads();  // raw rows of this tile in shared memory; Ud free
    // (a) per row (one warp per row): combine U0 + a1 U1 in place, row maximum,
    // then digits from shared memory (two passes keep the registers free)
    for (int rr = warp; rr < GM_RT; rr += GM_THREADS / 32) {
      float2* row0 = raw0 + rr * K16;
      float mx = 0.0f;
      for (int k = lane; k < K16; k += 32) {
        float2 x = row0[k];
        if (two) {
          x = df_add(x, df_mul(a.a1, raw1[rr * K16 + k]));
          row0[k] = x;
        }
        mx = fmaxf(mx, fabsf(x.x));
      }
      for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      const int E = exponent_above(mx);
      if (lane == 0) Er[rr] = E;
      __syncwarp();
      for (int cp = lane; 2 * cp < K16; cp += 32) {
        const float4 xx = *reinterpret_cast<const float4*>(row0 + 2 * cp);
        float d0[NDT], d1[NDT];
        digitsN<NDT>(xx.x, xx.y, E, d0);
        digitsN<NDT>(xx.z, xx.w, E, d1);
#pragma unroll
        for (int i = 0; i < NDT; ++i)
          *reinterpret_cast<uint32_t*>(Ud + ((size_t)i * GM_RT + rr) * uds + 2 * cp) =
              pack_bf16x2(d0[i], d1[i]);
      }
    }
    __syncthreads();  // digits ready, raw buffers free: prefetch the next tile
    if (tile + gridDim.x < ntiles) gm_stage(a, n, p, K16, (tile + gridDim.x) * GM_RT, raw0, raw1);
    // (c) tensor-core products, exact per digit-pair group
    float acc[NDT][2][4];
#pragma unroll
    for (int g = 0; g < NDT; ++g)
#pragma unroll
      for (int t = 0; t < 2; ++t)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[g][t][q] = 0.0f;
    const int ntl = NC / 8;
    const bool act0 = wc < ntl, act1 = wc + 4 < ntl;
    if (act0) {
      for (int ks = 0; ks < K16 / 16; ++ks) {
        uint32_t A[NDT][4];
        const int q = lane >> 3;
#pragma unroll
        for (int i = 0; i < NDT; ++i)
          ldsm_x4(A[i], Ud + ((size_t)i * GM_RT + wr * 16 + (lane & 7) + (q & 1) * 8) * uds +
                            ks * 16 + (q >> 1) * 8);
#pragma unroll
        for (int t = 0; t < 2; ++t) {
          if (t == 1 && !act1) break;
          const int nt = wc + 4 * t;
#pragma unroll
          for (int j = 0; j < NDT; ++j) {
            uint32_t B[2];
            const int l16 = lane & 15;
            ldsm_x2(B, Ms + ((size_t)j * NC + nt * 8 + (l16 & 7)) * mds + ks * 16 + (l16 >> 3) * 8);
#pragma unroll
            for (int i = 0; i < NDT - j; ++i) mma_bf16(acc[i + j][t], A[i], B);
          }
        }
      }
    }
    // (d) epilogue: df64 combination, scaling, elementwise terms, store
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      if (!(t == 0 ? act0 : act1)) continue;
      const int nt = wc + 4 * t;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int rr = wr * 16 + (lane >> 2) + h * 8;
        const int64_t R = r0 + rr;
        const int cc = nt * 8 + (lane & 3) * 2;
        if (R >= n) continue;
        float2 v[2];
#pragma unroll
        for (int e2 = 0; e2 < 2; ++e2) {
          float S[NDT];
#pragma unroll
          for (int g = 0; g < NDT; ++g) S[g] = acc[g][t][h * 2 + e2];
          // the same combination as the tcgen05 block product (bit-identical results)
          float2 w = combine_groups_fast<NDT, (NDT > 4 ? 4 : NDT - 1)>(S);
          int sc = Er[rr] + Fs[cc + e2] - 14;
          if (sc >= -126) {
            float f = exp2i(sc);
            v[e2] = make_float2(w.x * f, w.y * f);
          } else {
            float f1 = exp2i(sc / 2), f2 = exp2i(sc - sc / 2);
            v[e2] = make_float2(w.x * f1 * f2, w.y * f1 * f2);
          }
        }
        const int C = col0 + cc;
#pragma unroll
        for (int e2 = 0; e2 < 2; ++e2) {
          if (C + e2 >= p) continue;
          float2 y = v[e2];
          const int64_t idx = R * p + C + e2;
#pragma unroll
          for (int m = 0; m < 2; ++m)  // constant indices keep the arguments in parameter space
            if (m < a.ne) y = df_add(y, df_mul(a.ce[m], a.E[m][idx]));
          if (a.dot_self) df_dot_acc(dacc0, y, y);
          if (a.dot_with) df_dot_acc(dacc1, y, a.dot_with[idx]);
          a.out[idx] = y;
        }
      }
    }
  }
  cp_async_wait_all();
  if (a.dot_part) {
    __shared__ float2 red[2][GM_THREADS / 32];
    dacc0 = df_acc_done(dacc0);  // the running sums were left unnormalised
    dacc1 = df_acc_done(dacc1);
    for (int o = 16; o > 0; o >>= 1) {
      float2 t0 = make_float2(__shfl_xor_sync(0xffffffffu, dacc0.x, o), __shfl_xor_sync(0xffffffffu, dacc0.y, o));
      float2 t1 = make_float2(__shfl_xor_sync(0xffffffffu, dacc1.x, o), __shfl_xor_sync(0xffffffffu, dacc1.y, o));
      dacc0 = df_add(dacc0, t0);
      dacc1 = df_add(dacc1, t1);
    }
    if (lane == 0) {
      red[0][warp] = dacc0;
      red[1][warp] = dacc1;
    }
    __syncthreads();
    if (tid == 0) {
      float2 s0 = make_float2(0.f, 0.f), s1 = make_float2(0.f, 0.f);
      for (int w = 0; w < GM_THREADS / 32; ++w) {
        s0 = df_add(s0, red[0][w]);
        s1 = df_add(s1, red[1][w]);
      }
      int b = blockIdx.y * gridDim.x + blockIdx.x;
      a.dot_part[2 * b] = s0;
      a.dot_part[2 * b + 1] = s1;
    }
  }
}

// ---------------------------------------------------------------------------
// oz_gemm on the 5th-generation tensor cores (tcgen05), for K16 <= 64 (one
// slice of a longer contraction per launch) and the 7-digit split. 128-row tiles; the 7 digit planes of the tile's left operand
// and of the right operand live in shared memory in the no-swizzle K-major
// core-matrix layout (8 x 16-byte cores; K-adjacent cores 128 B apart, 8-row
// groups K16/8 * 128 B apart). One thread issues the 28 digit-pair products
// as M = 128, N = NC, K = 16 MMAs into 7 group accumulators in tensor memory
// (group g at columns g NC); the epilogue reads each row's group sums back
// (tcgen05.ld, TMEM lane = row) and combines them in df64 as the mma.sync
// kernel does. The group sums are exact integers either way, so both kernels
// give identical results.
// ---------------------------------------------------------------------------
constexpr int TC_M = 128;
constexpr int TC_WORKERS = 512;                // 16 warps: loads, digits, combination
constexpr int TC_THREADS = TC_WORKERS + 32;    // + one warp that issues the products
constexpr uint32_t TC_TMEM_COLS = 512;
constexpr int TC_WAIT_LIMIT = 1 << 24;

__device__ int g_oz_tc_timeouts;  // count of bounded waits that ran out
// polls allowed to a wait on the products of a tile or sub-chunk (host-settable,
// 0..TC_WAIT_LIMIT); the drain after a wait that ran out always polls up to
// TC_WAIT_LIMIT times
__device__ int g_oz_wait_limit = TC_WAIT_LIMIT;

__host__ __device__ inline size_t tc_plane_bytes(int rows, int K16) { return (size_t)rows * K16 * 2; }

// The left operand's digit planes; the epilogue stages the tile's combined
// products (TC_M rows of NC + 2 float2) in the same space once the products
// have completed, which a short contraction (K16 < 48) does not cover alone.
__host__ __device__ inline size_t tc_a_region(int K16, int NC) {
  const size_t planes = (size_t)ND * tc_plane_bytes(TC_M, K16), stage = (size_t)TC_M * (NC + 2) * 8;
  return planes > stage ? planes : stage;
}

size_t oz_gemm_tc_smem(int K16, int NC) {
  return tc_a_region(K16, NC) + ND * tc_plane_bytes(NC, K16) + (TC_M + 64) * sizeof(int) + 64;
}

__device__ __forceinline__ uint32_t tc_off(int r, int k, int K16) {
  return (uint32_t)((((r >> 3) * (K16 >> 3) + (k >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1));
}

// shared-memory matrix descriptor: start, leading (K) core stride 128 B,
// stride (8-row group) K16/8 * 128 B, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, int K16) {
  const uint64_t sbo = (uint64_t)((K16 >> 3) * 128);
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)(128 >> 4) << 16) | (((sbo >> 4) & 0x3FFFu) << 32) |
         ((uint64_t)1 << 46);
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t parity, int limit = TC_WAIT_LIMIT) {
  uint32_t done = 0;
  for (int it = 0; it < limit && !done; ++it) {
    asm volatile(
        "{\n.reg .pred P1;\nmbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n"
        "selp.b32 %0, 1, 0, P1;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
  }
  return done != 0;
}

// After a wait ran out: the issuing thread commits once more to the drain
// barrier, which completes when every product it has issued so far has
// completed (a commit tracks all earlier tcgen05 operations of its thread);
// every thread then waits for that with the full bound, so no product is in
// flight when the tensor memory is released.
__device__ __forceinline__ void tc_drain(bool issuing_thread, uint32_t mbd) {
  if (issuing_thread)
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbd)
                 : "memory");
  tc_wait(mbd, 0u, TC_WAIT_LIMIT);
}

__device__ __forceinline__ void tc_ld4(uint32_t r[4], uint32_t taddr) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr));
}

// FUSED: the left operand is U0 + a1 U1 (a separate instantiation, so that
// the fused load path's registers do not weigh on the other products)
template <bool FUSED>
__global__ void __launch_bounds__(TC_THREADS, 1)
oz_gemm_tc_kernel(int64_t n, int p, int p16, int K16, OzGemmArgs a) {
  extern __shared__ __align__(16) unsigned char tc_smem[];
  unsigned char* smem = tc_smem;
  const int col0 = blockIdx.y * 64;
  const int NC = min(64, p16 - col0);
  const uint32_t aplane = (uint32_t)tc_plane_bytes(TC_M, K16), bplane = (uint32_t)tc_plane_bytes(NC, K16);
  unsigned char* Ad = smem;
  unsigned char* Bd = Ad + tc_a_region(K16, NC);
  int* Er = reinterpret_cast<int*>(Bd + ND * bplane);
  int* Fs = Er + TC_M;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(Fs + 64);  // [0] products, [1] drain
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr bool two = FUSED;

  // right operand digits (Md[plane][n][k]) into the core-matrix layout
  for (int e = tid; e < ND * NC * (K16 / 8); e += TC_THREADS) {
    const int c = e % (K16 / 8), rowi = e / (K16 / 8), plane = rowi / NC, nn = rowi - plane * NC;
    const uint4 v = *reinterpret_cast<const uint4*>(a.Md + ((size_t)plane * p16 + col0 + nn) * K16 + c * 8);
    *reinterpret_cast<uint4*>(Bd + plane * bplane + tc_off(nn, c * 8, K16)) = v;
  }
  for (int e = tid; e < NC; e += TC_THREADS) Fs[e] = a.F[col0 + e];
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tslot)),
                 "r"(TC_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(mbar)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(mbar + 1)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  const int wait_limit = g_oz_wait_limit;
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NC >> 3) << 17) |
                         ((uint32_t)(TC_M >> 4) << 24);
  const uint32_t abase = smem_addr(Ad), bbase = smem_addr(Bd), mb = smem_addr(mbar);
  float2 dacc0 = make_float2(0.f, 0.f), dacc1 = make_float2(0.f, 0.f);
  float rmax = 0.f;  // largest row sum of |hi(out)| seen by this warp
  uint32_t phase = 0;
  bool failed = false;
  const int64_t ntiles = (n + TC_M - 1) / TC_M;
  // lane = (row rr = rb + lane / 4 of the warp's 8 rows, pair j = lane % 4)
  // holds columns 8c + 2j, 8c + 2j + 1 (c < 8); one round of 8 rows per warp
  // (16 warps, 128-row tiles). The next tile's rows are loaded (and the fused
  // left sum formed) while the current tile's products run.
  static_assert(TC_WORKERS / 32 * 8 == TC_M, "one 8-row round per worker warp");
  const bool issuer = warp == TC_WORKERS / 32;
  const int rb = warp * 8, rr = rb + (lane >> 2), j = lane & 3;
  float2 xr[16];
  auto load_tile = [&](int64_t t) {
    const int64_t R = t * TC_M + rr;
    const bool live = t < ntiles && R < n;
    const int64_t ob = R * a.ldu + a.kofs + 2 * j;  // the pair at k = 2 j
    if (two && live && a.vec16 && a.kw >= 64 && (ob & 1) == 0) {
      // the fused left sum over a full 64-column slice: each half-row's eight
      // 16-byte loads (four of each operand) are issued before any of the
      // df64 arithmetic that consumes them, so their latencies overlap
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float4 v[4], u[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          v[c] = *reinterpret_cast<const float4*>(a.U[0] + ob + 8 * (4 * h + c));
          u[c] = *reinterpret_cast<const float4*>(a.U[1] + ob + 8 * (4 * h + c));
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          xr[2 * (4 * h + c)] = df_add(make_float2(v[c].x, v[c].y), df_mul(a.a1, make_float2(u[c].x, u[c].y)));
          xr[2 * (4 * h + c) + 1] =
              df_add(make_float2(v[c].z, v[c].w), df_mul(a.a1, make_float2(u[c].z, u[c].w)));
        }
      }
      return;
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int k = 8 * c + 2 * j;
      float2 x0 = make_float2(0.f, 0.f), x1 = make_float2(0.f, 0.f);
      if (live && k < a.kw) {
        const int64_t o = R * a.ldu + a.kofs + k;
        if (a.vec16 && k + 1 < a.kw && (o & 1) == 0) {  // 16-byte aligned pair
          const float4 v = *reinterpret_cast<const float4*>(a.U[0] + o);
          x0 = make_float2(v.x, v.y);
          x1 = make_float2(v.z, v.w);
          if (two) {
            const float4 u = *reinterpret_cast<const float4*>(a.U[1] + o);
            x0 = df_add(x0, df_mul(a.a1, make_float2(u.x, u.y)));
            x1 = df_add(x1, df_mul(a.a1, make_float2(u.z, u.w)));
          }
        } else {
          x0 = a.U[0][o];
          if (two) x0 = df_add(x0, df_mul(a.a1, a.U[1][o]));
          if (k + 1 < a.kw) {
            x1 = a.U[0][o + 1];
            if (two) x1 = df_add(x1, df_mul(a.a1, a.U[1][o + 1]));
          }
        }
      }
      xr[2 * c] = x0;
      xr[2 * c + 1] = x1;
    }
  };
  if (!issuer) load_tile(blockIdx.x);
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t r0 = tile * TC_M;
    // (a) the tile's left operand: row maxima and digits; global reads were
    // 64-byte row segments, and the digit stores hit 32 different banks (row
    // stride 16 B, pair stride 4 B in a core matrix)
    if (!issuer) {
      float mx = 0.0f;
#pragma unroll
      for (int c = 0; c < 16; ++c) mx = fmaxf(mx, fabsf(xr[c].x));
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
      const int E = exponent_above(mx);
      if (j == 0) Er[rr] = E;
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        if (8 * c < K16) {
          float d0[ND], d1[ND];
          digitsN<ND>(xr[2 * c].x, xr[2 * c].y, E, d0);
          digitsN<ND>(xr[2 * c + 1].x, xr[2 * c + 1].y, E, d1);
#pragma unroll
          for (int i = 0; i < ND; ++i)
            *reinterpret_cast<uint32_t*>(Ad + i * aplane + tc_off(rr, 8 * c + 2 * j, K16)) =
                pack_bf16x2(d0[i], d1[i]);
        }
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // (b) the 28 digit-pair products, issued by the issuing warp
    // (descriptor start addresses advance in 16-byte units). For the left
    // plane i the right planes j = 0 .. 6 - i feed the groups g = i + j,
    // whose accumulators are adjacent in tensor memory, and the planes are
    // adjacent in shared memory: one MMA of N = run NC per run of planes
    // (N <= 256) -- 11 MMAs per 16 columns of K at NC = 64 instead of 28.
    // Each group still receives i = 0, 1, .. in order (and its sums are
    // exact integers in any order).
    if (issuer) {
      if (lane == 0) {
        const uint64_t da = tc_desc(abase, K16), db = tc_desc(bbase, K16);
        const uint32_t ap4 = aplane >> 4, bp4 = bplane >> 4;
        const uint32_t idesc0 = idesc & ~(0x3Fu << 17);
        const int maxrun = 256 / NC;
#pragma unroll
        for (int i = 0; i < ND; ++i)
          for (int j0 = 0; j0 < ND - i; j0 += maxrun) {
            const int run = min(maxrun, ND - i - j0);
            const uint32_t idn = idesc0 | ((uint32_t)((NC * run) >> 3) << 17);
            for (int ks = 0; ks < K16 / 16; ++ks)
              tc_mma(tmem + (uint32_t)((i + j0) * NC), da + i * ap4 + ks * 16, db + j0 * bp4 + ks * 16, idn,
                     (i > 0 || ks > 0) ? 1u : 0u);
          }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb)
                     : "memory");
      }
      __syncwarp();
    } else {
      load_tile(tile + gridDim.x);  // registers only: the digit planes are in use
    }
    // row-wise epilogue (all p <= 64 columns in this block, p even, aligned
    // blocks): warp w owns rows w + 16 k (k < 8), lane l columns 2l, 2l + 1
    // (lanes with 2l >= p idle); the first row's elementwise operands are
    // fetched now, each later row's one row ahead
    const bool rowwise = a.vec16 && col0 == 0 && p <= 64 && (p & 1) == 0;
    const bool lact = 2 * lane < p;
    float4 q0 = make_float4(0.f, 0.f, 0.f, 0.f), q1 = q0, q2 = q0;
    auto fetch_row = [&](int k) {
      const int64_t R = r0 + warp + 16 * k;
      if (R < n && lact) {
        const int64_t idx = R * p + col0 + 2 * lane;
        if (a.ne > 0) q0 = *reinterpret_cast<const float4*>(a.E[0] + idx);
        if (a.ne > 1) q1 = *reinterpret_cast<const float4*>(a.E[1] + idx);
        if (a.dot_with) q2 = *reinterpret_cast<const float4*>(a.dot_with + idx);
      }
    };
    if (rowwise && !issuer) fetch_row(0);
    const bool done = issuer || tc_wait(mb, phase, wait_limit);
    phase ^= 1u;
    if (__syncthreads_or(!done)) {
      failed = true;
      break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // (c) epilogue, part 1: warp w reads TMEM lanes 32 (w % 4) .. + 31 (its
    // rows) and the column quarter w / 4, 4 columns at a time; the combined
    // and scaled products go to shared memory (the left digit planes' space,
    // free once the products completed and sized for both), row stride
    // NC + 2 float2 so that every row starts on 16 bytes (16-byte stores and
    // loads, four wavefronts per warp access)
    float2* stage = reinterpret_cast<float2*>(Ad);
    const int ss = NC + 2;
    if (!issuer) {
      const int row = 32 * (warp & 3) + lane;
      const uint32_t lanes = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
      const int quarter = NC / 4, cbeg = (warp >> 2) * quarter;
      for (int c0 = cbeg; c0 < cbeg + quarter; c0 += 4) {
        uint32_t v[ND][4];
#pragma unroll
        for (int g = 0; g < ND; ++g) tc_ld4(v[g], lanes + (uint32_t)(g * NC + c0));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        float2 y[4];
#pragma unroll
        for (int e2 = 0; e2 < 4; ++e2) {
          float S[ND];
#pragma unroll
          for (int g = 0; g < ND; ++g) S[g] = __uint_as_float(v[g][e2]);
          const float2 w = combine_groups_fast<ND, 4>(S);
          const int sc = Er[row] + Fs[c0 + e2] - 14;
          if (sc >= -126) {
            const float f = exp2i(sc);
            y[e2] = make_float2(w.x * f, w.y * f);
          } else {
            const float f1 = exp2i(sc / 2), f2 = exp2i(sc - sc / 2);
            y[e2] = make_float2(w.x * f1 * f2, w.y * f1 * f2);
          }
        }
        float4* d4 = reinterpret_cast<float4*>(stage + row * ss + c0);
        d4[0] = make_float4(y[0].x, y[0].y, y[1].x, y[1].y);
        d4[1] = make_float4(y[2].x, y[2].y, y[3].x, y[3].y);
      }
    }
    __syncthreads();
    // part 2: row-contiguous pass over the tile: elementwise terms, dots and
    // the store, coalesced
    if (rowwise) {
      if (!issuer)
#pragma unroll 1
      for (int k = 0; k < TC_M / 16; ++k) {
        const int rr = warp + 16 * k;
        const int64_t R = r0 + rr;
        const float4 e0 = q0, e1 = q1, w2 = q2;
        if (k + 1 < TC_M / 16) fetch_row(k + 1);
        if (R >= n) continue;
        float2 y0 = make_float2(0.f, 0.f), y1 = y0;
        if (lact) {
          const float4 sv = *reinterpret_cast<const float4*>(stage + rr * ss + 2 * lane);
          y0 = make_float2(sv.x, sv.y);
          y1 = make_float2(sv.z, sv.w);
        }
        if (a.ne > 0) {
          y0 = df_add(y0, df_mul(a.ce[0], make_float2(e0.x, e0.y)));
          y1 = df_add(y1, df_mul(a.ce[0], make_float2(e0.z, e0.w)));
        }
        if (a.ne > 1) {
          y0 = df_add(y0, df_mul(a.ce[1], make_float2(e1.x, e1.y)));
          y1 = df_add(y1, df_mul(a.ce[1], make_float2(e1.z, e1.w)));
        }
        if (a.dot_self) {
          df_dot_acc(dacc0, y0, y0);
          df_dot_acc(dacc0, y1, y1);
        }
        if (a.dot_with) {
          df_dot_acc(dacc1, y0, make_float2(w2.x, w2.y));
          df_dot_acc(dacc1, y1, make_float2(w2.z, w2.w));
        }
        if (lact) *reinterpret_cast<float4*>(a.out + R * p + 2 * lane) = make_float4(y0.x, y0.y, y1.x, y1.y);
        if (a.rinf_part) {  // this row's sum_j |hi(out[r, j])|, the same in every lane
          float rs = fabsf(y0.x) + fabsf(y1.x);
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) rs += __shfl_xor_sync(0xffffffffu, rs, o);
          rmax = fmaxf(rmax, rs);
        }
      }
    } else
    for (int e = tid; e < TC_M * NC; e += TC_THREADS) {
      const int rr = e / NC, cc = e - rr * NC;
      const int64_t R = r0 + rr;
      const int C = col0 + cc;
      if (R >= n || C >= p) continue;
      float2 y = stage[rr * ss + cc];
      const int64_t idx = R * p + C;
#pragma unroll
      for (int m = 0; m < 2; ++m)  // constant indices keep the arguments in parameter space
        if (m < a.ne) y = df_add(y, df_mul(a.ce[m], a.E[m][idx]));
      if (a.dot_self) df_dot_acc(dacc0, y, y);
      if (a.dot_with) df_dot_acc(dacc1, y, a.dot_with[idx]);
      a.out[idx] = y;
    }
    // the next tile rewrites Er and the digit planes: every warp leaves the
    // epilogue first
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
  }
  if (failed) {
    // a product that did not complete in time: count it, drain the tensor
    // core (bounded), poison this block's rows so the caller sees non-finite
    // values, and release the tensor memory
    if (tid == 0) atomicAdd(&g_oz_tc_timeouts, 1);
    tc_wait(mb, phase ^ 1u, TC_WAIT_LIMIT);  // the tile's one pending commit
    tc_drain(issuer && lane == 0, smem_addr(mbar + 1));
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x)
      for (int e = tid; e < TC_M * NC; e += TC_THREADS) {
        const int64_t R = tile * TC_M + e / NC;
        const int c = e % NC;
        if (R < n && col0 + c < p) a.out[R * p + col0 + c] = make_float2(NAN, NAN);
      }
  }
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS));
  if (a.dot_part) {
    __shared__ float2 red[2][TC_THREADS / 32];
    dacc0 = df_acc_done(dacc0);  // the running sums were left unnormalised
    dacc1 = df_acc_done(dacc1);
    for (int o = 16; o > 0; o >>= 1) {
      float2 t0 = make_float2(__shfl_xor_sync(0xffffffffu, dacc0.x, o), __shfl_xor_sync(0xffffffffu, dacc0.y, o));
      float2 t1 = make_float2(__shfl_xor_sync(0xffffffffu, dacc1.x, o), __shfl_xor_sync(0xffffffffu, dacc1.y, o));
      dacc0 = df_add(dacc0, t0);
      dacc1 = df_add(dacc1, t1);
    }
    if ((tid & 31) == 0) {
      red[0][warp] = dacc0;
      red[1][warp] = dacc1;
    }
    __syncthreads();
    if (tid == 0) {
      float2 s0 = make_float2(0.f, 0.f), s1 = make_float2(0.f, 0.f);
      for (int w = 0; w < TC_THREADS / 32; ++w) {
        s0 = df_add(s0, red[0][w]);
        s1 = df_add(s1, red[1][w]);
      }
      const int b = blockIdx.y * gridDim.x + blockIdx.x;
      a.dot_part[2 * b] = s0;
      a.dot_part[2 * b + 1] = s1;
    }
  }
  if (a.rinf_part) {
    __shared__ float redm[TC_THREADS / 32];
    if (lane == 0) redm[warp] = rmax;
    __syncthreads();
    if (tid == 0) {
      float m = 0.f;
      for (int w = 0; w < TC_THREADS / 32; ++w) m = fmaxf(m, redm[w]);
      a.rinf_part[blockIdx.y * gridDim.x + blockIdx.x] = m;
    }
  }
}

// ---------------------------------------------------------------------------
// oz_gram: G = U^T V. Output in 64 x 64 blocks (blockIdx.y), rows in chunks of
// GR_KC = 64 processed by the blocks of blockIdx.x in turn. 16 warps, each a
// 16 x 16 output tile (2 n-tiles); per chunk the column exponents are taken
// over the chunk's rows, so each chunk's digit products are exact, and the
// chunk results are accumulated in df64 registers. The next chunk's raw rows
// are fetched with cp.async while the current chunk is on the tensor cores.
// ---------------------------------------------------------------------------
constexpr int GR_KC = 64;
constexpr int GR_THREADS = 512;
constexpr int GR_STRIDE = 64 + 8;

size_t oz_gram_smem(int nd = ND) {
  return (size_t)2 * nd * GR_KC * GR_STRIDE * 2 + (size_t)2 * GR_KC * 64 * sizeof(float2) +
         (4 * 128 + 4 * 64) * sizeof(int) + 64;
}

__device__ __forceinline__ void gr_stage(int64_t n, int p, int q, const float2* U, const float2* V,
                                         int i0, int j0, int64_t r0, float2* rawU, float2* rawV) {
  for (int e = threadIdx.x; e < 2 * GR_KC * 64; e += GR_THREADS) {
    const bool isv = e >= GR_KC * 64;
    const int e2 = isv ? e - GR_KC * 64 : e;
    const int r = e2 >> 6, c = e2 & 63;
    const int64_t R = r0 + r;
    const int ld = isv ? q : p, c0 = isv ? j0 : i0;
    const bool ok = R < n && c0 + c < ld;
    const float2* src = isv ? V : U;
    cp_async8((isv ? rawV : rawU) + e2, src + (ok ? R * ld + c0 + c : 0), ok);
  }
  cp_async_commit();
}

template <int NDT>
__global__ void __launch_bounds__(GR_THREADS)
oz_gram_kernel(int64_t n, int p, int q, const float2* __restrict__ U, const float2* __restrict__ V,
               int sym, int nbj, float2* part) {
  extern __shared__ __align__(16) unsigned char smem[];
  __nv_bfloat16* Ud = reinterpret_cast<__nv_bfloat16*>(smem);
  __nv_bfloat16* Vd = Ud + (size_t)NDT * GR_KC * GR_STRIDE;
  float2* rawU = reinterpret_cast<float2*>(Vd + (size_t)NDT * GR_KC * GR_STRIDE);
  float2* rawV = rawU + GR_KC * 64;
  int* cmx = reinterpret_cast<int*>(rawV + GR_KC * 64);  // [4][128] partial column maxima
  int* Eu = cmx + 4 * 128;
  int* Ev = Eu + 64;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int bi, bj;
  {
    int b = blockIdx.y;
    if (sym) {  // upper-triangular enumeration
      bi = 0;
      while (b >= nbj - bi) {
        b -= nbj - bi;
        ++bi;
      }
      bj = bi + b;
    } else {
      bi = b / nbj;
      bj = b - bi * nbj;
    }
  }
  const int i0 = bi * 64, j0 = bj * 64;
  const int wi = warp >> 2, wj = warp & 3;
  const bool active = (i0 + wi * 16 < p) && (j0 + wj * 16 < q) && !(sym && bi == bj && wi > wj);
  float2 res[2][4];
#pragma unroll
  for (int t = 0; t < 2; ++t)
#pragma unroll
    for (int e = 0; e < 4; ++e) res[t][e] = make_float2(0.f, 0.f);
  const int64_t nchunks = (n + GR_KC - 1) / GR_KC;
  if ((int64_t)blockIdx.x < nchunks)
    gr_stage(n, p, q, U, V, i0, j0, (int64_t)blockIdx.x * GR_KC, rawU, rawV);
  for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    cp_async_wait_all();
    __syncthreads();
    // (a) column maxima of |hi|: thread -> (column c of [U V], group of 16 rows)
    {
      const int c = tid & 127, g = tid >> 7;
      const float2* src = c < 64 ? rawU : rawV;
      const int cc = c & 63;
      float mx = 0.f;
#pragma unroll 4
      for (int r = g * 16; r < g * 16 + 16; ++r) mx = fmaxf(mx, fabsf(src[r * 64 + cc].x));
      cmx[g * 128 + c] = __float_as_int(mx);
    }
    __syncthreads();
    if (tid < 128) {
      float mx = fmaxf(fmaxf(__int_as_float(cmx[tid]), __int_as_float(cmx[128 + tid])),
                       fmaxf(__int_as_float(cmx[256 + tid]), __int_as_float(cmx[384 + tid])));
      if (tid < 64) Eu[tid] = exponent_above(mx);
      else Ev[tid - 64] = exponent_above(mx);
    }
    __syncthreads();
    // (b) digits: one thread per (row, pair of columns), U then V
    for (int e = tid; e < 2 * GR_KC * 32; e += GR_THREADS) {
      const bool isv = e >= GR_KC * 32;
      const int e2 = isv ? e - GR_KC * 32 : e;
      const int r = e2 >> 5, c = 2 * (e2 & 31);
      const float2* src = isv ? rawV : rawU;
      const float4 xx = *reinterpret_cast<const float4*>(src + r * 64 + c);
      const int* Ex = isv ? Ev : Eu;
      float d0[NDT], d1[NDT];
      digitsN<NDT>(xx.x, xx.y, Ex[c], d0);
      digitsN<NDT>(xx.z, xx.w, Ex[c + 1], d1);
      __nv_bfloat16* dst = isv ? Vd : Ud;
#pragma unroll
      for (int i = 0; i < NDT; ++i)
        *reinterpret_cast<uint32_t*>(dst + ((size_t)i * GR_KC + r) * GR_STRIDE + c) = pack_bf16x2(d0[i], d1[i]);
    }
    __syncthreads();  // digits ready, raw buffers free: prefetch the next chunk
    if (ch + gridDim.x < nchunks)
      gr_stage(n, p, q, U, V, i0, j0, (ch + gridDim.x) * GR_KC, rawU, rawV);
    if (active) {
      float acc[NDT][2][4];
#pragma unroll
      for (int g = 0; g < NDT; ++g)
#pragma unroll
        for (int t = 0; t < 2; ++t)
#pragma unroll
          for (int e = 0; e < 4; ++e) acc[g][t][e] = 0.0f;
#pragma unroll
      for (int ks = 0; ks < GR_KC / 16; ++ks) {
        uint32_t A[NDT][4];
        const int qq = lane >> 3;
#pragma unroll
        for (int i = 0; i < NDT; ++i)
          ldsm_x4_t(A[i], Ud + ((size_t)i * GR_KC + ks * 16 + (lane & 7) + (qq >> 1) * 8) * GR_STRIDE +
                              wi * 16 + (qq & 1) * 8);
#pragma unroll
        for (int t = 0; t < 2; ++t) {
#pragma unroll
          for (int j = 0; j < NDT; ++j) {
            uint32_t B[2];
            const int l16 = lane & 15;
            ldsm_x2_t(B, Vd + ((size_t)j * GR_KC + ks * 16 + (l16 & 7) + (l16 >> 3) * 8) * GR_STRIDE +
                             wj * 16 + t * 8);
#pragma unroll
            for (int i = 0; i < NDT - j; ++i) mma_bf16(acc[i + j][t], A[i], B);
          }
        }
      }
#pragma unroll
      for (int t = 0; t < 2; ++t)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int ii = wi * 16 + (lane >> 2) + (e >> 1) * 8;
          const int jj = wj * 16 + t * 8 + (lane & 3) * 2 + (e & 1);
          float S[NDT];
#pragma unroll
          for (int g = 0; g < NDT; ++g) S[g] = acc[g][t][e];
          float2 w = combine_groups<NDT>(S);
          int sc = Eu[ii] + Ev[jj] - 14;
          float f1 = exp2i(sc / 2), f2 = exp2i(sc - sc / 2);
          res[t][e] = df_add(res[t][e], make_float2(w.x * f1 * f2, w.y * f1 * f2));
        }
    }
  }
  cp_async_wait_all();
  if (active) {
    float2* out = part + ((size_t)blockIdx.x * gridDim.y + blockIdx.y) * 64 * 64;
#pragma unroll
    for (int t = 0; t < 2; ++t)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int ii = wi * 16 + (lane >> 2) + (e >> 1) * 8;
        const int jj = wj * 16 + t * 8 + (lane & 3) * 2 + (e & 1);
        out[ii * 64 + jj] = res[t][e];
      }
  }
}

// ---------------------------------------------------------------------------
// oz_gram on the 5th-generation tensor cores, one 64 x 64 output block per
// blockIdx.y (p, q <= 128), and the 7-digit split. Rows go in exponent chunks of EC rows (256 for U == V, 160
// otherwise), staged raw in shared memory by cp.async; the column exponents
// are taken over the whole chunk, and the chunk's digit-pair products are
// summed in tensor memory over its sub-chunks of SK rows (32, resp. 16) before
// one df64 combination per chunk. The group sums stay exact integers: per row
// |d_0 d_0| <= 2^14 and every other digit product is at most 128 * 72, so even
// the seven pairs of group 6 sum to less than 2^24 over 256 rows.
//
// The products are M = 128, N = 64 MMAs whose A operand stacks two
// consecutive digit planes of U, [U_2m; U_2m+1] (the planes are adjacent in
// shared memory, so this is one K-major operand of 128 rows). With B = V_j
// the top half (TMEM lanes 0..63) gets U_2m^T V_j, group 2m + j, and the
// bottom half (lanes 64..127) U_2m+1^T V_j, group 2m + 1 + j, both in the
// accumulator block h = 2m + j. So block h holds the even-digit part of
// group h in its top lanes and the odd-digit part of group h + 1 in its
// bottom lanes (block 6's bottom half, "group 7", is never read); 16 MMAs per
// 16 rows instead of 28. The two parts are combined separately (each an
// exact integer sum) and added once at the end of the kernel.
//
// Digit planes are double-buffered: sub-chunk s + 1 is cut while the tensor
// core works on sub-chunk s (one mbarrier per buffer). Sixteen worker warps
// stage, cut and combine; a seventeenth warp only issues the products, so
// that the issue never holds up a worker at the next barrier.
// ---------------------------------------------------------------------------
constexpr int TG_WORKERS = 512;
constexpr int TG_THREADS = TG_WORKERS + 32;
constexpr int TG_RS = 66;              // raw row stride in float2 (528 B: rows on 16 B)
// Chunk geometry: U == V: 256-row exponent chunks in 32-row sub-chunks, raw
// stage 256 rows, digit buffers of 7 planes + a pad plane (32 KB); U != V:
// 160-row chunks in 16-row sub-chunks, raw stage 160 rows of U then 160 of
// V, digit buffers of 7 + 7 planes (28 KB). Per row a stacked accumulator
// gains at most 4 * 128 * 72 < 28800 < 2^24 / 256, so both stay exact.
template <bool SYM>
struct TgGeom {
  static constexpr int EC = SYM ? 256 : 160;
  static constexpr int SK = SYM ? 32 : 16;
  static constexpr int RAWR = SYM ? EC : 2 * EC;    // raw stage rows
  static constexpr int NG = RAWR / 32;              // 32-row groups of the maxima pass
  static constexpr uint32_t DBUF = SYM ? 32768u : 28672u;
  static constexpr size_t smem() {
    return (size_t)RAWR * TG_RS * sizeof(float2) + 2 * DBUF + NG * 64 * sizeof(float) + 128 * sizeof(int) +
           128 * sizeof(float) + 64;
  }
};
static_assert(TgGeom<true>::smem() <= 227 * 1024 && TgGeom<false>::smem() <= 227 * 1024, "shared memory");
static_assert(TgGeom<false>::EC % (2 * TgGeom<false>::SK) == 0 && TgGeom<true>::EC % (2 * TgGeom<true>::SK) == 0,
              "an even number of sub-chunks per chunk");

size_t oz_gram_tc_smem(bool sym) { return sym ? TgGeom<true>::smem() : TgGeom<false>::smem(); }

// digitsN with the frame's scale s = 2^(7-E) given; the rounding constants
// 1.5 * 2^(23 - 7i) as literals
template <int N>
__device__ __forceinline__ void digits_scaled(float h, float l, float s, float d[N]) {
  constexpr float kRound[7] = {12582912.0f, 98304.0f, 768.0f, 6.0f, 0.046875f, 0.0003662109375f,
                               2.86102294921875e-06f};
  float a = __fmul_rn(h, s);
  const float b = __fmul_rn(l, s);
#pragma unroll
  for (int i = 0; i < N; ++i) {
    if (i == 3) a = __fadd_rn(a, b);
    const float di = __fsub_rn(__fadd_rn(a, kRound[i]), kRound[i]);
    d[i] = di;
    if (i + 1 < N) a = __fsub_rn(a, di);
  }
}


__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool valid) {
  uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
  int sz = valid ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(sz));
}

template <bool SYM>
__global__ void __launch_bounds__(TG_THREADS, 1)
oz_gram_tc_kernel(int64_t n, int p, int q, const float2* __restrict__ U, const float2* __restrict__ V,
                  int vec16, float2* part, int nbj, int tri) {
  using Geo = TgGeom<SYM>;
  // the 64 x 64 output block of this CTA: U's columns 64 bi .., V's 64 bj ..
  // (blockIdx.y over the nbi x nbj blocks, or with tri over the upper
  // triangle bi <= bj row by row)
  int bi = 0, bj = (int)blockIdx.y;
  if (tri) {
    int y = (int)blockIdx.y;
    while (y >= nbj - bi) {
      y -= nbj - bi;
      ++bi;
    }
    bj = bi + y;
  } else {
    bi = (int)blockIdx.y / nbj;
    bj = (int)blockIdx.y - bi * nbj;
  }
  const int cu0 = 64 * bi, cv0 = 64 * bj;
  const int wu = min(64, p - cu0), wv = min(64, q - cv0);  // live columns of the block
  constexpr int EC = Geo::EC, SK = Geo::SK, NSUB = EC / SK, RAWR = Geo::RAWR, NG = Geo::NG;
  constexpr uint32_t TG_DBUF = Geo::DBUF;
  constexpr uint32_t plane = 64u * SK * 2;  // one digit plane: 64 columns x SK rows, bf16
  extern __shared__ __align__(16) unsigned char tg_smem[];
  float2* raw = reinterpret_cast<float2*>(tg_smem);
  unsigned char* dig = tg_smem + (size_t)RAWR * TG_RS * sizeof(float2);
  float* cmx = reinterpret_cast<float*>(dig + 2 * TG_DBUF);  // [NG][64] partial column maxima
  int* Eu = reinterpret_cast<int*>(cmx + NG * 64);  // after all NG groups of maxima
  int* Ev = Eu + 64;
  float* Fu = reinterpret_cast<float*>(Ev + 64);  // the exponents as scales 2^(E-7)
  float* Fv = Fu + 64;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(Fv + 64);     // one per digit buffer, then the drain
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 3);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool issuer = warp == TG_WORKERS / 32;
  // the pad plane after the 7 planes of U (U == V) is read by the bottom half
  // of the [U_6; U_7] operand, whose products land in the unused "group 7"
  if (SYM && !issuer)
    for (int e = tid; e < 2 * (int)(plane / 16); e += TG_WORKERS) {
      const int b = e / (int)(plane / 16), o = e - b * (int)(plane / 16);
      *reinterpret_cast<uint4*>(dig + b * TG_DBUF + 7 * plane + 16 * o) = make_uint4(0u, 0u, 0u, 0u);
    }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tslot)),
                 "r"(TC_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(mbar)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(mbar + 1)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(mbar + 2)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const int wait_limit = g_oz_wait_limit;
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(64 >> 3) << 17) |
                         ((uint32_t)(128 >> 4) << 24);
  const uint32_t dbase = smem_addr(dig);
  const uint32_t mb0 = smem_addr(mbar), mb1 = smem_addr(mbar + 1);
  uint32_t ph0 = 0u, ph1 = 0u;  // phases of the two buffers' barriers
  const float* Fvv = SYM ? Fu : Fv;
  // combine: worker warp w reads TMEM lanes 32 (w % 4) .. + 31, i.e. output
  // row a = 32 (w % 2) + lane of the top (w % 4 < 2) or bottom half, columns
  // 16 (w / 4) .. + 15
  const int quarter = warp & 3, arow = 32 * (quarter & 1) + lane, cb = 16 * ((warp >> 2) & 3);
  const bool top = quarter < 2;
  float2 res[16];
#pragma unroll
  for (int e = 0; e < 16; ++e) res[e] = make_float2(0.f, 0.f);
  bool failed = false;
  const int64_t nchunks = (n + EC - 1) / EC;

  // raw rows of chunk ch (workers): U rows (256, or 160 then V's 160),
  // zero-filled outside the matrix
  auto stage = [&](int64_t ch) {
    const int64_t r0 = ch * EC;
    if (vec16) {
      for (int e = tid; e < RAWR * 32; e += TG_WORKERS) {
        const int row = e >> 5, c = 2 * (e & 31);
        const bool isv = !SYM && row >= EC;
        const int64_t R = r0 + (isv ? row - EC : row);
        const int ld = isv ? q : p;
        const float2* src = (isv ? V + cv0 : U + cu0);
        const bool ok = R < n && c < (isv ? wv : wu);
        cp_async16(raw + row * TG_RS + c, src + (ok ? R * ld + c : 0), ok);
      }
    } else {
      for (int e = tid; e < RAWR * 64; e += TG_WORKERS) {
        const int row = e >> 6, c = e & 63;
        const bool isv = !SYM && row >= EC;
        const int64_t R = r0 + (isv ? row - EC : row);
        const int ld = isv ? q : p;
        const float2* src = (isv ? V + cv0 : U + cu0);
        const bool ok = R < n && c < (isv ? wv : wu);
        cp_async8(raw + row * TG_RS + c, src + (ok ? R * ld + c : 0), ok);
      }
    }
    cp_async_commit();
  };

  // the rows of sub-chunk sub only (SK rows of U, and of V), into the raw
  // rows that sub-chunk occupies: restaged for the next chunk as soon as the
  // current chunk's sub-chunk has been cut, so that the copies spread over
  // the chunk instead of queueing at its end
  auto stage_sub = [&](int64_t ch, int sub) {
    const int64_t r0 = ch * EC + sub * SK;
    if (vec16) {
      for (int e = tid; e < 2 * SK * 32 / (SYM ? 2 : 1); e += TG_WORKERS) {
        const int rr = e >> 5, c = 2 * (e & 31);
        const bool isv = !SYM && rr >= SK;
        const int lr = isv ? rr - SK : rr;
        const int64_t R = r0 + lr;
        const int ld = isv ? q : p;
        const float2* src = (isv ? V + cv0 : U + cu0);
        const bool ok = R < n && c < (isv ? wv : wu);
        cp_async16(raw + ((isv ? EC : 0) + sub * SK + lr) * TG_RS + c, src + (ok ? R * ld + c : 0), ok);
      }
    } else {
      for (int e = tid; e < 2 * SK * 64 / (SYM ? 2 : 1); e += TG_WORKERS) {
        const int rr = e >> 6, c = e & 63;
        const bool isv = !SYM && rr >= SK;
        const int lr = isv ? rr - SK : rr;
        const int64_t R = r0 + lr;
        const int ld = isv ? q : p;
        const float2* src = (isv ? V + cv0 : U + cu0);
        const bool ok = R < n && c < (isv ? wv : wu);
        cp_async8(raw + ((isv ? EC : 0) + sub * SK + lr) * TG_RS + c, src + (ok ? R * ld + c : 0), ok);
      }
    }
    cp_async_commit();
  };

  // digit item of this worker (one per sub-chunk): column c, rows
  // 4 qd .. 4 qd + 3 of the sub-chunk, of U or (isv) of V. Lanes cover 8
  // columns x 2 quads x 2 row octets, so a warp's 8-byte stores fill 2 x 32
  // banks and its raw loads 2 x 32 banks.
  const bool isv = !SYM && tid >= 256;
  const int loc = SYM ? tid : (tid & 255);
  const int ic = 8 * ((loc >> 5) & 7) + (lane & 7);
  const int iq = 2 * (((lane >> 4) & 1) + 2 * (loc >> 8)) + ((lane >> 3) & 1);
  const int irow = (isv ? EC : 0) + 4 * iq;

  if (!issuer && (int64_t)blockIdx.x < nchunks) stage(blockIdx.x);
  for (int64_t ch = blockIdx.x; ch < nchunks && !failed; ch += gridDim.x) {
    if (!issuer) cp_async_wait_all();
    __syncthreads();
    // (a) column maxima of |hi| over the chunk: thread -> column c, 32 rows
    // of raw row group g (g < NG / 2: U, else V when U != V)
    if (!issuer) {
      const int c = tid & 63;
      for (int g = tid >> 6; g < NG; g += TG_WORKERS / 64) {
        float mx = 0.f;
#pragma unroll 8
        for (int k = 0; k < 32; ++k) mx = fmaxf(mx, fabsf(raw[(32 * g + k) * TG_RS + c].x));
        cmx[g * 64 + c] = mx;
      }
    }
    __syncthreads();
    if (tid < (SYM ? 64 : 128)) {
      const int c = tid & 63, g0 = (tid < 64) ? 0 : NG / 2, ng = SYM ? NG : NG / 2;
      float m = 0.f;
      for (int g = g0; g < g0 + ng; ++g) m = fmaxf(m, cmx[g * 64 + c]);
      const int E = exponent_above(m);
      if (tid < 64) {
        Eu[c] = E;
        Fu[c] = exp2i(E - 7);
      } else {
        Ev[c] = E;
        Fv[c] = exp2i(E - 7);
      }
    }
    __syncthreads();
    // (b) sub-chunks: cut into digit buffer s % 2, products on the tensor core
    for (int s = 0; s < NSUB; ++s) {
      const int buf = s & 1;
      bool ok = true;
      // the products of sub-chunk s - 2 read this buffer; the phase bit moves
      // on only once every thread saw them complete, so that after a wait
      // that ran out ph0 / ph1 still name each barrier's pending commit
      if (s >= 2 && !issuer) ok = tc_wait(buf ? mb1 : mb0, buf ? ph1 : ph0, wait_limit);
      if (!issuer && ok) {
        unsigned char* dst = dig + buf * TG_DBUF + (isv ? 7 * plane : 0);
        const int r = irow + s * SK;
        const float scut = exp2i(7 - (isv ? Ev : Eu)[ic]);
        float d[4][ND];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const float2 x = raw[(r + t) * TG_RS + ic];
          digits_scaled<ND>(x.x, x.y, scut, d[t]);
        }
#pragma unroll
        for (int i = 0; i < ND; ++i)
          *reinterpret_cast<uint2*>(dst + i * plane + tc_off(ic, 4 * iq, SK)) =
              make_uint2(pack_bf16x2(d[0][i], d[1][i]), pack_bf16x2(d[2][i], d[3][i]));
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
      if (s >= 2) {
        if (buf) ph1 ^= 1u;
        else ph0 ^= 1u;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (issuer) {
        if (lane == 0) {
          const uint32_t ab = dbase + buf * TG_DBUF, bb = SYM ? ab : ab + 7 * plane;
          const uint64_t da = tc_desc(ab, SK), db = tc_desc(bb, SK);
          const uint32_t acc0 = s > 0 ? 1u : 0u;
          // V's planes j0 .. j0 + run - 1 are adjacent in shared memory and so
          // are their accumulator blocks 2m + j0 .. in tensor memory: one
          // MMA of N = 64 run per run of up to 4 planes (6 MMAs per 16 rows
          // instead of 16 of N = 64; the per-instruction cost dominates at
          // N = 64)
          const uint32_t idesc0 = idesc & ~(0x3Fu << 17);
#pragma unroll
          for (int m = 0; m < 4; ++m)
#pragma unroll
            for (int j0 = 0; j0 < ND - 2 * m; j0 += 4) {
              const int run = (ND - 2 * m - j0) < 4 ? (ND - 2 * m - j0) : 4;
              const uint32_t idn = idesc0 | ((uint32_t)((64 * run) >> 3) << 17);
#pragma unroll
              for (int ks = 0; ks < SK / 16; ++ks)
                tc_mma(tmem + (uint32_t)((2 * m + j0) * 64), da + ((2 * m * plane + ks * 256) >> 4),
                       db + ((j0 * plane + ks * 256) >> 4), idn, (m > 0 || ks > 0) ? 1u : acc0);
            }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           buf ? mb1 : mb0)
                       : "memory");
        }
        __syncwarp();
      } else if (ch + gridDim.x < nchunks) {
        stage_sub(ch + gridDim.x, s);  // sub-chunk s's raw rows are free (every worker cut it)
      }
    }
    if (failed) break;
    // (c) the last two sub-chunks' products, then the combination
    bool ok = true;
    if (!issuer) {
      ok = tc_wait(mb0, ph0, wait_limit);
      ok = tc_wait(mb1, ph1, wait_limit) && ok;
    }
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    ph0 ^= 1u;
    ph1 ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!issuer) {
      const float fu = Fu[arow];
      const uint32_t lanes = tmem + ((uint32_t)(32 * quarter) << 16);
#pragma unroll
      for (int c0 = 0; c0 < 16; c0 += 4) {
        uint32_t v[ND][4];
#pragma unroll
        for (int h = 0; h < ND; ++h)
          if (top || h < ND - 1) tc_ld4(v[h], lanes + (uint32_t)(h * 64 + cb + c0));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          float S[ND];
#pragma unroll
          for (int h = 0; h < ND; ++h) S[h] = __uint_as_float(v[h][e]);
          // top: groups 0..6 (even digits of U); bottom: groups 1..6 (odd
          // digits), block h holding group h + 1, each sum carrying its weight
          // groups 4..6 in float32
          const float2 w = top ? combine_groups_fast<ND, 4>(S) : combine_groups_fast<ND - 1, 3>(S);
          const float fv = Fvv[cb + c0 + e];
          res[c0 + e] = df_add(res[c0 + e], make_float2(w.x * fu * fv, w.y * fu * fv));
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
  }
  if (!issuer) cp_async_wait_all();
  if (failed) {
    // a product that did not complete in time: count it, drain the tensor
    // core (bounded), and report non-finite partial sums. Each barrier has
    // exactly one pending commit here (sub-chunks s - 2 and s - 1, or the
    // chunk's last two), named by ph0 / ph1; waiting for both lets their
    // arrivals land before the block exits, and the final commit covers
    // anything else issued.
    if (tid == 0) atomicAdd(&g_oz_tc_timeouts, 1);
    tc_wait(mb0, ph0, TC_WAIT_LIMIT);
    tc_wait(mb1, ph1, TC_WAIT_LIMIT);
    tc_drain(issuer && lane == 0, smem_addr(mbar + 2));
#pragma unroll
    for (int e = 0; e < 16; ++e) res[e] = make_float2(NAN, NAN);
  }
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS));
  // odd-digit parts (bottom half) onto the even-digit parts, once per block
  float2* st = raw;  // 64 x 65 float2
  if (!issuer && !top) {
#pragma unroll
    for (int e = 0; e < 16; ++e) st[arow * 65 + cb + e] = res[e];
  }
  __syncthreads();
  if (!issuer && top) {
    float2* out = part + ((size_t)blockIdx.x * gridDim.y + blockIdx.y) * 4096;
#pragma unroll
    for (int e = 0; e < 16; ++e) out[arow * 64 + cb + e] = df_add(res[e], st[arow * 65 + cb + e]);
  }
}

// ---------------------------------------------------------------------------
// oz_gram_tc_ring_kernel: the tcgen05 Gram for 16-byte aligned blocks of even
// width (one 64 x 64 output block per blockIdx.y, as oz_gram_tc_kernel).
//
// The kernel above stages a whole exponent chunk raw, which fills shared
// memory and leaves room for two digit buffers only; its sub-chunk loop then
// waits on the tensor core every other sub-chunk, and the chunk stays short.
// Here the column exponents of a chunk come from two maxima warps that read
// the chunk's rows one chunk ahead of the workers: 1D bulk copies
// (cp.async.bulk, completion counted on an mbarrier per slot, no registers
// held) of whole batches of rows into small per-warp rings of slots, reduced
// from shared memory. The workers then stage the rows raw sub-chunk by
// sub-chunk through a ring of NR slots (16-byte cp.async, NR - 1 sub-chunks
// ahead; the rows come from L2, where the maxima warps' read left them), cut
// them into NB digit buffers with one mbarrier each, and combine once per
// chunk of EC rows (512 for U == V, 384 otherwise: there part of the second
// reads already miss L2, but the fewer combinations pay for it). Exactness of the
// accumulators: as for oz_gram_tc_kernel, 28800 EC < 2^24 for chunks of up
// to 582 rows.
//
// Roles: warps 0..15 stage, cut and combine; warp 16 issues the products;
// warps 17 and 18 compute the maxima, taking alternate batches, each with
// its own ring and copies (reading a chunk's rows costs one warp more issue
// slots than it gets beside four busy workers), and merge their maxima once
// per chunk. Workers and the issuing warp meet at named barrier 1 every
// sub-chunk, the maxima warps at named barrier 2 at each chunk's end; all 19
// warps meet at barrier 0 once per chunk, where the maxima warps hand over
// the next chunk's exponents. Every thread passes the same sequence of
// barrier-0 arrivals whatever fails: a timeout only turns later work off
// (and the partial sums into NaN).
// ---------------------------------------------------------------------------
constexpr int TR_WORKERS = 512;
constexpr int TR_THREADS = TR_WORKERS + 96;  // + the issuing warp + two maxima warps
constexpr int TR_BAR_COUNT = TR_WORKERS + 32;
template <bool SYM, int NDT = ND>
struct TrGeom {
  static constexpr int EC = SYM ? 512 : 384;       // exponent chunk rows
  static constexpr int SK = SYM ? 32 : 16;         // sub-chunk rows
  static constexpr int NSUB = EC / SK;             // sub-chunks per chunk
  static constexpr int NB = 3;                     // digit buffers
  static constexpr int NR = 4;                     // raw slots (staging NR - 1 sub-chunks ahead)
  static constexpr int MSW = SYM ? 3 : 4;          // maxima slots per maxima warp
  static constexpr int MS = 2 * MSW;
  static constexpr int MB = SYM ? 16 : 8;          // rows per operand in one maxima slot
  static constexpr int NMB = EC / MB;              // maxima batches per chunk
  static constexpr uint32_t PLANE = 64u * SK * 2;  // one digit plane: 64 columns x SK rows, bf16
  // U == V: NDT planes and a zero pad plane; U != V: NDT planes of U, NDT of V
  static constexpr uint32_t DBUF = (uint32_t)(SYM ? NDT + 1 : 2 * NDT) * PLANE;
  static constexpr size_t RAW_SLOT = (size_t)32 * TG_RS * sizeof(float2);
  static constexpr size_t MSLOT = (size_t)16 * 64 * sizeof(float2);  // 16 rows of 64 df64
  // raw slots, digit buffers, maxima slots, exponents and scales [2][128]
  // each, the maxima warps' scratch [128], two flags, barriers (digit
  // buffers, drain, maxima slots), TMEM slot
  static constexpr size_t smem() {
    return NR * RAW_SLOT + NB * (size_t)DBUF + MS * MSLOT + 2 * 256 * sizeof(int) + 128 * sizeof(float) + 16 +
           (NB + 1 + MS) * sizeof(uint64_t) + 16;
  }
};
static_assert(TrGeom<true>::smem() <= 227 * 1024 && TrGeom<false>::smem() <= 227 * 1024, "shared memory");
static_assert(TrGeom<true>::NR == 4 && TrGeom<false>::NR == 4, "wait_group<NR - 2> below");
static_assert(TrGeom<false>::NR * TrGeom<false>::RAW_SLOT >= 64 * 65 * sizeof(float2) &&
                  TrGeom<true>::NR * TrGeom<true>::RAW_SLOT >= 64 * 65 * sizeof(float2),
              "final stage fits the raw ring");

size_t oz_gram_tc_ring_smem(bool sym, int nd) {
  return nd == 3 ? (sym ? TrGeom<true, 3>::smem() : TrGeom<false, 3>::smem())
                 : (sym ? TrGeom<true>::smem() : TrGeom<false>::smem());
}

template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// named barrier 2 (the two maxima warps) with an OR over v
__device__ __forceinline__ bool bar2_or(bool v) {
  uint32_t r;
  asm volatile(
      "{\n.reg .pred p, q;\nsetp.ne.u32 p, %1, 0;\nbar.red.or.pred q, 2, 64, p;\nselp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)v)
      : "memory");
  return r != 0;
}

// named barrier 1 (workers and the issuing warp) with an OR over v
__device__ __forceinline__ bool bar1_or(bool v) {
  uint32_t r;
  asm volatile(
      "{\n.reg .pred p, q;\nsetp.ne.u32 p, %1, 0;\nbar.red.or.pred q, 1, %2, p;\nselp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)v), "n"(TR_BAR_COUNT)
      : "memory");
  return r != 0;
}

template <bool SYM, int NDT>
__global__ void __launch_bounds__(TR_THREADS, 1)
oz_gram_tc_ring_kernel(int64_t n, int p, int q, const float2* __restrict__ U, const float2* __restrict__ V,
                       float2* part, int nbj, int tri) {
  using Geo = TrGeom<SYM, NDT>;
  int bi = 0, bj = (int)blockIdx.y;
  if (tri) {
    int y = (int)blockIdx.y;
    while (y >= nbj - bi) {
      y -= nbj - bi;
      ++bi;
    }
    bj = bi + y;
  } else {
    bi = (int)blockIdx.y / nbj;
    bj = (int)blockIdx.y - bi * nbj;
  }
  const int cu0 = 64 * bi, cv0 = 64 * bj;
  const int wu = min(64, p - cu0), wv = min(64, q - cv0);  // live columns (even: p, q even)
  constexpr int EC = Geo::EC, SK = Geo::SK, NSUB = Geo::NSUB, NB = Geo::NB, NR = Geo::NR;
  constexpr int MS = Geo::MS, MSW = Geo::MSW, MB = Geo::MB, NMB = Geo::NMB;
  static_assert(NMB % 2 == 0, "the maxima warps take alternate batches");
  constexpr uint32_t plane = Geo::PLANE, DBUF = Geo::DBUF;
  extern __shared__ __align__(16) unsigned char tr_smem[];
  float2* raw = reinterpret_cast<float2*>(tr_smem);  // NR slots of 32 rows
  unsigned char* dig = tr_smem + NR * Geo::RAW_SLOT;
  float2* mslot = reinterpret_cast<float2*>(dig + NB * DBUF);  // MS slots of 16 rows x 64
  int* Ex = reinterpret_cast<int*>(mslot + MS * 16 * 64);     // [chunk parity][U's 64, V's 64]
  float* Fx = reinterpret_cast<float*>(Ex + 256);              // the same as scales 2^(E-7)
  volatile float* mscr = Fx + 256;                              // maxima warp 1's maxima, [U's 64, V's 64]
  volatile int* flags = reinterpret_cast<volatile int*>(Fx + 384);  // [0] workers failed, [1] maxima failed
  uint64_t* mbar = reinterpret_cast<uint64_t*>(Fx + 384 + 4);  // NB digit buffers, drain, MS maxima slots
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + NB + 1 + MS);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool issuer = warp == TR_WORKERS / 32, maxw = warp > TR_WORKERS / 32;
  const int mw = warp - TR_WORKERS / 32 - 1;  // maxima warp 0 or 1
  const bool worker = tid < TR_WORKERS;
  if (SYM && worker)
    for (int e = tid; e < NB * (int)(plane / 16); e += TR_WORKERS) {
      const int b = e / (int)(plane / 16), o = e - b * (int)(plane / 16);
      *reinterpret_cast<uint4*>(dig + b * DBUF + NDT * plane + 16 * o) = make_uint4(0u, 0u, 0u, 0u);
    }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tslot)),
                 "r"(TC_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int b = 0; b < NB + 1 + MS; ++b)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(mbar + b)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    flags[0] = 0;
    flags[1] = 0;
  }
  const int nchunks = (int)((n + EC - 1) / EC);  // n < 2^34 (checked by the caller)
  const int nmy = (int)blockIdx.x < nchunks ? (nchunks - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int G = nmy * NSUB;
  const uint32_t mbase = smem_addr(mbar), msbase = smem_addr(mbar + NB + 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const int wait_limit = g_oz_wait_limit;

  if (maxw) {
    // ---- the maxima warps: chunk j's column maxima, one chunk ahead ----
    // batch gb = j NMB + b covers rows b MB .. b MB + MB - 1 of this CTA's
    // chunk j: cells 0..MB-1 hold U's rows, cells MB..15 V's (U != V). The
    // warps take alternate batches (b % 2 == mw; NMB is even), each through
    // its own ring of MSW slots, and merge their maxima once per chunk.
    // Where the block spans whole rows (64 columns or fewer), a batch's rows
    // are contiguous: one copy per operand, rows ld apart in the slot;
    // otherwise one copy per row, rows 64 apart (the copy engine's cost per
    // copy made 16 copies of 512 B per batch the bottleneck).
    const int total = nmy * NMB / 2;  // this warp's batches
    const bool contU = wu == p, contV = SYM ? contU : wv == q;
    const int strU = contU ? p : 64, strV = contV ? q : 64;
    auto batch_rows = [&](int t, int64_t& R0) {  // first row of this warp's t-th batch
      const int gb = 2 * t + mw;
      const int j = gb / NMB, b = gb - j * NMB;
      R0 = ((int64_t)blockIdx.x + (int64_t)j * gridDim.x) * EC + (int64_t)b * MB;
    };
    auto slot_of = [&](int t) { return mslot + (size_t)(mw * MSW + t % MSW) * 16 * 64; };
    auto bar_of = [&](int t) { return msbase + 8u * (uint32_t)(mw * MSW + t % MSW); };
    auto issue = [&](int t) {
      int64_t R0;
      batch_rows(t, R0);
      const int64_t left = n - R0;
      const int nv = left <= 0 ? 0 : (left < MB ? (int)left : MB);
      float2* sl = slot_of(t);
      uint32_t bytes = 0;
      const float2* src = U;
      float2* dst = sl;
      if (contU) {
        if (lane == 0 && nv > 0) {
          bytes = (uint32_t)nv * (uint32_t)p * 8u;
          src = U + (size_t)R0 * p;
        }
      } else if (lane < MB && lane < nv) {
        bytes = (uint32_t)wu * 8u;
        src = U + (size_t)(R0 + lane) * p + cu0;
        dst = sl + lane * 64;
      }
      if (!SYM) {
        if (contV) {
          if (lane == 16 && nv > 0) {
            bytes = (uint32_t)nv * (uint32_t)q * 8u;
            src = V + (size_t)R0 * q;
            dst = sl + MB * 64;
          }
        } else if (lane >= 16 && lane < 16 + MB && lane - 16 < nv) {
          bytes = (uint32_t)wv * 8u;
          src = V + (size_t)(R0 + lane - 16) * q + cv0;
          dst = sl + (MB + lane - 16) * 64;
        }
      }
      const uint32_t tot = __reduce_add_sync(0xffffffffu, bytes);
      const uint32_t mb = bar_of(t);
      if (lane == 0)
        asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(mb),
                     "r"(tot)
                     : "memory");
      __syncwarp();
      if (bytes)
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                smem_addr(dst)),
            "l"(src), "r"(bytes), "r"(mb)
            : "memory");
    };
    const bool lu = 2 * lane < wu, lv = 2 * lane < wv;
    float mu0 = 0.f, mu1 = 0.f, mv0 = 0.f, mv1 = 0.f;  // columns 2 lane, 2 lane + 1 of U and V
    bool dead = false;
    int issued_t = 0, done_t = 0;
    for (; issued_t < MSW - 1 && issued_t < total; ++issued_t) issue(issued_t);
    for (int j = 0; j <= nmy; ++j) {
      if (j < nmy) {
        for (int t = j * (NMB / 2); t < (j + 1) * (NMB / 2); ++t) {
          if (dead) break;
          if (issued_t < total) issue(issued_t++);
          if (!tc_wait(bar_of(t), (uint32_t)((t / MSW) & 1), wait_limit)) {
            dead = true;
            if (lane == 0) {
              atomicAdd(&g_oz_tc_timeouts, 1);
              flags[1] = 1;
            }
            break;
          }
          done_t = t + 1;
          int64_t R0;
          batch_rows(t, R0);
          const int64_t left = n - R0;  // cells i % MB below it are live
          const float2* sl = slot_of(t) + 2 * lane;
          if (left >= MB && lu && (SYM || lv)) {
            float4 v[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              const bool isvc = !SYM && i >= MB;
              v[i] = *reinterpret_cast<const float4*>(sl + (isvc ? MB * 64 + (i - MB) * strV : i * strU));
            }
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              if (!SYM && i >= MB) {
                mv0 = fmaxf(mv0, fabsf(v[i].x));
                mv1 = fmaxf(mv1, fabsf(v[i].z));
              } else {
                mu0 = fmaxf(mu0, fabsf(v[i].x));
                mu1 = fmaxf(mu1, fabsf(v[i].z));
              }
            }
          } else {
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              const bool isvc = !SYM && i >= MB;
              const int li = isvc ? i - MB : i;
              if (li < left && (isvc ? lv : lu)) {
                const float4 v =
                    *reinterpret_cast<const float4*>(sl + (isvc ? MB * 64 + li * strV : li * strU));
                if (isvc) {
                  mv0 = fmaxf(mv0, fabsf(v.x));
                  mv1 = fmaxf(mv1, fabsf(v.z));
                } else {
                  mu0 = fmaxf(mu0, fabsf(v.x));
                  mu1 = fmaxf(mu1, fabsf(v.z));
                }
              }
            }
          }
          // the slot's generic reads before the next bulk copy into it
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          __syncwarp();
        }
        // chunk j's exponents and scales (parity slot j & 1; the workers
        // finished chunk j - 2, its last user, before the last barrier):
        // warp 1's maxima through the scratch, then warp 0 publishes
        const int es = j & 1;
        if (mw == 1) {
          mscr[2 * lane] = mu0;
          mscr[2 * lane + 1] = mu1;
          mscr[64 + 2 * lane] = mv0;
          mscr[64 + 2 * lane + 1] = mv1;
        }
        dead = bar2_or(dead);
        if (mw == 0) {
          mu0 = fmaxf(mu0, mscr[2 * lane]);
          mu1 = fmaxf(mu1, mscr[2 * lane + 1]);
          const int e0 = exponent_above(mu0), e1 = exponent_above(mu1);
          Ex[es * 128 + 2 * lane] = e0;
          Ex[es * 128 + 2 * lane + 1] = e1;
          Fx[es * 128 + 2 * lane] = exp2i(e0 - 7);
          Fx[es * 128 + 2 * lane + 1] = exp2i(e1 - 7);
          if (!SYM) {
            mv0 = fmaxf(mv0, mscr[64 + 2 * lane]);
            mv1 = fmaxf(mv1, mscr[64 + 2 * lane + 1]);
            const int f0 = exponent_above(mv0), f1 = exponent_above(mv1);
            Ex[es * 128 + 64 + 2 * lane] = f0;
            Ex[es * 128 + 64 + 2 * lane + 1] = f1;
            Fx[es * 128 + 64 + 2 * lane] = exp2i(f0 - 7);
            Fx[es * 128 + 64 + 2 * lane + 1] = exp2i(f1 - 7);
          }
        }
        mu0 = mu1 = mv0 = mv1 = 0.f;
        // warp 0 has read the scratch before warp 1 writes the next chunk's
        bar2_or(false);
      }
      // j == 0: before the workers' first chunk; j >= 1: at the end of their
      // chunk j - 1; j == nmy: at the end of their last chunk
      __syncthreads();
      if (flags[0]) dead = true;
    }
    // copies still in flight (a timeout, or the workers' failure, stopped
    // the reads): wait for each with the full bound before the block exits
    for (int t = done_t; t < issued_t; ++t) tc_wait(bar_of(t), (uint32_t)((t / MSW) & 1), TC_WAIT_LIMIT);
  } else {
    // ---- workers (staging, cut, combination) and the issuing warp ----
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(64 >> 3) << 17) |
                           ((uint32_t)(128 >> 4) << 24);
    const uint32_t dbase = smem_addr(dig);
    // staging: worker -> raw rows r = tid / 32 and r + 16 of a slot, columns
    // c, c + 1 (c = 2 (tid % 32)), one 16-byte copy each; raw row r + 16 is
    // U's row r + 16 (U == V) or V's row r (U != V)
    const int sr = tid >> 5, sc = 2 * (tid & 31);
    const bool sokA = sc < wu, sokB = sc < (SYM ? wu : wv);
    const int ldA = p, ldB = SYM ? p : q;
    const float2* sA = U + cu0 + sc + (int64_t)sr * ldA;
    const float2* sB = SYM ? U + cu0 + sc + (int64_t)(sr + 16) * ldA : V + cv0 + sc + (int64_t)sr * ldB;
    const int64_t rA0 = sr, rB0 = SYM ? sr + 16 : sr;
    auto stage_sub = [&](int g) {
      if (g < G) {
        const int64_t r0 = (int64_t)((int)blockIdx.x + (g / NSUB) * (int)gridDim.x) * EC + (g % NSUB) * SK;
        float2* slot = raw + (size_t)(g % NR) * (32 * TG_RS) + sr * TG_RS + sc;
        const bool okA = sokA && r0 + rA0 < n, okB = sokB && r0 + rB0 < n;
        cp_async16(slot, okA ? sA + r0 * ldA : U, okA);
        cp_async16(slot + 16 * TG_RS, okB ? sB + r0 * ldB : U, okB);
      }
      cp_async_commit();
    };
    // combine: worker warp w reads TMEM lanes 32 (w % 4) .. + 31, i.e. output
    // row a = 32 (w % 2) + lane of the top (w % 4 < 2) or bottom half, columns
    // 16 (w / 4) .. + 15
    const int quarter = warp & 3, arow = 32 * (quarter & 1) + lane, cb = 16 * ((warp >> 2) & 3);
    const bool top = quarter < 2;
    float2 res[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) res[e] = make_float2(0.f, 0.f);
    // digit item of this worker (one per sub-chunk): column c, rows
    // 4 qd .. 4 qd + 3 of the sub-chunk, of U or (isv) of V
    const bool isv = !SYM && tid >= 256;
    const int loc = SYM ? tid : (tid & 255);
    const int ic = 8 * ((loc >> 5) & 7) + (lane & 7);
    const int iq = 2 * (((lane >> 4) & 1) + 2 * (loc >> 8)) + ((lane >> 3) & 1);
    const int irow = (isv ? SK : 0) + 4 * iq;
    const uint32_t doff = (isv ? NDT * plane : 0) + tc_off(ic, 4 * iq, SK);
    bool failed = false;
    int issued = 0;  // sub-chunks whose products were issued (the same in every thread)
    if (worker) {
      for (int g = 0; g < NR - 1; ++g) stage_sub(g);
      cp_async_wait_group<NR - 2>();
    }
    __syncthreads();  // the maxima warps have written chunk 0's exponents
    float scut = worker ? exp2i(7 - Ex[(isv ? 64 : 0) + ic]) : 0.f;
    for (int g = 0; g < G; ++g) {
      const int k = g / NSUB;
      const int s = g - k * NSUB;
      const int buf = g % NB;
      const int es = k & 1;
      if (!failed) {
        bool ok = true;
        if (worker) {
          // this buffer's previous products (sub-chunk g - NB) are done
          if (g >= NB) ok = tc_wait(mbase + 8u * buf, (uint32_t)((g / NB - 1) & 1), wait_limit);
          if (ok) {
            const float2* slot = raw + (size_t)(g % NR) * (32 * TG_RS) + irow * TG_RS + ic;
            unsigned char* dst = dig + buf * DBUF + doff;
            float d[4][NDT];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
              const float2 x = slot[t * TG_RS];
              digits_scaled<NDT>(x.x, x.y, scut, d[t]);
            }
#pragma unroll
            for (int i = 0; i < NDT; ++i)
              *reinterpret_cast<uint2*>(dst + i * plane) =
                  make_uint2(pack_bf16x2(d[0][i], d[1][i]), pack_bf16x2(d[2][i], d[3][i]));
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          }
          // raw rows NR - 1 sub-chunks ahead, into the slot cut one sub-chunk
          // ago (free since the last barrier); then this thread's copies of
          // sub-chunk g + 1 are complete, and the barrier publishes them
          stage_sub(g + NR - 1);
          cp_async_wait_group<NR - 2>();
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        if (bar1_or(!ok)) {
          failed = true;
        } else {
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          if (issuer) {
            if (lane == 0) {
              const uint32_t ab = dbase + buf * DBUF, bb = SYM ? ab : ab + NDT * plane;
              const uint64_t da = tc_desc(ab, SK), db = tc_desc(bb, SK);
              const uint32_t acc0 = s > 0 ? 1u : 0u;
              const uint32_t idesc0 = idesc & ~(0x3Fu << 17);
#pragma unroll
              for (int m = 0; m < 4; ++m)
#pragma unroll
                for (int j0 = 0; j0 < NDT - 2 * m; j0 += 4) {
                  const int run = (NDT - 2 * m - j0) < 4 ? (NDT - 2 * m - j0) : 4;
                  const uint32_t idn = idesc0 | ((uint32_t)((64 * run) >> 3) << 17);
#pragma unroll
                  for (int ks = 0; ks < SK / 16; ++ks)
                    tc_mma(tmem + (uint32_t)((2 * m + j0) * 64), da + ((2 * m * plane + ks * 256) >> 4),
                           db + ((j0 * plane + ks * 256) >> 4), idn, (m > 0 || ks > 0) ? 1u : acc0);
                }
              asm volatile(
                  "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbase +
                                                                                                  8u * buf)
                  : "memory");
            }
            __syncwarp();
          }
          issued = g + 1;
        }
      }
      if (s < NSUB - 1) continue;
      // chunk end: its last products (a commit covers every earlier product
      // of the issuing thread), then the combination
      if (!failed) {
        bool ok2 = true;
        if (worker) ok2 = tc_wait(mbase + 8u * buf, (uint32_t)((g / NB) & 1), wait_limit);
        if (bar1_or(!ok2)) {
          failed = true;
        } else if (worker) {
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const float fu = Fx[es * 128 + arow];
          const float* Fv = Fx + es * 128 + (SYM ? 0 : 64) + cb;
          const uint32_t lanes = tmem + ((uint32_t)(32 * quarter) << 16);
#pragma unroll
          for (int c0 = 0; c0 < 16; c0 += 4) {
            uint32_t v[NDT][4];
#pragma unroll
            for (int h = 0; h < NDT; ++h)
              if (top || h < NDT - 1) tc_ld4(v[h], lanes + (uint32_t)(h * 64 + cb + c0));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              float S[NDT];
#pragma unroll
              for (int h = 0; h < NDT; ++h) S[h] = __uint_as_float(v[h][e]);
              // top: groups 0..6 (even digits of U); bottom: groups 1..6
              // (odd digits), block h holding group h + 1
              const float2 w = top ? combine_groups_fast<NDT, (NDT > 4 ? 4 : NDT - 1)>(S)
                                   : combine_groups_fast<NDT - 1, (NDT > 4 ? 3 : NDT - 2)>(S);
              const float fv = Fv[c0 + e];
              res[c0 + e] = df_add(res[c0 + e], make_float2(w.x * fu * fv, w.y * fu * fv));
            }
          }
        }
      }
      if (failed && tid == 0) flags[0] = 1;
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      // with the maxima warp: the next chunk's exponents are in parity slot
      // es ^ 1, and this chunk's TMEM reads are done before its products
      __syncthreads();
      if (flags[1]) failed = true;
      if (worker) scut = exp2i(7 - Ex[(es ^ 1) * 128 + (isv ? 64 : 0) + ic]);
    }
    if (worker) cp_async_wait_all();
    if (failed) {
      // a product or a maxima copy that did not complete in time: drain the
      // tensor core (bounded) and report non-finite partial sums. Each
      // buffer's barrier has at most one pending commit (its last issued
      // sub-chunk); the final commit covers anything else issued.
      if (tid == 0 && !flags[1]) atomicAdd(&g_oz_tc_timeouts, 1);
      for (int b = 0; b < NB; ++b) {
        const int last = issued - 1 - ((issued - 1 - b) % NB + NB) % NB;  // last g' < issued, g' % NB == b
        if (last >= 0) tc_wait(mbase + 8u * b, (uint32_t)((last / NB) & 1), TC_WAIT_LIMIT);
      }
      tc_drain(issuer && lane == 0, mbase + 8u * NB);
#pragma unroll
      for (int e = 0; e < 16; ++e) res[e] = make_float2(NAN, NAN);
    }
    // (the final stage below reuses the raw ring)
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS));
    float2* st = raw;  // 64 x 65 float2: odd-digit parts (bottom half) onto the even-digit parts
    if (worker && !top) {
#pragma unroll
      for (int e = 0; e < 16; ++e) st[arow * 65 + cb + e] = res[e];
    }
    __syncthreads();
    if (worker && top) {
      float2* out = part + ((size_t)blockIdx.x * gridDim.y + blockIdx.y) * 4096;
#pragma unroll
      for (int e = 0; e < 16; ++e) out[arow * 64 + cb + e] = df_add(res[e], st[arow * 65 + cb + e]);
    }
    return;
  }
  // the maxima warps: the two barriers of the block's end
  __syncthreads();
  __syncthreads();
}

// Fixed-order sum of the per-block partials into G (float64, p x q); the
// symmetric case fills the lower triangle from the upper one.
__global__ void oz_gram_reduce_kernel(int p, int q, int nsplit, int nblk, int sym, int nbj,
                                      const float2* part, double* G) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= p * q) return;
  int i = e / q, j = e - i * q;
  int si = i, sj = j;
  if (sym && i > j) {
    si = j;
    sj = i;
  }
  int bi = si / 64, bj = sj / 64;
  int b;
  if (sym) {
    b = 0;
    for (int r = 0; r < bi; ++r) b += nbj - r;
    b += bj - bi;
  } else {
    b = bi * nbj + bj;
  }
  int ii = si - bi * 64, jj = sj - bj * 64;
  if (sym && bi == bj && (ii / 16) > (jj / 16)) {  // lower warp tile inside a diagonal block
    int t = ii;
    ii = jj;
    jj = t;
  }
  float2 s = make_float2(0.f, 0.f);
  // unrolled so that several partials are in flight at once (same order)
#pragma unroll 8
  for (int k = 0; k < nsplit; ++k) s = df_add(s, part[((size_t)k * nblk + b) * 4096 + ii * 64 + jj]);
  G[e] = df_to_double(s);
}

// The same for a symmetric Gram whose upper-triangle blocks (bi <= bj, row by
// row) were computed in full by the tcgen05 kernel: entry (i, j) is read
// from the upper triangle, so G is exactly symmetric.
__global__ void oz_gram_reduce_tri_kernel(int p, int nsplit, int nblk, int nbj, const float2* part, double* G) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= p * p) return;
  const int i = e / p, j = e - i * p;
  const int si = min(i, j), sj = max(i, j);
  const int bi = si / 64, bj = sj / 64;
  int b = 0;
  for (int r = 0; r < bi; ++r) b += nbj - r;
  b += bj - bi;
  const int ii = si - bi * 64, jj = sj - bj * 64;
  float2 s = make_float2(0.f, 0.f);
#pragma unroll 8
  for (int k = 0; k < nsplit; ++k) s = df_add(s, part[((size_t)k * nblk + b) * 4096 + ii * 64 + jj]);
  G[e] = df_to_double(s);
}

// ---------------------------------------------------------------------------
// host wrappers
// ---------------------------------------------------------------------------
int pad16(int x) { return (x + 15) / 16 * 16; }

size_t oz_rhs_bytes(int p, int nk) {
  (void)nk;
  return (size_t)ND * pad16(p) * pad16(p) * sizeof(__nv_bfloat16) + pad16(p) * sizeof(int) + 256;
}

gsi_status oz_gemm(int64_t n, int p, int nk, const float2* const U[2], const double* const M[2],
                   const double s[2], int ne, const float2* const E[2], const float2 ce[2],
                   float2* out, float2* dot_part, const float2* dot_with, bool dot_self,
                   void* rhs_ws, cudaStream_t st, int* nparts, int nd, float* rinf_part,
                   bool* rinf_done) {
  if (rinf_done) *rinf_done = false;
  if (nk < 1 || nk > 2 || ne < 0 || ne > 2 || p < 1 || p > 128 || (nd != 3 && nd != ND))
    return GSI_ERR_ARG;
  bool fuse = nk == 2 && M[1] == M[0] && s[0] != 0.0;
  if (fuse && oz_gemm_smem(pad16(p), std::min(64, pad16(p)), 2, nd) > 227 * 1024) fuse = false;
  if (nk == 2 && !fuse) {
    // OUT = s0 U0 M0 + E terms, then OUT += s1 U1 M1
    const float2* U0[2] = {U[0], U[0]};
    const double* M0[2] = {M[0], M[0]};
    double s0[2] = {s[0], 0.0};
    GSI_TRY(oz_gemm(n, p, 1, U0, M0, s0, ne, E, ce, out, nullptr, nullptr, false, rhs_ws, st,
                    nullptr, nd));
    const float2* U1[2] = {U[1], U[1]};
    const double* M1[2] = {M[1], M[1]};
    double s1[2] = {s[1], 0.0};
    const float2* E1[2] = {out, out};
    float2 c1[2] = {make_float2(1.f, 0.f), make_float2(0.f, 0.f)};
    return oz_gemm(n, p, 1, U1, M1, s1, 1, E1, c1, out, dot_part, dot_with, dot_self, rhs_ws, st,
                   nparts, nd, rinf_part, rinf_done);
  }
  const int p16 = pad16(p), K16 = p16;
  const int ncs = (p16 + 63) / 64;
  if (ncs > 1)
    for (int k = 0; k < nk; ++k)
      if (U[k] == out) return GSI_ERR_ARG;  // column slices would race on in-place rows
  __nv_bfloat16* Md = reinterpret_cast<__nv_bfloat16*>(rhs_ws);
  int* F = reinterpret_cast<int*>(reinterpret_cast<char*>(rhs_ws) +
                                  (size_t)ND * p16 * K16 * sizeof(__nv_bfloat16));
  OzGemmArgs a{};
  a.U[0] = U[0];
  a.U[1] = fuse ? U[1] : U[0];
  a.fuse_u1 = fuse ? 1 : 0;
  a.a1 = fuse ? df_from_double(s[1] / s[0]) : make_float2(0.f, 0.f);
  a.ne = ne;
  for (int m = 0; m < ne; ++m) {
    a.E[m] = E[m];
    a.ce[m] = ce[m];
  }
  a.Md = Md;
  a.F = F;
  a.out = out;
  a.dot_part = dot_part;
  a.dot_with = dot_with;
  a.dot_self = dot_self ? 1 : 0;
  a.ldu = p;
  a.kofs = 0;
  a.kw = p;
  {
    const void* ptrs[6] = {a.U[0], a.U[1], ne > 0 ? E[0] : nullptr, ne > 1 ? E[1] : nullptr, dot_with, out};
    a.vec16 = 1;
    for (const void* q : ptrs)
      if (((uintptr_t)q & 15) != 0) a.vec16 = 0;
  }
  const int NCmax = std::min(64, p16);
  if (nd == ND && tensor_path() != 1) {
    // The tcgen05 kernel holds a 128-row tile of the left operand's digits for
    // a contraction of at most 64: a longer one (p > 64) is cut into nks
    // slices of equal width kc, one launch each. Every slice is an exact
    // digit product with its own row and column powers of two; the slices
    // are summed in df64 through the output (E_0 = OUT, c_0 = 1 from the
    // second slice on), the caller's elementwise terms go with the first
    // slice and the dot partials are taken on the last, which writes OUT.
    const int nks = (p16 + 63) / 64;
    const int kc = std::min(p, pad16((p + nks - 1) / nks));
    int gx = (int)std::min<int64_t>((n + TC_M - 1) / TC_M, (int64_t)sm_count());
    gx = std::max(gx, 1);
    if (nparts) *nparts = gx * ncs;
    // the row sums are formed where one warp holds whole rows (the kernel's
    // row-wise epilogue: one column block, even p, aligned blocks)
    const bool rows = rinf_part && a.vec16 && ncs == 1 && (p & 1) == 0;
    if (rinf_done) *rinf_done = rows;
    for (int h = 0; h < nks; ++h) {
      const int k0 = h * kc, kw = std::min(kc, p - k0);
      const int K16h = pad16(kw);
      oz_prep_rhs_kernel<<<p16, 128, 0, st>>>(p, p16, 1, K16h, M[0], M[0], s[0], 0.0, Md, F, k0, kw);
      GSI_LAUNCH_CHECK();
      OzGemmArgs b = a;
      b.kofs = k0;
      b.kw = kw;
      if (h > 0) {
        b.ne = 1;
        b.E[0] = out;
        b.ce[0] = make_float2(1.f, 0.f);
      }
      const bool last = h == nks - 1;
      if (!last) {
        b.dot_part = nullptr;
        b.dot_with = nullptr;
        b.dot_self = 0;
      }
      b.rinf_part = last && rows ? rinf_part : nullptr;
      const size_t tsm = oz_gemm_tc_smem(K16h, NCmax);
      auto kern = b.fuse_u1 ? oz_gemm_tc_kernel<true> : oz_gemm_tc_kernel<false>;
      GSI_CUDA_TRY(ensure_dyn_smem((const void*)kern, (int)tsm));
      kern<<<dim3(gx, ncs), TC_THREADS, tsm, st>>>(n, p, p16, K16h, b);
      GSI_LAUNCH_CHECK();
    }
    return GSI_OK;
  }
  oz_prep_rhs_kernel<<<p16, 128, 0, st>>>(p, p16, 1, K16, M[0], M[0], s[0], 0.0, Md, F, 0, p);
  GSI_LAUNCH_CHECK();
  size_t smem = oz_gemm_smem(K16, NCmax, fuse ? 2 : 1, nd);
  auto kern = nd == 3 ? oz_gemm_kernel<3> : oz_gemm_kernel<ND>;
  GSI_CUDA_TRY(ensure_dyn_smem((const void*)kern, (int)smem));
  int64_t ntiles = (n + GM_RT - 1) / GM_RT;
  int per_sm = 1;
  GSI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, GM_THREADS, smem));
  per_sm = std::max(per_sm, 1);
  int gx = (int)std::min<int64_t>(ntiles, (int64_t)sm_count() * per_sm / ncs);
  gx = std::max(gx, 1);
  if (nparts) *nparts = gx * ncs;
  kern<<<dim3(gx, ncs), GM_THREADS, smem, st>>>(n, p, p16, K16, a);
  GSI_LAUNCH_CHECK();
  return GSI_OK;
}

gsi_status oz_set_wait_limit(int limit) {
  const int v = (limit < 0 || limit > TC_WAIT_LIMIT) ? TC_WAIT_LIMIT : limit;
  GSI_CUDA_TRY(cudaMemcpyToSymbol(g_oz_wait_limit, &v, sizeof(int)));
  return GSI_OK;
}

gsi_status oz_timeouts_async(int* host_dst, cudaStream_t st) {
  GSI_CUDA_TRY(cudaMemcpyFromSymbolAsync(host_dst, g_oz_tc_timeouts, sizeof(int), 0, cudaMemcpyDeviceToHost, st));
  return GSI_OK;
}

int oz_gemm_max_parts(int p) {
  int ncs = (pad16(p) + 63) / 64;
  return sm_count() * 8 * ncs;  // up to 8 resident blocks per SM for small digit counts
}

int oz_gram_blocks(int p, int q, bool sym) {
  int nbi = (p + 63) / 64, nbj = (q + 63) / 64;
  return sym ? nbi * (nbi + 1) / 2 : nbi * nbj;
}

int oz_gram_splits(int64_t n, int p, int q, bool sym) {
  int nb = oz_gram_blocks(p, q, sym);
  int64_t chunks = (n + GR_KC - 1) / GR_KC;
  int s = std::max(1, sm_count() / nb);
  return (int)std::max<int64_t>(1, std::min<int64_t>(s, chunks));
}

size_t oz_gram_scratch_bytes(int64_t n, int p, int q, bool sym) {
  return (size_t)oz_gram_splits(n, p, q, sym) * oz_gram_blocks(p, q, sym) * 4096 * sizeof(float2);
}

__global__ void oz_gram_reduce_df_kernel(int p, int q, int nsplit, int nbj, const float2* part,
                                         float2* G) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)p * q) return;
  int i = (int)(e / q), j = (int)(e - (int64_t)i * q);
  int bi = i / 64, bj = j / 64;
  int b = bi * nbj + bj;
  int nblk = ((p + 63) / 64) * nbj;
  int ii = i - bi * 64, jj = j - bj * 64;
  float2 s = make_float2(0.f, 0.f);
#pragma unroll 8
  for (int k = 0; k < nsplit; ++k) s = df_add(s, part[((size_t)k * nblk + b) * 4096 + ii * 64 + jj]);
  G[e] = s;
}

gsi_status oz_gram(int64_t n, int p, int q, const float2* U, const float2* V, bool sym, double* G,
                   float2* scratch, cudaStream_t st, int nd, float2* Gdf, int reserve_sms) {
  if (p < 1 || q < 1 || q > 128 || (sym && (p != q || Gdf)) || (nd != 3 && nd != ND) ||
      (!G && !Gdf) || (p > 128 && !Gdf))
    return GSI_ERR_ARG;
  const int nbj = (q + 63) / 64;
  const int nblk = oz_gram_blocks(p, q, sym);
  int ns = oz_gram_splits(n, p, q, sym);
  if (reserve_sms > 0) ns = std::max(1, std::min(ns, (sm_count() - reserve_sms) / nblk));
  const int tp = tensor_path();
  // 16-byte copies need even row lengths and 16-byte aligned bases
  const bool vec16 = ((p | q) & 1) == 0 && ((uintptr_t)U & 15) == 0 && ((uintptr_t)V & 15) == 0;
  bool tri = false;  // symmetric Gram from full upper-triangle blocks
  // 16-byte aligned blocks of even width: the kernel with the maxima warps
  // (it counts its sub-chunks in 32 bits: n < 2^34). Its maxima warps copy
  // a batch's rows in one piece where the block spans whole rows (p, q <=
  // 64); 64-column blocks of wider matrices take one copy per row, where the
  // whole-chunk kernel is as fast for 7 digits, so those stay with it.
  const bool ring = tp != 1 && vec16 && n < ((int64_t)1 << 34) && ((p <= 64 && q <= 64) || nd == 3);
  if (ring) {
    const bool one = p <= 64 && q <= 64;
    tri = sym && !one;
    const bool ksym = sym && one;
    const size_t tsm = oz_gram_tc_ring_smem(ksym, nd);
    auto kern = nd == 3 ? (ksym ? oz_gram_tc_ring_kernel<true, 3> : oz_gram_tc_ring_kernel<false, 3>)
                        : (ksym ? oz_gram_tc_ring_kernel<true, ND> : oz_gram_tc_ring_kernel<false, ND>);
    GSI_CUDA_TRY(ensure_dyn_smem((const void*)kern, (int)tsm));
    kern<<<dim3(ns, one ? 1 : nblk), TR_THREADS, tsm, st>>>(n, p, q, U, V, scratch, one ? 1 : nbj,
                                                            tri ? 1 : 0);
    GSI_LAUNCH_CHECK();
  } else if (nd == ND && p <= 64 && q <= 64 && tp != 1) {
    // one 64 x 64 output block; every partial entry is written
    const size_t tsm = oz_gram_tc_smem(sym);
    auto kern = sym ? oz_gram_tc_kernel<true> : oz_gram_tc_kernel<false>;
    GSI_CUDA_TRY(ensure_dyn_smem((const void*)kern, (int)tsm));
    kern<<<ns, TG_THREADS, tsm, st>>>(n, p, q, U, V, vec16 ? 1 : 0, scratch, 1, 0);
    GSI_LAUNCH_CHECK();
  } else if (nd == ND && tp != 1) {
    // several 64 x 64 output blocks (p or q > 64), one per blockIdx.y, each
    // by the U != V kernel; a symmetric Gram computes the upper-triangle
    // blocks only and is mirrored by the reduction
    tri = sym;
    const size_t tsm = oz_gram_tc_smem(false);
    GSI_CUDA_TRY(ensure_dyn_smem((const void*)oz_gram_tc_kernel<false>, (int)tsm));
    oz_gram_tc_kernel<false><<<dim3(ns, nblk), TG_THREADS, tsm, st>>>(n, p, q, U, V, vec16 ? 1 : 0, scratch, nbj,
                                                                     tri ? 1 : 0);
    GSI_LAUNCH_CHECK();
  } else {
    size_t smem = oz_gram_smem(nd);
    auto kern = nd == 3 ? oz_gram_kernel<3> : oz_gram_kernel<ND>;
    GSI_CUDA_TRY(ensure_dyn_smem((const void*)kern, (int)smem));
    GSI_CUDA_TRY(cudaMemsetAsync(scratch, 0, (size_t)ns * nblk * 4096 * sizeof(float2), st));
    kern<<<dim3(ns, nblk), GR_THREADS, smem, st>>>(n, p, q, U, V, sym ? 1 : 0, nbj, scratch);
    GSI_LAUNCH_CHECK();
  }
  if (Gdf) {
    oz_gram_reduce_df_kernel<<<ceil_div((int64_t)p * q, 256), 256, 0, st>>>(p, q, ns, nbj, scratch, Gdf);
  } else if (tri) {
    oz_gram_reduce_tri_kernel<<<ceil_div(p * q, 256), 256, 0, st>>>(p, ns, nblk, nbj, scratch, G);
  } else {
    oz_gram_reduce_kernel<<<ceil_div(p * q, 256), 256, 0, st>>>(p, q, ns, nblk, sym ? 1 : 0, nbj,
                                                                scratch, G);
  }
  GSI_LAUNCH_CHECK();
  return GSI_OK;
}

}  // namespace gsi
