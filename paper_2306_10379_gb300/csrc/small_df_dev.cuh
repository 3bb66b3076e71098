// Device code of the p x p step without the float64 pipe (see small_df.cu):
// float32 Jacobi refined to df64, the line search, and the polar normaliser
// by the first-order expansion in the eigenbasis. Every function runs in
// the whole calling thread block with blockDim-strided loops.
#pragma once
#include <math.h>

#include "alg3.cuh"
#include "blas_f64.cuh"
#include "df.cuh"

namespace gsi {

struct SdWs {
  float *Af, *Vf;                    // p x p float32
  float2 *Bd, *Vd, *Td, *Ud;         // p x p df64
  double *al, *be, *ga, *ze, *sv;    // p
  float *rc, *rs;                    // rotations (float32 stage)
  double *dc, *ds;                   // rotations (df64 stage)
  float2 *fc, *fs;                   // the df64 rotations as df64 numbers
  int *ri, *rj;
};

__host__ __device__ inline size_t sd_bytes(int p) {
  size_t q = (size_t)p * p;
  return 2 * q * sizeof(float) + 4 * q * sizeof(float2) + 5 * (size_t)p * sizeof(double) +
         64 * (2 * sizeof(float) + 2 * sizeof(double) + 2 * sizeof(float2) + 2 * sizeof(int)) + 512;
}

// Layout: df64 matrices first, then the float32 Jacobi matrices and vectors.
// With `split`, the df64 part lives in global memory (base) and the rest in
// shared memory (sbase).
static __device__ SdWs sd_carve(unsigned char* base, int p, unsigned char* sbase = nullptr) {
  size_t q = (size_t)p * p;
  SdWs w;
  unsigned char* cur = base;
  auto take = [&](size_t bytes) {
    unsigned char* r = cur;
    cur += (bytes + 15) & ~(size_t)15;
    return r;
  };
  w.Bd = (float2*)take(q * sizeof(float2));
  w.Vd = (float2*)take(q * sizeof(float2));
  w.Td = (float2*)take(q * sizeof(float2));
  w.Ud = (float2*)take(q * sizeof(float2));
  if (sbase) cur = sbase;
  w.Af = (float*)take(q * sizeof(float));
  w.Vf = (float*)take(q * sizeof(float));
  w.al = (double*)take(p * sizeof(double));
  w.be = (double*)take(p * sizeof(double));
  w.ga = (double*)take(p * sizeof(double));
  w.ze = (double*)take(p * sizeof(double));
  w.sv = (double*)take(p * sizeof(double));
  w.dc = (double*)take(64 * sizeof(double));
  w.ds = (double*)take(64 * sizeof(double));
  w.fc = (float2*)take(64 * sizeof(float2));
  w.fs = (float2*)take(64 * sizeof(float2));
  w.rc = (float*)take(64 * sizeof(float));
  w.rs = (float*)take(64 * sizeof(float));
  w.ri = (int*)take(64 * sizeof(int));
  w.rj = (int*)take(64 * sizeof(int));
  return w;
}

// Round-robin ordering: in round r (0 <= r < m - 1) slot 0 pairs r with the
// fixed index m - 1 and slot k pairs (r + k) and (r - k) modulo m - 1; both
// sums lie in [0, 2 (m - 1)), so one conditional subtraction reduces them.
static __device__ __forceinline__ void pair_of(int r, int k, int m, int p, int& i, int& j) {
  int a, b;
  if (k == 0) {
    a = r;
    b = m - 1;
  } else {
    a = r + k;
    if (a >= m - 1) a -= m - 1;
    b = r + (m - 1) - k;
    if (b >= m - 1) b -= m - 1;
  }
  i = min(a, b);
  j = max(a, b);
  if (j >= p) j = -1;  // paired with the dummy index of an odd p: identity on i
}

// The warps' partial sums are added in warp order by one thread and the
// total broadcast: one float64 add per warp instead of one per thread and
// warp on the slow float64 pipe.
static __device__ double block_sum(double v, double* red) {
  __shared__ double total;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    total = s;
  }
  __syncthreads();
  return total;
}

// float32 Jacobi on Af (p x p), rotations accumulated into Vf.
static __device__ int jacobi_f32(int p, float* A, float* V, SdWs& w, double* red, int max_sweeps,
                          double rel_tol) {
  const int m = (p + 1) & ~1, half = m / 2;
  // rotation tables held in registers for the whole call
  float* const rc = w.rc;
  float* const rs = w.rs;
  int* const ri = w.ri;
  int* const rj = w.rj;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
      double a = A[e];
      tot += a * a;
      if (e / p != e % p) off += a * a;
    }
    off = block_sum(off, red);
    tot = block_sum(tot, red);
    if (!(off > rel_tol * rel_tol * tot)) break;  // float32 stage
    for (int r = 0; r < m - 1; ++r) {
      for (int k = threadIdx.x; k < half; k += blockDim.x) {
        int i, j;
        pair_of(r, k, m, p, i, j);
        float c = 1.f, s = 0.f;
        if (j >= 0) {
          float aij = A[i * p + j];
          if (aij != 0.f) {
            float th = (A[j * p + j] - A[i * p + i]) / (2.f * aij);
            float t = (fabsf(th) > 1e18f) ? 0.5f / th
                                           : copysignf(1.f, th) / (fabsf(th) + sqrtf(th * th + 1.f));
            c = rsqrtf(t * t + 1.f);
            s = t * c;
          }
        }
        rc[k] = c;
        rs[k] = s;
        ri[k] = i;
        rj[k] = j;
      }
      __syncthreads();
      // 2 x 2 block (k, l) of J^T A J
      auto upd_a = [&](int k, int l) {
        int ik = ri[k], jk = rj[k], il = ri[l], jl = rj[l];
        float ck = rc[k], sk = rs[k], cl = rc[l], sl = rs[l];
        float x00 = A[ik * p + il];
        float x01 = jl >= 0 ? A[ik * p + jl] : 0.f;
        float x10 = jk >= 0 ? A[jk * p + il] : 0.f;
        float x11 = (jk >= 0 && jl >= 0) ? A[jk * p + jl] : 0.f;
        // right: columns (il, jl) by J_l
        float y00 = cl * x00 - sl * x01, y01 = sl * x00 + cl * x01;
        float y10 = cl * x10 - sl * x11, y11 = sl * x10 + cl * x11;
        // left: rows (ik, jk) by J_k^T
        float z00 = ck * y00 - sk * y10, z10 = sk * y00 + ck * y10;
        float z01 = ck * y01 - sk * y11, z11 = sk * y01 + ck * y11;
        if (k == l) z01 = z10 = 0.f;
        A[ik * p + il] = z00;
        if (jl >= 0) A[ik * p + jl] = z01;
        if (jk >= 0) A[jk * p + il] = z10;
        if (jk >= 0 && jl >= 0) A[jk * p + jl] = z11;
      };
      // columns (il, jl) of row `row` of V by J_l. Lanes run over rotations
      // (columns), not rows: rows are p apart in shared memory and would all
      // fall in one bank
      auto upd_v = [&](int row, int l) {
        int il = ri[l], jl = rj[l];
        if (jl < 0) return;
        float cl = rc[l], sl = rs[l];
        float vi = V[row * p + il], vj = V[row * p + jl];
        V[row * p + il] = cl * vi - sl * vj;
        V[row * p + jl] = sl * vi + cl * vj;
      };
      if (half <= 32) {  // rotation l <-> lane: no index division
        const int nw = blockDim.x >> 5, wp = threadIdx.x >> 5, ln = threadIdx.x & 31;
        if (ln < half) {
          for (int k = wp; k < half; k += nw) upd_a(k, ln);
          for (int row = wp; row < p; row += nw) upd_v(row, ln);
        }
      } else {
        for (int e = threadIdx.x; e < half * half; e += blockDim.x) {
          int k = e / half;
          upd_a(k, e - k * half);
        }
        for (int e = threadIdx.x; e < half * p; e += blockDim.x) {
          int row = e / half;
          upd_v(row, e - row * half);
        }
      }
      __syncthreads();
    }
  }
  return sweep;
}

static __device__ __forceinline__ float2 df_neg(float2 a) { return make_float2(-a.x, -a.y); }

static __device__ __forceinline__ float2 two_prod_df(float a, float b) {
  float p = __fmul_rn(a, b);
  return make_float2(p, __fmaf_rn(a, b, -p));
}

// 1/sqrt(q) in df64 for q > 0: float32 seed, one Newton step y += y (1 - q y^2) / 2
static __device__ __forceinline__ float2 df_rsqrt(float2 q) {
  float y0 = 1.0f / sqrtf(q.x);
  float2 y = make_float2(y0, 0.f);
  float2 qy2 = df_mul(q, df_mul(y, y));
  float2 e = df_add(make_float2(1.f, 0.f), df_neg(qy2));
  return df_add(y, df_mul(y, make_float2(0.5f * e.x, 0.5f * e.y)));
}

// df64 Jacobi sweeps on the nearly diagonal Bd, rotations (computed in
// float64) accumulated into Vd.
static __device__ int jacobi_df(int p, float2* A, float2* V, SdWs& w, double* red, int max_sweeps) {
  const int m = (p + 1) & ~1, half = m / 2;
  // rotation tables held in registers for the whole call
  float2* const fc = w.fc;
  float2* const fs = w.fs;
  int* const act_k = reinterpret_cast<int*>(w.ds);  // rotation k active (1) or identity (0)
  int* const ri = w.ri;
  int* const rj = w.rj;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
      double a = df_to_double(A[e]);
      tot += a * a;
      if (e / p != e % p) off += a * a;
    }
    off = block_sum(off, red);
    tot = block_sum(tot, red);
    if (!(off > 1e-27 * tot)) break;
    for (int r = 0; r < m - 1; ++r) {
      for (int k = threadIdx.x; k < half; k += blockDim.x) {
        int i, j;
        pair_of(r, k, m, p, i, j);
        // angle from float32 data (a small error in the angle only leaves a
        // tiny off-diagonal entry for the next sweep); c and s then made an
        // exact rotation in df64: c = 1/sqrt(1 + t^2), s = t c
        float2 c = make_float2(1.f, 0.f), s = make_float2(0.f, 0.f);
        bool act = false;
        if (j >= 0) {
          float2 aij = A[i * p + j];
          float2 dif = df_add(A[j * p + j], df_neg(A[i * p + i]));
          float scale = fabsf(A[i * p + i].x) + fabsf(A[j * p + j].x);
          if (aij.x != 0.f && fabsf(aij.x) > 1e-17f * scale) {
            float th = dif.x / (2.f * aij.x);
            float t = (fabsf(th) > 1e18f) ? 0.5f / th
                                           : copysignf(1.f, th) / (fabsf(th) + sqrtf(th * th + 1.f));
            float2 t2 = two_prod_df(t, t);
            float2 q = df_add(make_float2(1.f, 0.f), t2);  // 1 + t^2
            c = df_rsqrt(q);
            s = df_mul(make_float2(t, 0.f), c);
            act = true;
          }
        }
        fc[k] = c;
        fs[k] = s;
        act_k[k] = act ? 1 : 0;
        ri[k] = i;
        rj[k] = j;
      }
      __syncthreads();
      auto upd_a = [&](int k, int l) {
        int ik = ri[k], jk = rj[k], il = ri[l], jl = rj[l];
        if (act_k[k] == 0 && act_k[l] == 0) return;
        float2 ck = fc[k], sk = fs[k];
        float2 cl = fc[l], sl = fs[l];
        const float2 zero = make_float2(0.f, 0.f);
        float2 x00 = A[ik * p + il];
        float2 x01 = jl >= 0 ? A[ik * p + jl] : zero;
        float2 x10 = jk >= 0 ? A[jk * p + il] : zero;
        float2 x11 = (jk >= 0 && jl >= 0) ? A[jk * p + jl] : zero;
        float2 y00 = df_add(df_mul(cl, x00), df_neg(df_mul(sl, x01)));
        float2 y01 = df_add(df_mul(sl, x00), df_mul(cl, x01));
        float2 y10 = df_add(df_mul(cl, x10), df_neg(df_mul(sl, x11)));
        float2 y11 = df_add(df_mul(sl, x10), df_mul(cl, x11));
        float2 z00 = df_add(df_mul(ck, y00), df_neg(df_mul(sk, y10)));
        float2 z10 = df_add(df_mul(sk, y00), df_mul(ck, y10));
        float2 z01 = df_add(df_mul(ck, y01), df_neg(df_mul(sk, y11)));
        float2 z11 = df_add(df_mul(sk, y01), df_mul(ck, y11));
        if (k == l) z01 = z10 = make_float2(0.f, 0.f);
        A[ik * p + il] = z00;
        if (jl >= 0) A[ik * p + jl] = z01;
        if (jk >= 0) A[jk * p + il] = z10;
        if (jk >= 0 && jl >= 0) A[jk * p + jl] = z11;
      };
      auto upd_v = [&](int row, int l) {
        int il = ri[l], jl = rj[l];
        if (jl < 0 || act_k[l] == 0) return;
        float2 cl = fc[l], sl = fs[l];
        float2 vi = V[row * p + il], vj = V[row * p + jl];
        V[row * p + il] = df_add(df_mul(cl, vi), df_neg(df_mul(sl, vj)));
        V[row * p + jl] = df_add(df_mul(sl, vi), df_mul(cl, vj));
      };
      if (half <= 32) {  // rotation l <-> lane: no index division
        const int nw = blockDim.x >> 5, wp = threadIdx.x >> 5, ln = threadIdx.x & 31;
        if (ln < half) {
          for (int k = wp; k < half; k += nw) upd_a(k, ln);
          for (int row = wp; row < p; row += nw) upd_v(row, ln);
        }
      } else {
        for (int e = threadIdx.x; e < half * half; e += blockDim.x) {
          int k = e / half;
          upd_a(k, e - k * half);
        }
        for (int e = threadIdx.x; e < half * p; e += blockDim.x) {
          int row = e / half;
          upd_v(row, e - row * half);
        }
      }
      __syncthreads();
    }
  }
  return sweep;
}

// acc += a * b (df64 operands), exact leading product and sum, all second
// order terms gathered in the low word
static __device__ __forceinline__ void mac_df(float& sh, float& se, float2 a, float2 b) {
  float pr = __fmul_rn(a.x, b.x);
  float pe = __fmaf_rn(a.x, b.x, -pr);
  float2 t = two_sum(sh, pr);
  sh = t.x;
  se = __fadd_rn(se, __fadd_rn(t.y, __fmaf_rn(a.x, b.y, __fmaf_rn(a.y, b.x, pe))));
}

// Out = op(X) Y, op = transpose if tx; df64 p x p, block-parallel; the
// result goes to Out (df64) or, with Out null, to Outd (float64). For
// p <= 64 a thread forms the 2 x 2 outputs (i, i + 1) x (j, j + 32), i from
// its warp, j its lane: the row operand is a warp broadcast and each loaded
// value serves two products, which halves the shared-memory loads of the
// one-output-per-thread form. Every output sums over k in the same order
// either way.
static __device__ void mm_df_to(int p, const float2* X, bool tx, const float2* Y, float2* Out, double* Outd) {
  auto put = [&](int e, float sh, float se) {
    const float2 v = fast_two_sum(sh, se);
    if (Out) Out[e] = v;
    else Outd[e] = df_to_double(v);
  };
  if (p <= 64) {
    const int nw = blockDim.x >> 5, wp = threadIdx.x >> 5, ln = threadIdx.x & 31;
    const int j0 = ln, j1 = ln + 32;
    const bool c0 = j0 < p, c1 = j1 < p;
    const int sx = tx ? p : 1;
    const float2 zero = make_float2(0.f, 0.f);
    for (int i = 2 * wp; i < p; i += 2 * nw) {
      const bool r1 = i + 1 < p;
      const float2* x0p = X + (tx ? i : i * p);
      const float2* x1p = X + (tx ? i + 1 : (i + 1) * p);
      float h00 = 0.f, e00 = 0.f, h01 = 0.f, e01 = 0.f, h10 = 0.f, e10 = 0.f, h11 = 0.f, e11 = 0.f;
      for (int k = 0; k < p; ++k) {
        const float2 x0 = x0p[k * sx], x1 = r1 ? x1p[k * sx] : zero;
        const float2 y0 = c0 ? Y[k * p + j0] : zero, y1 = c1 ? Y[k * p + j1] : zero;
        mac_df(h00, e00, x0, y0);
        mac_df(h01, e01, x0, y1);
        mac_df(h10, e10, x1, y0);
        mac_df(h11, e11, x1, y1);
      }
      if (c0) put(i * p + j0, h00, e00);
      if (c1) put(i * p + j1, h01, e01);
      if (r1 && c0) put((i + 1) * p + j0, h10, e10);
      if (r1 && c1) put((i + 1) * p + j1, h11, e11);
    }
  } else {
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
      int i = e / p, j = e - i * p;
      float sh = 0.f, se = 0.f;
      for (int k = 0; k < p; ++k) mac_df(sh, se, tx ? X[k * p + i] : X[i * p + k], Y[k * p + j]);
      put(e, sh, se);
    }
  }
  __syncthreads();
}

static __device__ void mm_df(int p, const float2* X, bool tx, const float2* Y, float2* Out) {
  mm_df_to(p, X, tx, Y, Out, nullptr);
}

// Out = G V with G float64 (symmetrised), V df64; G is converted once into Gd.
static __device__ void mm_f64_df(int p, const double* G, const float2* V, float2* Out, float2* Gd) {
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
    int i = e / p, j = e - i * p;
    Gd[e] = df_from_double(0.5 * (G[i * p + j] + G[j * p + i]));
  }
  __syncthreads();
  mm_df(p, Gd, false, V, Out);
}

// d_i = sum_k V[k,i] T[k,i]  (the diagonal of V^T (G V))
static __device__ void col_dots(int p, const float2* V, const float2* T, double* d) {
  for (int i = threadIdx.x; i < p; i += blockDim.x) {
    float sh = 0.f, se = 0.f;
    for (int k = 0; k < p; ++k) mac_df(sh, se, V[k * p + i], T[k * p + i]);
    d[i] = df_to_double(fast_two_sum(sh, se));
  }
  __syncthreads();
}

// Eigenbasis of the symmetric float64 G (p x p) into w.Vd (df64), w.Bd = V^T G V
// (diagonal up to rounding).
static __device__ void eig_refined(int p, const double* G, SdWs& w, double* red, double* diag) {
  const int q = p * p;
  for (int e = threadIdx.x; e < q; e += blockDim.x) {
    int i = e / p, j = e - i * p;
    w.Af[e] = (float)(0.5 * (G[i * p + j] + G[j * p + i]));
    w.Vf[e] = (i == j) ? 1.f : 0.f;
  }
  __syncthreads();
  // float32 sweeps down to ~1e-5 relative off-diagonal mass (above float32's
  // rounding floor); the df64 sweeps below converge quadratically from there
  long long c0 = clock64();
  int s32 = jacobi_f32(p, w.Af, w.Vf, w, red, 12, 1e-5);
  long long c1 = clock64();
  // V <- V0 (3 I - V0^T V0) / 2 in df64
  for (int e = threadIdx.x; e < q; e += blockDim.x) w.Ud[e] = make_float2(w.Vf[e], 0.f);
  __syncthreads();
  mm_df(p, w.Ud, true, w.Ud, w.Td);  // T = V0^T V0
  for (int e = threadIdx.x; e < q; e += blockDim.x) {
    int i = e / p, j = e - i * p;
    float2 t = w.Td[e];
    w.Td[e] = df_add(make_float2(i == j ? 1.5f : 0.f, 0.f), make_float2(-0.5f * t.x, -0.5f * t.y));
  }
  __syncthreads();
  mm_df(p, w.Ud, false, w.Td, w.Vd);  // V = V0 (1.5 I - 0.5 T)
  // second Newton-Schulz step: orthonormal to df64 rounding
  mm_df(p, w.Vd, true, w.Vd, w.Td);
  for (int e = threadIdx.x; e < q; e += blockDim.x) {
    int i = e / p, j = e - i * p;
    float2 t = w.Td[e];
    w.Td[e] = df_add(make_float2(i == j ? 1.5f : 0.f, 0.f), make_float2(-0.5f * t.x, -0.5f * t.y));
  }
  __syncthreads();
  mm_df(p, w.Vd, false, w.Td, w.Ud);
  for (int e = threadIdx.x; e < q; e += blockDim.x) w.Vd[e] = w.Ud[e];
  __syncthreads();
  mm_f64_df(p, G, w.Vd, w.Td, w.Ud);  // T = G V
  mm_df(p, w.Vd, true, w.Td, w.Bd);   // B' = V^T G V
  long long c2 = clock64();
  int s64 = jacobi_df(p, w.Bd, w.Vd, w, red, 4);
  if (threadIdx.x == 0 && diag) {
    diag[0] = (double)(c1 - c0);
    diag[1] = (double)(c2 - c1);
    diag[2] = (double)(clock64() - c2);
    diag[3] = s32;
    diag[4] = s64;
  }
}

// M = V [diag(s^-1/2) + F o Df] V^T for S' = V^T S V held in w.Bd (s = diag,
// F = off-diagonal). Returns 5 if some s_i <= 0.
static __device__ int inv_sqrt_in_basis(int p, SdWs& w, double* M, int* flag) {
  const int q = p * p;
  __shared__ double smax;
  if (threadIdx.x == 0) {
    *flag = 0;
    double m = 0.0;
    for (int i = 0; i < p; ++i) m = fmax(m, df_to_double(w.Bd[i * p + i]));
    smax = m;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < p; i += blockDim.x) {
    double s = df_to_double(w.Bd[i * p + i]);
    // numerically singular: below the df64 rounding level of the largest
    if (!(s > 1e-13 * smax) || !isfinite(s)) *flag = 5;
    w.sv[i] = s > 0.0 ? sqrt(s) : 1.0;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < q; e += blockDim.x) {
    int i = e / p, j = e - i * p;
    double v;
    if (i == j) {
      v = 1.0 / w.sv[i];
    } else {
      double ri = w.sv[i], rj = w.sv[j];
      v = -df_to_double(w.Bd[e]) / (ri * rj * (ri + rj));
    }
    w.Ud[e] = df_from_double(v);
  }
  __syncthreads();
  mm_df(p, w.Vd, false, w.Ud, w.Td);  // T = V N
  // M = T V^T: V^T into the free Ud, then a plain product into M (float64)
  for (int e = threadIdx.x; e < q; e += blockDim.x) {
    int i = e / p, j = e - i * p;
    w.Ud[j * p + i] = w.Vd[e];
  }
  __syncthreads();
  mm_df_to(p, w.Td, false, w.Ud, nullptr, M);
  return *flag;
}

// One p x p step for one problem, run by the whole calling block. mode 0:
// eigenbasis of B, line-search coefficients, the step t of Alg. 3 and
// M = S^{-1/2}; mode 1: M = B^{-1/2}; mode 2: eigenvectors of B (passed as
// B) into M, eigenvalues into XD[0..p), unsorted. Mode 0 in two launches:
// mode 3 only finds the eigenbasis of B and leaves V (p x p df64) and the
// diagonal of V^T B V (p df64) in eig; mode 4 takes them from there and
// does the rest. out: t, phi(t), Brent evaluations, status (0 or 5),
// beta_max, cycle counts (5..12).
static __device__ void small_df_body(int mode, int p, const double* C, const double* B,
                                     const double* Gam, const double* Z, const double* XX,
                                     const double* XD, double* M, double* out, SdWs& w, double* red,
                                     int* flagp, double* sh_tp, float2* eig = nullptr) {
  double& sh_t = *sh_tp;
  const int q = p * p;
  long long t0 = clock64();
  if (mode == 4) {
    for (int e = threadIdx.x; e < q; e += blockDim.x) w.Vd[e] = eig[e];
    for (int i = threadIdx.x; i < p; i += blockDim.x) w.Bd[i * p + i] = eig[q + i];
    __syncthreads();
  } else {
    eig_refined(p, B, w, red, out + 8);
  }
  long long t1 = clock64();
  if (mode == 3) {
    for (int e = threadIdx.x; e < q; e += blockDim.x) eig[e] = w.Vd[e];
    for (int i = threadIdx.x; i < p; i += blockDim.x) eig[q + i] = w.Bd[i * p + i];
    if (threadIdx.x == 0) out[5] = (double)(t1 - t0);
    return;
  }
  if (mode == 2) {
    // Rayleigh-Ritz: eigenvectors of C (here passed as B) into M (float64),
    // eigenvalues into XD[0..p) (unsorted; column i of M belongs to XD[i])
    for (int e = threadIdx.x; e < q; e += blockDim.x) M[e] = df_to_double(w.Vd[e]);
    for (int i = threadIdx.x; i < p; i += blockDim.x)
      const_cast<double*>(XD)[i] = df_to_double(w.Bd[i * p + i]);
    if (threadIdx.x == 0) out[3] = 0.0;
    return;
  }
  if (mode == 1) {
    int st = inv_sqrt_in_basis(p, w, M, flagp);
    if (threadIdx.x == 0) {
      out[0] = out[1] = out[2] = 0.0;
      out[3] = (double)st;
    }
    return;
  }
  for (int i = threadIdx.x; i < p; i += blockDim.x) w.be[i] = fmax(df_to_double(w.Bd[i * p + i]), 0.0);
  __syncthreads();
  mm_f64_df(p, C, w.Vd, w.Td, w.Ud);
  col_dots(p, w.Vd, w.Td, w.al);
  mm_f64_df(p, Gam, w.Vd, w.Td, w.Ud);
  col_dots(p, w.Vd, w.Td, w.ga);
  mm_f64_df(p, Z, w.Vd, w.Td, w.Ud);
  col_dots(p, w.Vd, w.Td, w.ze);
  long long t2 = clock64();
  if (threadIdx.x < 32) {
    int ev = 0;
    double t = get_mu_warp(p, w.al, w.be, w.ga, w.ze, &ev);
    double bmax = 0.0;
    for (int i = 0; i < p; ++i) bmax = fmax(bmax, w.be[i]);
    double ph = phi_model_warp(t, p, w.al, w.be, w.ga, w.ze);
    if (threadIdx.x == 0) {
      sh_t = t;
      out[0] = t;
      out[1] = ph;
      out[2] = (double)ev;
      out[4] = bmax;
    }
  }
  __syncthreads();
  const double t = sh_t;
  // S' = V^T S V with S = XX + t (XD + XD^T) + t^2 B
  for (int e = threadIdx.x; e < q; e += blockDim.x) {
    int i = e / p, j = e - i * p;
    double sij = 0.5 * (XX[i * p + j] + XX[j * p + i]) + t * (XD[i * p + j] + XD[j * p + i]) +
                 t * t * 0.5 * (B[i * p + j] + B[j * p + i]);
    w.Ud[e] = df_from_double(sij);
  }
  __syncthreads();
  mm_df(p, w.Ud, false, w.Vd, w.Td);  // T = S V
  mm_df(p, w.Vd, true, w.Td, w.Bd);   // S' = V^T T
  long long t3 = clock64();
  int st = inv_sqrt_in_basis(p, w, M, flagp);
  if (threadIdx.x == 0) {
    out[3] = (double)st;
    // cycles spent: eigenbasis (mode 3 wrote it), coefficients, line
    // search, polar normaliser
    if (mode != 4) out[5] = (double)(t1 - t0);
    out[6] = (double)(t3 - t1);
    out[7] = (double)(clock64() - t3);
  }
}

}  // namespace gsi
