// Batched solver: many independent problems A_i (CSR, float32 entries, the
// dominant p_i-dimensional subspace of each) iterated together by the
// methods of Alg. 2 / Alg. 4 with the exact line search of Alg. 3 and the
// one-matvec recursion of Eq. (save_matvec), exactly as the single-problem
// solver does it, but with every decision taken on the device so that whole
// iterations -- and the whole solve -- run without the host.
//
// Work decomposition. Every problem's rows are cut into tiles of `tile_rows`
// rows; the tile table (problem, first row, rows) lists the problems by
// descending p, then descending n, so the tiles of one problem are adjacent.
// The n x p work of one pass (Gram products, residual, direction update,
// SpMM, retraction) is done by persistent grid-stride kernels over that table;
// each tile is skipped unless its problem's flags select it. Gram products
// leave float64 partial sums per tile, summed per problem in tile order
// (deterministic). The p x p step runs one thread block per problem in
// float64. Small control kernels (one thread per problem) take the decisions
// of the single-problem iteration: stop test, Polak-Ribiere beta, restart,
// explicit recompute of AX, step counting.
//
// Block data are df64 (float2 hi + lo); operator entries float32 (exact for
// the graph Laplacians with float32-rounded shifts this path is meant for).
// The pass sequence is captured once into a CUDA graph whose while-node runs
// passes until no problem is active, so one graph launch performs the solve;
// a host loop over the same passes is kept for tuning and stepping.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "alg3.cuh"
#include "common.cuh"
#include "df.cuh"
#include "oz.cuh"
#include "small_df_dev.cuh"

namespace gsi {
namespace {

constexpr int BT = 256;    // threads of the tile kernels
constexpr int BS = 256;    // threads of the per-problem p x p kernel
constexpr int PMAX = 32;   // largest block width of a batched problem
constexpr int RC = 32;     // rows per staged chunk in the Gram kernel
constexpr int NG = 4;      // Gram products per tile slot
constexpr int kTileMin = 64;  // fewest rows of a tile

enum : int32_t {
  F_ACTIVE = 1,    // still iterating
  F_STEP = 2,      // takes a step in this pass
  F_Y = 4,         // Y = A X explicitly at the end of this pass
  F_DIR = 8,       // CG direction update with the previous direction
  F_RESTART = 16,  // CG restart: D = R
  F_START = 32     // orthonormalisation / Rayleigh-Ritz passes
};

struct BProb {
  int32_t n, p, tmin, pad;  // tmin: fewest rows of one of its tiles
  int64_t roff, boff, ppoff;
  double anorm;
};

struct BTile {
  int32_t prob, row0, rows, pad;
  int64_t part;  // offset (doubles) of the tile's Gram partials
};

struct BState {
  int32_t flags, status, iters, matvecs, restarts, evals, y_fresh, have_prev, converged;
  int32_t rsel;  // R[rsel] holds the residual of the last step; R[1 - rsel] this pass's
  double rr, rp, rr_prev, rinf, res0_inf, rel, rel_inf, t, beta, bmax, trace;
};

struct BDev {
  int32_t nprob, cg, max_iters, recompute_every, explicit_ax, k_restart, body_bound;
  int32_t tile_max, target_tiles;
  double tol;
  const BProb* prob;
  const int32_t* order;  // problems by descending p, descending n, index
  BTile* tile;           // this pass's tiles, built on the device
  int2* ptile;           // per problem: first tile, number of tiles
  int32_t* ntiles;       // number of tiles of this pass
  BState* st;
  const int64_t* rowptr;
  const int32_t* colidx;
  const float* val;
  float2 *X, *Y, *D, *W;
  float2* R[2];
  double *Cm, *Km, *Mm, *XDm, *theta, *G4, *parts, *tdots;
  int32_t* counter;  // [0] passes run, [1] problems still active, [2] this pass had work
};

// this pass's residual of problem i
__device__ __forceinline__ float2* rcur(const BDev& d, int i) { return d.st[i].rsel ? d.R[0] : d.R[1]; }

// (h, e) += a x with a, x df64: the leading product exactly (TwoProd) and
// added exactly (TwoSum); the second-order terms go to e.
__device__ __forceinline__ void bmac(float& h, float& e, float2 a, float2 x) {
  float p = __fmul_rn(a.x, x.x);
  float pe = __fmaf_rn(a.x, x.x, -p);
  float2 t = two_sum(h, p);
  h = t.x;
  e = __fadd_rn(e, __fadd_rn(t.y, __fmaf_rn(a.x, x.y, __fmaf_rn(a.y, x.x, pe))));
}

// (h, e) += a x with a float32 (an operator entry), x df64
__device__ __forceinline__ void bmac_f(float& h, float& e, float a, float2 x) {
  float p = __fmul_rn(a, x.x);
  float pe = __fmaf_rn(a, x.x, -p);
  float2 t = two_sum(h, p);
  h = t.x;
  e = __fadd_rn(e, __fadd_rn(t.y, __fmaf_rn(a, x.y, pe)));
}

__device__ __forceinline__ void renorm(float& h, float& e) {
  float2 s = fast_two_sum(h, e);
  h = s.x;
  e = s.y;
}

__device__ __forceinline__ float2 dneg(float2 a) { return make_float2(-a.x, -a.y); }

// block sum of a double, result valid in thread 0
__device__ double bsum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
  __syncthreads();
  return s;
}

__device__ float bmaxf(float v, float* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  float s = 0.f;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s = fmaxf(s, red[i]);
  __syncthreads();
  return s;
}

// ---- Gram partials ---------------------------------------------------------
// G = 1: sel 0 -> X^T Y, sel 1 -> X^T X, sel 2 -> X^T W.
// G = 4: D^T D, D^T W, D^T R, X^T X (the line-search Grams, Eqs. (diags),
// (CG_linesearch_D), and the measured X^T X of the polar factor).
// A thread owns 2 x 2 output blocks and a subset of the tile's rows; partial
// sums are df64 in registers, float64 in the tile's slot.
template <int G>
__global__ void __launch_bounds__(BT) b_gram_kernel(BDev d, int32_t mask, int32_t sel) {
  constexpr int NA = G == 4 ? 4 : 2;
  constexpr int UPT = G == 4 ? 4 : 1;  // most units per thread (p = 32)
  __shared__ __align__(16) float4 sm[NA][RC * PMAX / 2];
  __shared__ double red[BT * 4];
  const int tid = threadIdx.x;
  const int nt = *d.ntiles;
  for (int t = blockIdx.x; t < nt; t += gridDim.x) {
    const BTile tl = d.tile[t];
    if (!(d.st[tl.prob].flags & mask)) continue;
    const BProb pr = d.prob[tl.prob];
    const int p = pr.p, nb = p >> 1, nbb = nb * nb;
    const int units = G * nbb;
    const bool wide = units >= BT;
    const int upt = wide ? units / BT : 1;
    const int S = wide ? 1 : BT / units;
    const int s = wide ? 0 : tid / units;
    const int ub = wide ? tid : tid % units;
    const float2* src[NA];
    int nload;
    if (G == 4) {
      src[0] = d.D;
      src[1] = d.W;
      src[2] = rcur(d, tl.prob);
      src[3] = d.X;
      nload = 4;
    } else {
      src[0] = d.X;
      src[1] = sel == 0 ? d.Y : d.W;
      nload = sel == 1 ? 1 : 2;
    }
    int ia[UPT], ib[UPT], bi[UPT], bj[UPT];
#pragma unroll
    for (int u = 0; u < UPT; ++u) {
      const int unit = ub + u * BT;
      const int g = unit / max(nbb, 1), rem = unit - g * nbb;
      bi[u] = rem / nb;
      bj[u] = rem - bi[u] * nb;
      if (G == 4) {
        ia[u] = g == 3 ? 3 : 0;
        ib[u] = g == 3 ? 3 : g;
      } else {
        ia[u] = 0;
        ib[u] = nload == 1 ? 0 : 1;
      }
    }
    float h[UPT][4], e[UPT][4];
#pragma unroll
    for (int u = 0; u < UPT; ++u)
#pragma unroll
      for (int q = 0; q < 4; ++q) h[u][q] = e[u][q] = 0.f;
    for (int c0 = 0; c0 < tl.rows; c0 += RC) {
      const int rows = min(RC, tl.rows - c0);
      const int64_t off = pr.boff + (int64_t)(tl.row0 + c0) * p;
      __syncthreads();
      for (int a = 0; a < nload; ++a) {
        const float4* g4 = reinterpret_cast<const float4*>(src[a] + off);
        for (int i = tid; i < rows * nb; i += BT) sm[a][i] = g4[i];
      }
      __syncthreads();
      for (int r = s; r < rows; r += S) {
#pragma unroll
        for (int u = 0; u < UPT; ++u) {
          if (u < upt) {
            const float4 a = sm[ia[u]][r * nb + bi[u]];
            const float4 b = sm[ib[u]][r * nb + bj[u]];
            bmac(h[u][0], e[u][0], make_float2(a.x, a.y), make_float2(b.x, b.y));
            bmac(h[u][1], e[u][1], make_float2(a.x, a.y), make_float2(b.z, b.w));
            bmac(h[u][2], e[u][2], make_float2(a.z, a.w), make_float2(b.x, b.y));
            bmac(h[u][3], e[u][3], make_float2(a.z, a.w), make_float2(b.z, b.w));
          }
        }
      }
#pragma unroll
      for (int u = 0; u < UPT; ++u)
#pragma unroll
        for (int q = 0; q < 4; ++q) renorm(h[u][q], e[u][q]);
    }
    double* out = d.parts + tl.part;
    if (wide) {
#pragma unroll
      for (int u = 0; u < UPT; ++u) {
        if (u < upt) {
          const int unit = ub + u * BT, g = unit / nbb;
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int i = 2 * bi[u] + (q >> 1), j = 2 * bj[u] + (q & 1);
            out[(int64_t)g * p * p + i * p + j] = (double)h[u][q] + (double)e[u][q];
          }
        }
      }
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) red[(s * units + ub) * 4 + q] = (double)h[0][q] + (double)e[0][q];
      __syncthreads();
      for (int k = tid; k < units * 4; k += BT) {
        double v = 0.0;
        for (int z = 0; z < S; ++z) v += red[z * units * 4 + k];
        const int unit = k >> 2, q = k & 3, g = unit / nbb, rem = unit - g * nbb;
        const int i = 2 * (rem / nb) + (q >> 1), j = 2 * (rem % nb) + (q & 1);
        out[(int64_t)g * p * p + i * p + j] = v;
      }
      __syncthreads();
    }
  }
}

// ---- the pass's tile table ---------------------------------------------------

// exclusive prefix sum over a block of 1024 threads; *total gets the sum
template <typename T>
__device__ T block_exscan(T v, T* wbuf, T* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  T x = v;
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wbuf[w] = x;
  __syncthreads();
  if (w == 0) {
    T z = wbuf[lane];
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, z, o);
      if (lane >= o) z += y;
    }
    wbuf[lane] = z;  // inclusive sums of the warp totals
  }
  __syncthreads();
  const T before = (w > 0 ? wbuf[w - 1] : T(0)) + x - v;
  *total = wbuf[31];
  __syncthreads();
  return before;
}

// Tiles for the problems selected by mask, in the fixed problem order. With
// S the selected rows and T = ceil(S / target_tiles), problem i is cut into
// tiles of T_i = min(tile_max, max(tmin_i, T)) rows (the last one ragged):
// while every problem is active the tiles are tile_max rows long; when few
// remain they shrink to spread those problems over the whole GPU, down to
// tmin_i = 64 rows. One block of 1024 threads.
__global__ void __launch_bounds__(1024) b_plan_kernel(BDev d, int32_t mask) {
  __shared__ long long wl[32];
  __shared__ int wi[32];
  const int tid = threadIdx.x;
  long long S = 0;
  for (int k = tid; k < d.nprob; k += 1024) {
    const int i = d.order[k];
    if (d.st[i].flags & mask) S += d.prob[i].n;
  }
  long long tot = 0;
  const long long before = block_exscan<long long>(S, wl, &tot);
  (void)before;
  S = tot;
  const long long T = S > 0 ? (S + d.target_tiles - 1) / d.target_tiles : 1;
  int base_t = 0;
  long long base_p = 0;
  for (int c0 = 0; c0 < d.nprob; c0 += 1024) {
    const int k = c0 + tid;
    int i = -1, cnt = 0, Ti = 1;
    long long psz = 0;
    if (k < d.nprob) {
      i = d.order[k];
      if (d.st[i].flags & mask) {
        const BProb pr = d.prob[i];
        Ti = (int)min((long long)d.tile_max, max((long long)pr.tmin, T));
        cnt = (pr.n + Ti - 1) / Ti;
        psz = (long long)cnt * NG * pr.p * pr.p;
      }
    }
    int tot_t = 0;
    long long tot_p = 0;
    const int off_t = block_exscan<int>(cnt, wi, &tot_t);
    const long long off_p = block_exscan<long long>(psz, wl, &tot_p);
    if (i >= 0) {
      const BProb pr = d.prob[i];
      const int t0 = base_t + off_t;
      d.ptile[i] = make_int2(t0, cnt);
      const long long slot = (long long)NG * pr.p * pr.p;
      for (int j = 0; j < cnt; ++j) {
        BTile tl;
        tl.prob = i;
        tl.row0 = j * Ti;
        tl.rows = min(Ti, pr.n - j * Ti);
        tl.pad = 0;
        tl.part = base_p + off_p + j * slot;
        d.tile[t0 + j] = tl;
      }
    }
    base_t += tot_t;
    base_p += tot_p;
  }
  if (tid == 0) {
    *d.ntiles = base_t;
    if (mask == F_ACTIVE) d.counter[2] = S > 0 ? 1 : 0;
  }
}

// Sums of the tile partials of problems selected by mask: ng products of
// p x p, product g symmetrised as (G + G^T)/2 when bit g of symmask is set;
// into Cm (dst 0) or the problem's four line-search Grams in G4 (dst 1).
// A problem's tile slots are consecutive. Block = 32 entries x 8 tile
// groups: warp w sums the tiles j = w, w + 8, ... in ascending order (lanes
// on consecutive entries), then the 8 group sums are added in group order.
// Grid (nprob, chunks of 32 entries).
__global__ void __launch_bounds__(256) b_reduce_kernel(BDev d, int32_t mask, int32_t ng,
                                                       int32_t symmask, int32_t dst) {
  __shared__ double ra[8][32], rb[8][32];
  const int i = blockIdx.x;
  if (!(d.st[i].flags & mask)) return;
  const BProb pr = d.prob[i];
  const int2 pt = d.ptile[i];
  const int p = pr.p, q = p * p;
  const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
  const int e = blockIdx.y * 32 + lane;
  if ((int)blockIdx.y * 32 >= ng * q || pt.y == 0) return;
  const bool ok = e < ng * q;
  const int g = ok ? e / q : 0, rem = e - g * q, r = rem / p, c = rem - r * p;
  const bool sym = ok && ((symmask >> g) & 1);
  const int e2 = g * q + c * p + r;
  const int64_t slot = (int64_t)NG * q;
  const double* P0 = d.parts + d.tile[pt.x].part;
  double a = 0.0, bb = 0.0;
  if (ok) {
    int j = grp;
    for (; j + 24 < pt.y; j += 32) {  // four tiles of this group per round
      const double x0 = P0[j * slot + e], x1 = P0[(j + 8) * slot + e];
      const double x2 = P0[(j + 16) * slot + e], x3 = P0[(j + 24) * slot + e];
      a += x0;
      a += x1;
      a += x2;
      a += x3;
      if (sym) {
        const double y0 = P0[j * slot + e2], y1 = P0[(j + 8) * slot + e2];
        const double y2 = P0[(j + 16) * slot + e2], y3 = P0[(j + 24) * slot + e2];
        bb += y0;
        bb += y1;
        bb += y2;
        bb += y3;
      }
    }
    for (; j < pt.y; j += 8) {
      a += P0[j * slot + e];
      if (sym) bb += P0[j * slot + e2];
    }
  }
  ra[grp][lane] = a;
  rb[grp][lane] = bb;
  __syncthreads();
  if (grp == 0 && ok) {
    double sa = 0.0, sb = 0.0;
    for (int k = 0; k < 8; ++k) {
      sa += ra[k][lane];
      sb += rb[k][lane];
    }
    double* out = dst == 0 ? d.Cm + pr.ppoff : d.G4 + (int64_t)NG * pr.ppoff;
    out[e] = sym ? 0.5 * (sa + sb) : sa;
  }
}

// ---- row-local block updates ------------------------------------------------
// thread <-> (row group rg, column j); a pass covers BT / p rows.

// R = Y - X C in place with <R,R>, <R,R_prev> and max_r sum_j |R_rj|; D = R
// where the direction is the gradient (SD, first CG step).
__global__ void __launch_bounds__(BT) b_resid_kernel(BDev d) {
  __shared__ float2 cs[PMAX * PMAX];
  __shared__ float2 xs[BT];
  __shared__ double red[BT / 32];
  __shared__ float redf[BT / 32];
  const int tid = threadIdx.x;
  const int nt = *d.ntiles;
  for (int t = blockIdx.x; t < nt; t += gridDim.x) {
    const BTile tl = d.tile[t];
    const int32_t flags = d.st[tl.prob].flags;
    if (!(flags & F_ACTIVE)) continue;
    const BProb pr = d.prob[tl.prob];
    const int p = pr.p, RP = BT / p, j = tid % p, rg = tid / p;
    const bool have_prev = d.st[tl.prob].have_prev != 0;
    const bool want_rp = d.cg && have_prev;
    const bool copy_d = !d.cg || !have_prev;
    const int rsel = d.st[tl.prob].rsel;
    const float2* __restrict__ Rold = rsel ? d.R[1] : d.R[0];
    float2* __restrict__ Rnew = rsel ? d.R[0] : d.R[1];
    __syncthreads();
    for (int e = tid; e < p * p; e += BT) cs[e] = df_from_double(d.Cm[pr.ppoff + e]);
    __syncthreads();
    float rrh = 0.f, rre = 0.f, rph = 0.f, rpe = 0.f, rinf = 0.f;
    for (int r0 = 0; r0 < tl.rows; r0 += RP) {
      const int r = r0 + rg;
      const bool ok = r < tl.rows;
      const int64_t idx = pr.boff + (int64_t)(tl.row0 + r) * p + j;
      if (ok) xs[tid] = d.X[idx];
      __syncthreads();
      float ab = 0.f;
      if (ok) {
        float ah = 0.f, ae = 0.f;
        for (int k = 0; k < p; ++k) bmac(ah, ae, xs[rg * p + k], cs[k * p + j]);
        const float2 xc = fast_two_sum(ah, ae);
        const float2 rn = df_add(d.Y[idx], dneg(xc));
        if (want_rp) bmac(rph, rpe, rn, Rold[idx]);
        Rnew[idx] = rn;
        if (copy_d) d.D[idx] = rn;
        bmac(rrh, rre, rn, rn);
        ab = fabsf(rn.x);
      }
      for (int o = 1; o < p; o <<= 1) ab += __shfl_xor_sync(0xffffffffu, ab, o);
      rinf = fmaxf(rinf, ab);
      renorm(rrh, rre);
      renorm(rph, rpe);
      __syncthreads();
    }
    const double v0 = bsum((double)rrh + (double)rre, red);
    const double v1 = bsum((double)rph + (double)rpe, red);
    const float v2 = bmaxf(rinf, redf);
    if (tid == 0) {
      d.tdots[(int64_t)t * 4 + 0] = v0;
      d.tdots[(int64_t)t * 4 + 1] = v1;
      d.tdots[(int64_t)t * 4 + 2] = (double)v2;
    }
  }
}

// CG direction (Eq. (Pnew) with the projection transport): D <- R + beta D -
// X (beta K) in place, with <D, R>.
__global__ void __launch_bounds__(BT) b_dir_kernel(BDev d) {
  __shared__ float2 ks[PMAX * PMAX];
  __shared__ float2 xs[BT];
  __shared__ double red[BT / 32];
  const int tid = threadIdx.x;
  const int nt = *d.ntiles;
  for (int t = blockIdx.x; t < nt; t += gridDim.x) {
    const BTile tl = d.tile[t];
    if (!(d.st[tl.prob].flags & F_DIR)) continue;
    const BProb pr = d.prob[tl.prob];
    const int p = pr.p, RP = BT / p, j = tid % p, rg = tid / p;
    const double beta = d.st[tl.prob].beta;
    const float2 bd = df_from_double(beta);
    const float2* __restrict__ Rc = rcur(d, tl.prob);
    __syncthreads();
    for (int e = tid; e < p * p; e += BT) ks[e] = df_from_double(beta * d.Km[pr.ppoff + e]);
    __syncthreads();
    float drh = 0.f, dre = 0.f;
    for (int r0 = 0; r0 < tl.rows; r0 += RP) {
      const int r = r0 + rg;
      const bool ok = r < tl.rows;
      const int64_t idx = pr.boff + (int64_t)(tl.row0 + r) * p + j;
      if (ok) xs[tid] = d.X[idx];
      __syncthreads();
      if (ok) {
        float ah = 0.f, ae = 0.f;
        for (int k = 0; k < p; ++k) bmac(ah, ae, xs[rg * p + k], ks[k * p + j]);
        const float2 xk = fast_two_sum(ah, ae);
        const float2 rv = Rc[idx];
        const float2 dn = df_add(df_add(rv, df_mul(bd, d.D[idx])), dneg(xk));
        d.D[idx] = dn;
        bmac(drh, dre, dn, rv);
      }
      renorm(drh, dre);
      __syncthreads();
    }
    const double v = bsum((double)drh + (double)dre, red);
    if (tid == 0) d.tdots[(int64_t)t * 4 + 3] = v;
  }
}

// D = R (CG restart)
__global__ void __launch_bounds__(BT) b_copy_kernel(BDev d) {
  const int nt = *d.ntiles;
  for (int t = blockIdx.x; t < nt; t += gridDim.x) {
    const BTile tl = d.tile[t];
    if (!(d.st[tl.prob].flags & F_RESTART)) continue;
    const BProb pr = d.prob[tl.prob];
    const int64_t b = pr.boff + (int64_t)tl.row0 * pr.p, cnt = (int64_t)tl.rows * pr.p;
    const float2* __restrict__ Rc = rcur(d, tl.prob);
    for (int64_t e = threadIdx.x; e < cnt; e += BT) d.D[b + e] = Rc[b + e];
  }
}

// Block matvec (Sec. 6.1): which 0 -> W = A D (step problems), 1 -> Y = A X,
// 2 -> W = A X; thread <-> (row, column j): the p lanes of a row read the
// gathered neighbour rows as p consecutive df64 entries.
__global__ void __launch_bounds__(BT) b_spmm_kernel(BDev d, int32_t mask, int32_t which) {
  const int tid = threadIdx.x;
  const float2* in = which == 0 ? d.D : d.X;
  float2* out = which == 1 ? d.Y : d.W;
  const int nt = *d.ntiles;
  for (int t = blockIdx.x; t < nt; t += gridDim.x) {
    const BTile tl = d.tile[t];
    if (!(d.st[tl.prob].flags & mask)) continue;
    const BProb pr = d.prob[tl.prob];
    const int p = pr.p, RP = BT / p, j = tid % p, rg = tid / p;
    const float2* xin = in + pr.boff + j;
    for (int r = rg; r < tl.rows; r += RP) {
      const int64_t gr = pr.roff + tl.row0 + r;
      const int64_t kb = d.rowptr[gr], ke = d.rowptr[gr + 1];
      float h = 0.f, e = 0.f;
      for (int64_t k = kb; k < ke; ++k) bmac_f(h, e, __ldg(d.val + k), xin[(int64_t)__ldg(d.colidx + k) * p]);
      out[pr.boff + (int64_t)(tl.row0 + r) * p + j] = fast_two_sum(h, e);
    }
  }
}

// mode 0 (step problems): X <- (X + tD) M and, unless Y is recomputed,
// Y <- (Y + tW) M (Eqs. (Ynew), (save_matvec)); mode 1: X <- X M;
// mode 2: W <- X M (X unchanged).
__global__ void __launch_bounds__(BT) b_retract_kernel(BDev d, int32_t mode) {
  __shared__ float2 ms[PMAX * PMAX];
  __shared__ float2 zs[BT];
  const int tid = threadIdx.x;
  const int32_t mask = mode == 0 ? F_STEP : F_START;
  const int nt = *d.ntiles;
  for (int t = blockIdx.x; t < nt; t += gridDim.x) {
    const BTile tl = d.tile[t];
    const int32_t flags = d.st[tl.prob].flags;
    if (!(flags & mask)) continue;
    const BProb pr = d.prob[tl.prob];
    const int p = pr.p, RP = BT / p, j = tid % p, rg = tid / p;
    const float2 td = df_from_double(mode == 0 ? d.st[tl.prob].t : 0.0);
    const bool upd_y = mode == 0 && !(flags & F_Y);
    __syncthreads();
    for (int e = tid; e < p * p; e += BT) ms[e] = df_from_double(d.Mm[pr.ppoff + e]);
    __syncthreads();
    float2* xo = mode == 2 ? d.W : d.X;
    for (int r0 = 0; r0 < tl.rows; r0 += RP) {
      const int r = r0 + rg;
      const bool ok = r < tl.rows;
      const int64_t idx = pr.boff + (int64_t)(tl.row0 + r) * p + j;
      if (ok) {
        float2 z = d.X[idx];
        if (mode == 0) z = df_add(z, df_mul(td, d.D[idx]));
        zs[tid] = z;
      }
      __syncthreads();
      if (ok) {
        float ah = 0.f, ae = 0.f;
        for (int k = 0; k < p; ++k) bmac(ah, ae, zs[rg * p + k], ms[k * p + j]);
        xo[idx] = fast_two_sum(ah, ae);
      }
      __syncthreads();
      if (upd_y) {
        if (ok) zs[tid] = df_add(d.Y[idx], df_mul(td, d.W[idx]));
        __syncthreads();
        if (ok) {
          float ah = 0.f, ae = 0.f;
          for (int k = 0; k < p; ++k) bmac(ah, ae, zs[rg * p + k], ms[k * p + j]);
          d.Y[idx] = fast_two_sum(ah, ae);
        }
        __syncthreads();
      }
    }
  }
}

// ---- the p x p step, one block per problem ------------------------------------
// The step of the single-problem df64 path (float32 Jacobi refined to df64,
// Alg. 3 in float64, M = S^{-1/2} by the first-order expansion in the
// eigenbasis), run by one block per problem on its reduced Grams.
// mode 0 (step problems): X^T D = (I - X^T X)(C + beta K); the step t and
//   M; K_next = M (X^T D + t D^T D); the recompute decision.
// mode 1 (F_START): M = (X^T X)^{-1/2}.
// mode 2 (F_START): Rayleigh-Ritz, C' = U diag(theta) U^T, theta descending,
//   M = U.
__global__ void __launch_bounds__(BS) b_small_kernel(BDev d, int32_t mode) {
  const int i = blockIdx.x;
  const int32_t mask = mode == 0 ? F_STEP : F_START;
  if (!(d.st[i].flags & mask)) return;
  extern __shared__ __align__(16) unsigned char sm_dyn[];
  __shared__ double red[BS / 32];
  __shared__ int flag;
  __shared__ double sh_t;
  __shared__ double outs[16];
  __shared__ int order[PMAX];
  const int tid = threadIdx.x;
  const BProb pr = d.prob[i];
  const int p = pr.p, q = p * p;
  SdWs w = sd_carve(sm_dyn, p);
  double* M = d.Mm + pr.ppoff;
  double* XD = d.XDm + pr.ppoff;
  const double* C = d.Cm + pr.ppoff;
  const double* G4 = d.G4 + (int64_t)NG * pr.ppoff;  // D^T D, D^T W, D^T R, X^T X
  if (mode == 1) {
    small_df_body(1, p, nullptr, G4, nullptr, nullptr, nullptr, nullptr, M, outs, w, red, &flag, &sh_t);
    __syncthreads();
    if (tid == 0 && outs[3] != 0.0) {
      d.st[i].status = GSI_ERR_BREAKDOWN;
      d.st[i].flags = 0;
    }
    return;
  }
  if (mode == 2) {
    small_df_body(2, p, nullptr, G4, nullptr, nullptr, nullptr, XD, M, outs, w, red, &flag, &sh_t);
    __syncthreads();
    if (tid == 0) {
      for (int k = 0; k < p; ++k) order[k] = k;
      for (int a = 0; a < p; ++a) {  // selection sort, descending
        int best = a;
        for (int c = a + 1; c < p; ++c)
          if (XD[order[c]] > XD[order[best]]) best = c;
        const int tmp = order[a];
        order[a] = order[best];
        order[best] = tmp;
      }
    }
    double* tmp = reinterpret_cast<double*>(w.Td);  // q doubles of scratch
    for (int e = tid; e < q; e += BS) tmp[e] = M[e];
    __syncthreads();
    for (int k = tid; k < p; k += BS) d.theta[pr.ppoff + k] = XD[order[k]];
    for (int e = tid; e < q; e += BS) {
      const int r = e / p, c = e - r * p;
      M[e] = tmp[r * p + order[c]];
    }
    return;
  }
  const double beta_used = d.st[i].beta;
  const double* Bm = G4;
  const double* XX = G4 + 3 * q;
  double* G2 = reinterpret_cast<double*>(w.Ud);  // q doubles of scratch
  for (int e = tid; e < q; e += BS)
    G2[e] = beta_used != 0.0 ? C[e] + beta_used * d.Km[pr.ppoff + e] : C[e];
  __syncthreads();
  for (int e = tid; e < q; e += BS) {
    const int r = e / p, c = e - r * p;
    double s = 0.0;
    for (int k = 0; k < p; ++k) s = fma(XX[r * p + k], G2[k * p + c], s);
    XD[e] = G2[e] - s;
  }
  __syncthreads();
  small_df_body(0, p, C, Bm, G4 + q, d.cg ? G4 + 2 * q : Bm, XX, XD, M, outs, w, red, &flag, &sh_t);
  __syncthreads();
  const double t = outs[0];
  if (!isfinite(t) || outs[3] != 0.0) {
    if (tid == 0) {
      d.st[i].status = isfinite(t) ? GSI_ERR_BREAKDOWN : GSI_ERR_NONFINITE;
      d.st[i].flags = 0;
    }
    return;
  }
  if (d.cg) {  // K_next = M (X^T D + t D^T D)
    double* T = reinterpret_cast<double*>(w.Ud);
    for (int e = tid; e < q; e += BS) T[e] = XD[e] + t * Bm[e];
    __syncthreads();
    for (int e = tid; e < q; e += BS) {
      const int r = e / p, c = e - r * p;
      double s = 0.0;
      for (int k = 0; k < p; ++k) s = fma(M[r * p + k], T[k * p + c], s);
      d.Km[pr.ppoff + e] = s;
    }
  }
  if (tid == 0) {
    BState s = d.st[i];
    s.t = t;
    s.evals = (int)outs[2];
    s.bmax = outs[4];
    const bool recompute = d.explicit_ax || t * sqrt(fmax(s.bmax, 0.0)) < 1e3 * ALG3_EPS ||
                           (d.recompute_every > 0 && (s.iters + 1) % d.recompute_every == 0);
    if (recompute) s.flags |= F_Y;
    d.st[i] = s;
  }
}

// ---- control (one thread per problem) -----------------------------------------

// sum over the lanes of a warp in a fixed order; lane 0's value for all
__device__ __forceinline__ double wsum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return __shfl_sync(0xffffffffu, v, 0);
}

__device__ __forceinline__ double wmax(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// after the residual: stop test, explicit-AX request, Polak-Ribiere beta
// (one warp per problem; lanes sum the tiles' dots)
__global__ void __launch_bounds__(128) b_ctl1_kernel(BDev d) {
  const int i = blockIdx.x * 4 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (i >= d.nprob) return;
  if (!(d.st[i].flags & F_ACTIVE)) return;
  const BProb pr = d.prob[i];
  const int2 pt = d.ptile[i];
  double rr = 0.0, rp = 0.0, rinf = 0.0;
  for (int t = pt.x + lane; t < pt.x + pt.y; t += 32) {
    rr += d.tdots[(int64_t)t * 4 + 0];
    rp += d.tdots[(int64_t)t * 4 + 1];
    rinf = fmax(rinf, d.tdots[(int64_t)t * 4 + 2]);
  }
  rr = wsum(rr);
  rp = wsum(rp);
  rinf = wmax(rinf);
  if (lane != 0) return;
  BState s = d.st[i];
  double tr = 0.0;
  for (int k = 0; k < pr.p; ++k) tr += d.Cm[pr.ppoff + k * pr.p + k];
  s.rr = rr;
  s.rp = rp;
  s.rinf = rinf;
  s.trace = tr;
  s.flags = F_ACTIVE;
  if (!isfinite(rr)) {
    s.status = GSI_ERR_NONFINITE;
    s.flags = 0;
    d.st[i] = s;
    return;
  }
  if (s.res0_inf < 0.0) s.res0_inf = rinf;
  s.rel = sqrt(rr) / pr.anorm;
  s.rel_inf = s.res0_inf > 0.0 ? rinf / s.res0_inf : 0.0;
  if (s.rel <= d.tol || s.iters >= d.max_iters) {
    if (!s.y_fresh) {
      s.flags |= F_Y;  // the final residual is always taken with an explicit AX
    } else {
      s.converged = s.rel <= d.tol;
      s.status = s.converged ? GSI_OK : GSI_ERR_NOCONV;
      s.flags = 0;
    }
  } else {
    s.flags |= F_STEP;
    s.beta = 0.0;
    if (d.cg && s.have_prev) {
      s.beta = (rr - rp) / s.rr_prev;
      s.flags |= F_DIR;
    }
  }
  d.st[i] = s;
}

// after the direction update: restart when <D, R> <= 0 or every k_restart
// (one warp per problem)
__global__ void __launch_bounds__(128) b_ctl2_kernel(BDev d) {
  const int i = blockIdx.x * 4 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (i >= d.nprob) return;
  if (!(d.st[i].flags & F_DIR)) return;
  const int2 pt = d.ptile[i];
  double dr = 0.0;
  for (int t = pt.x + lane; t < pt.x + pt.y; t += 32) dr += d.tdots[(int64_t)t * 4 + 3];
  dr = wsum(dr);
  if (lane != 0) return;
  BState s = d.st[i];
  const bool due = d.k_restart > 0 && s.iters % d.k_restart == 0;
  if (due || !(dr > 0.0)) {
    s.flags |= F_RESTART;
    s.restarts++;
    s.beta = 0.0;
  }
  d.st[i] = s;
}

// end of a pass: step bookkeeping; counts the problems still active and ends
// the graph's while-loop when none is (or when the pass bound is reached)
__global__ void __launch_bounds__(1024) b_ctl3_kernel(BDev d, int32_t use_cond,
                                                      cudaGraphConditionalHandle h) {
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  int mine = 0;
  for (int i = threadIdx.x; i < d.nprob; i += blockDim.x) {
    BState s = d.st[i];
    if (s.flags & F_STEP) {
      const bool y = (s.flags & F_Y) != 0;
      s.iters++;
      s.matvecs += y ? 2 : 1;
      s.y_fresh = y ? 1 : 0;
      s.rr_prev = s.rr;
      s.have_prev = 1;
      s.rsel = 1 - s.rsel;  // this step's residual becomes the previous one
    } else if (s.flags & F_Y) {
      s.y_fresh = 1;
      s.matvecs++;
    }
    s.flags &= F_ACTIVE;
    if (s.flags) ++mine;
    d.st[i] = s;
  }
  atomicAdd(&cnt, mine);
  __syncthreads();
  if (threadIdx.x == 0) {
    const int passes = d.counter[0] += d.counter[2];
    d.counter[1] = cnt;
    if (use_cond && (cnt == 0 || passes >= d.body_bound)) cudaGraphSetConditional(h, 0);
  }
}

__global__ void b_init_kernel(BDev d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.nprob) return;
  BState s;
  memset(&s, 0, sizeof(s));
  s.flags = F_ACTIVE | F_START;
  s.res0_inf = -1.0;
  s.y_fresh = 1;
  s.rel = s.rel_inf = NAN;
  d.st[i] = s;
}

// start finished: Y = A X was the first matvec
__global__ void b_started_kernel(BDev d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.nprob) return;
  BState s = d.st[i];
  s.flags &= ~F_START;
  s.matvecs = 1;
  d.st[i] = s;
}

// flags |= F_START for every problem (Rayleigh-Ritz), remembering the flags
__global__ void b_mark_kernel(BDev d, int32_t set, int32_t* saved) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.nprob) return;
  if (set) {
    saved[i] = d.st[i].flags;
    d.st[i].flags = d.st[i].status == GSI_ERR_BREAKDOWN || d.st[i].status == GSI_ERR_NONFINITE
                        ? 0
                        : F_START;
  } else {
    d.st[i].flags = saved[i];
  }
}

}  // namespace


// The problem order (descending p, then descending n, then ascending index)
// and the tile table of one pass over the problems with active[i] != 0 (all
// when active is empty), by the rule of b_plan_kernel. Host-only; it states
// the rule the device follows, for the library's callers and its tests.
gsi_status batched_plan(int nprob, const int32_t* n, const int32_t* p,
                        const std::vector<int32_t>& active, int tile_max, int target_tiles,
                        std::vector<int32_t>& order, std::vector<int32_t>& tprob,
                        std::vector<int32_t>& trow0, std::vector<int32_t>& trows) {
  if (nprob < 1 || !n || !p || tile_max < 1 || target_tiles < 1) return GSI_ERR_ARG;
  order.resize(nprob);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    if (p[a] != p[b]) return p[a] > p[b];
    if (n[a] != n[b]) return n[a] > n[b];
    return a < b;
  });
  auto on = [&](int i) { return active.empty() || active[i] != 0; };
  long long S = 0;
  for (int i = 0; i < nprob; ++i)
    if (on(i)) S += n[i];
  const long long T = S > 0 ? (S + target_tiles - 1) / target_tiles : 1;
  tprob.clear();
  trow0.clear();
  trows.clear();
  for (int k = 0; k < nprob; ++k) {
    const int i = order[k];
    if (!on(i)) continue;
    const long long tmin = kTileMin;
    const int Ti = (int)std::min((long long)tile_max, std::max(tmin, T));
    for (int r = 0; r < n[i]; r += Ti) {
      tprob.push_back(i);
      trow0.push_back(r);
      trows.push_back(std::min(Ti, n[i] - r));
    }
  }
  return GSI_OK;
}

}  // namespace gsi

using namespace gsi;

struct gsi_batch {
  cudaStream_t st = nullptr, cap = nullptr;
  int nprob = 0, pmax = 0;
  gsi_opts o{};
  std::vector<int32_t> n, p;
  std::vector<BProb> hprob;
  int64_t rows = 0, elems = 0, pp = 0, nnz = 0;
  int64_t* rowptr = nullptr;
  int32_t* colidx = nullptr;
  float* val = nullptr;
  double* X0 = nullptr;
  float2 *X = nullptr, *Y = nullptr, *D = nullptr, *W = nullptr;
  float2* R[2] = {nullptr, nullptr};
  BProb* prob = nullptr;
  int32_t* order = nullptr;
  BTile* tile = nullptr;
  int2* ptile = nullptr;
  int32_t* ntiles = nullptr;
  BState* state = nullptr;
  double *Cm = nullptr, *Km = nullptr, *Mm = nullptr, *XDm = nullptr, *theta = nullptr, *G4 = nullptr;
  double* parts = nullptr;
  double* tdots = nullptr;
  int32_t* counter = nullptr;
  int32_t* saved = nullptr;
  int32_t* hcounter = nullptr;  // pinned
  size_t parts_cap = 0, tiles_cap = 0;
  int tile_max = 2048, ctas_per_sm = 4, tiles_per_cta = 2, grid = 1;
  size_t small_smem = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  cudaGraphConditionalHandle handle = 0;
  bool ritz_valid = false;
  std::vector<BState> hstate;
  std::vector<void*> allocs;
};

namespace {

gsi_status balloc(gsi_batch* b, void** ptr, size_t bytes) {
  cudaError_t e = cudaMalloc(ptr, std::max<size_t>(bytes, 256));
  if (e != cudaSuccess) return cuda_status(e);
  b->allocs.push_back(*ptr);
  return GSI_OK;
}

void bfree(gsi_batch* b, void* ptr) {
  if (!ptr) return;
  auto it = std::find(b->allocs.begin(), b->allocs.end(), ptr);
  if (it != b->allocs.end()) b->allocs.erase(it);
  cudaFree(ptr);
}

BDev make_dev(gsi_batch* b) {
  BDev d{};
  d.nprob = b->nprob;
  d.cg = b->o.method == GSI_CG;
  d.max_iters = b->o.max_iters;
  d.recompute_every = b->o.recompute_every;
  d.explicit_ax = b->o.explicit_ax;
  d.k_restart = b->o.k_restart;
  d.body_bound = 2 * std::max(b->o.max_iters, 0) + 4;
  d.tile_max = b->tile_max;
  d.target_tiles = b->grid * b->tiles_per_cta;
  d.tol = b->o.tol;
  d.prob = b->prob;
  d.order = b->order;
  d.tile = b->tile;
  d.ptile = b->ptile;
  d.ntiles = b->ntiles;
  d.st = b->state;
  d.rowptr = b->rowptr;
  d.colidx = b->colidx;
  d.val = b->val;
  d.X = b->X;
  d.Y = b->Y;
  d.R[0] = b->R[0];
  d.R[1] = b->R[1];
  d.D = b->D;
  d.W = b->W;
  d.Cm = b->Cm;
  d.Km = b->Km;
  d.Mm = b->Mm;
  d.XDm = b->XDm;
  d.theta = b->theta;
  d.G4 = b->G4;
  d.parts = b->parts;
  d.tdots = b->tdots;
  d.counter = b->counter;
  return d;
}

void drop_graph(gsi_batch* b) {
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->gexec = nullptr;
  b->graph = nullptr;
}

// tile shape parameters; tile and partial-sum buffers sized for the finest
// tiles the rule can produce (every problem at min(tile_max, tmin_i) rows)
gsi_status set_tiles(gsi_batch* b, int tile_max, int ctas_per_sm, int tiles_per_cta) {
  size_t tiles = 0, parts = 0;
  for (int i = 0; i < b->nprob; ++i) {
    const int ti = std::min(tile_max, kTileMin);
    const size_t c = (size_t)((b->n[i] + ti - 1) / ti);
    tiles += c;
    parts += c * NG * b->p[i] * b->p[i];
  }
  GSI_CUDA_TRY(cudaStreamSynchronize(b->st));
  drop_graph(b);
  if (parts > b->parts_cap) {
    bfree(b, b->parts);
    b->parts = nullptr;
    GSI_TRY(balloc(b, (void**)&b->parts, parts * sizeof(double)));
    b->parts_cap = parts;
  }
  if (tiles > b->tiles_cap) {
    bfree(b, b->tile);
    bfree(b, b->tdots);
    b->tile = nullptr;
    b->tdots = nullptr;
    GSI_TRY(balloc(b, (void**)&b->tile, tiles * sizeof(BTile)));
    GSI_TRY(balloc(b, (void**)&b->tdots, tiles * 4 * sizeof(double)));
    b->tiles_cap = tiles;
  }
  b->tile_max = tile_max;
  b->ctas_per_sm = ctas_per_sm;
  b->tiles_per_cta = tiles_per_cta;
  b->grid = std::max(1, sm_count() * ctas_per_sm);
  return GSI_OK;
}

inline int pgrid(int nprob, int threads) { return (nprob + threads - 1) / threads; }

// the reduction grid: problems x chunks of 32 of the ng * pmax^2 entries
inline dim3 rgrid(gsi_batch* b, int ng) {
  return dim3((unsigned)b->nprob, (unsigned)((ng * b->pmax * b->pmax + 31) / 32));
}

// one pass of the iteration for every active problem
gsi_status launch_pass(gsi_batch* b, cudaStream_t s, int32_t use_cond) {
  const BDev d = make_dev(b);
  const int g = b->grid, np = b->nprob;
  b_plan_kernel<<<1, 1024, 0, s>>>(d, F_ACTIVE);
  GSI_LAUNCH_CHECK();
  b_gram_kernel<1><<<g, BT, 0, s>>>(d, F_ACTIVE, 0);  // C = X^T Y
  GSI_LAUNCH_CHECK();
  b_reduce_kernel<<<rgrid(b, 1), 256, 0, s>>>(d, F_ACTIVE, 1, 1, 0);
  GSI_LAUNCH_CHECK();
  b_resid_kernel<<<g, BT, 0, s>>>(d);  // R = Y - X C
  GSI_LAUNCH_CHECK();
  b_ctl1_kernel<<<pgrid(np, 4), 128, 0, s>>>(d);
  GSI_LAUNCH_CHECK();
  if (d.cg) {
    b_dir_kernel<<<g, BT, 0, s>>>(d);
    GSI_LAUNCH_CHECK();
    b_ctl2_kernel<<<pgrid(np, 4), 128, 0, s>>>(d);
    GSI_LAUNCH_CHECK();
    b_copy_kernel<<<g, BT, 0, s>>>(d);
    GSI_LAUNCH_CHECK();
  }
  b_spmm_kernel<<<g, BT, 0, s>>>(d, F_STEP, 0);  // W = A D
  GSI_LAUNCH_CHECK();
  b_gram_kernel<NG><<<g, BT, 0, s>>>(d, F_STEP, 0);
  GSI_LAUNCH_CHECK();
  // D^T D, D^T W, X^T X symmetrised; D^T R as it is
  b_reduce_kernel<<<rgrid(b, NG), 256, 0, s>>>(d, F_STEP, NG, 1 | 2 | 8, 1);
  GSI_LAUNCH_CHECK();
  b_small_kernel<<<np, BS, b->small_smem, s>>>(d, 0);
  GSI_LAUNCH_CHECK();
  b_retract_kernel<<<g, BT, 0, s>>>(d, 0);
  GSI_LAUNCH_CHECK();
  b_spmm_kernel<<<g, BT, 0, s>>>(d, F_Y, 1);  // Y = A X where requested
  GSI_LAUNCH_CHECK();
  b_ctl3_kernel<<<1, 1024, 0, s>>>(d, use_cond, b->handle);
  GSI_LAUNCH_CHECK();
  return GSI_OK;
}

// X0 -> df64, two polar orthonormalisations, Y = A X
gsi_status start(gsi_batch* b) {
  const BDev d = make_dev(b);
  const int g = b->grid, np = b->nprob;
  cudaStream_t s = b->st;
  GSI_TRY(df_from_f64(b->elems, b->X0, b->X, s));
  b_init_kernel<<<pgrid(np, 128), 128, 0, s>>>(d);
  GSI_LAUNCH_CHECK();
  b_plan_kernel<<<1, 1024, 0, s>>>(d, F_START);
  GSI_LAUNCH_CHECK();
  for (int pass = 0; pass < 2; ++pass) {
    b_gram_kernel<1><<<g, BT, 0, s>>>(d, F_START, 1);  // X^T X
    GSI_LAUNCH_CHECK();
    b_reduce_kernel<<<rgrid(b, 1), 256, 0, s>>>(d, F_START, 1, 1, 1);
    GSI_LAUNCH_CHECK();
    b_small_kernel<<<np, BS, b->small_smem, s>>>(d, 1);
    GSI_LAUNCH_CHECK();
    b_retract_kernel<<<g, BT, 0, s>>>(d, 1);
    GSI_LAUNCH_CHECK();
  }
  b_spmm_kernel<<<g, BT, 0, s>>>(d, F_START, 1);
  GSI_LAUNCH_CHECK();
  b_started_kernel<<<pgrid(np, 128), 128, 0, s>>>(d);
  GSI_LAUNCH_CHECK();
  GSI_CUDA_TRY(cudaMemsetAsync(b->counter, 0, 3 * sizeof(int32_t), s));
  b->ritz_valid = false;
  return GSI_OK;
}

gsi_status read_state(gsi_batch* b) {
  b->hstate.resize(b->nprob);
  GSI_CUDA_TRY(cudaMemcpyAsync(b->hstate.data(), b->state, (size_t)b->nprob * sizeof(BState),
                               cudaMemcpyDeviceToHost, b->st));
  GSI_CUDA_TRY(cudaStreamSynchronize(b->st));
  return GSI_OK;
}

gsi_status build_graph(gsi_batch* b) {
  drop_graph(b);
  GSI_CUDA_TRY(cudaGraphCreate(&b->graph, 0));
  GSI_CUDA_TRY(cudaGraphConditionalHandleCreate(&b->handle, b->graph, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = b->handle;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  GSI_CUDA_TRY(cudaGraphAddNode(&node, b->graph, nullptr, nullptr, 0, &np));
  cudaGraph_t body = np.conditional.phGraph_out[0];
  GSI_CUDA_TRY(cudaStreamBeginCaptureToGraph(b->cap, body, nullptr, nullptr, 0,
                                             cudaStreamCaptureModeThreadLocal));
  gsi_status s = launch_pass(b, b->cap, 1);
  cudaGraph_t captured = nullptr;
  cudaError_t e = cudaStreamEndCapture(b->cap, &captured);
  if (s != GSI_OK) return s;
  GSI_CUDA_TRY(e);
  GSI_CUDA_TRY(cudaGraphInstantiate(&b->gexec, b->graph, 0));
  return GSI_OK;
}

}  // namespace

extern "C" {

gsi_status gsi_batched_plan(int32_t nprob, const int32_t* n, const int32_t* p, const int32_t* active,
                            int32_t tile_max, int32_t target_tiles, int32_t* order, int32_t* ntiles,
                            int32_t* tile_prob, int32_t* tile_row0, int32_t* tile_rows,
                            int32_t capacity) {
  if (!ntiles || nprob < 1) return GSI_ERR_ARG;
  std::vector<int32_t> act, o, tp, tr0, trs;
  if (active) act.assign(active, active + nprob);
  GSI_TRY(batched_plan(nprob, n, p, act, tile_max, target_tiles, o, tp, tr0, trs));
  *ntiles = (int32_t)tp.size();
  if (order) std::copy(o.begin(), o.end(), order);
  if (tile_prob || tile_row0 || tile_rows) {
    if ((int64_t)capacity < (int64_t)tp.size()) return GSI_ERR_ARG;
    if (tile_prob) std::copy(tp.begin(), tp.end(), tile_prob);
    if (tile_row0) std::copy(tr0.begin(), tr0.end(), tile_row0);
    if (tile_rows) std::copy(trs.begin(), trs.end(), tile_rows);
  }
  return GSI_OK;
}

gsi_status gsi_batched_destroy(gsi_batch* b) {
  if (!b) return GSI_ERR_ARG;
  if (b->st) cudaStreamSynchronize(b->st);
  drop_graph(b);
  if (b->cap) cudaStreamDestroy(b->cap);
  for (void* ptr : b->allocs) cudaFree(ptr);
  if (b->hcounter) cudaFreeHost(b->hcounter);
  delete b;
  return GSI_OK;
}

gsi_status gsi_batched_create(int32_t nprob, const int32_t* n, const int32_t* p,
                              const int64_t* rowptr, const int32_t* colidx, const float* val,
                              const double* X0, const double* anorm, const gsi_opts* o,
                              void* stream, gsi_batch** out) {
  if (!out || nprob < 1 || !n || !p || !rowptr || !colidx || !val || !X0) return GSI_ERR_ARG;
  *out = nullptr;
  gsi_opts opts;
  gsi_default_opts(&opts);
  if (o) opts = *o;
  if ((opts.method != GSI_SD && opts.method != GSI_CG) || (opts.which != 1 && opts.which != -1) ||
      opts.max_iters < 0 || !(opts.tol >= 0.0))
    return GSI_ERR_ARG;
  // problem sizes and the concatenated CSR are checked on the host: the
  // kernels index with them unchecked
  int64_t rows = 0, elems = 0, pp = 0;
  int pmax = 0;
  for (int i = 0; i < nprob; ++i) {
    const int pi = p[i];
    if (pi != 2 && pi != 4 && pi != 8 && pi != 16 && pi != 32) return GSI_ERR_ARG;
    if (n[i] < 2 * pi) return GSI_ERR_ARG;
    pmax = std::max(pmax, pi);
    rows += n[i];
    elems += (int64_t)n[i] * pi;
    pp += (int64_t)pi * pi;
  }
  if (rowptr[0] != 0) return GSI_ERR_ARG;
  for (int64_t r = 0; r < rows; ++r)
    if (rowptr[r + 1] < rowptr[r]) return GSI_ERR_ARG;
  const int64_t nnz = rowptr[rows];
  {
    int64_t r = 0;
    for (int i = 0; i < nprob; ++i) {
      for (int64_t k = 0; k < n[i]; ++k, ++r)
        for (int64_t e = rowptr[r]; e < rowptr[r + 1]; ++e)
          if (colidx[e] < 0 || colidx[e] >= n[i]) return GSI_ERR_ARG;
    }
  }
  gsi_batch* b = new gsi_batch();
  b->st = (cudaStream_t)stream;
  b->nprob = nprob;
  b->pmax = pmax;
  b->o = opts;
  b->n.assign(n, n + nprob);
  b->p.assign(p, p + nprob);
  b->rows = rows;
  b->elems = elems;
  b->pp = pp;
  b->nnz = nnz;
  b->hprob.resize(nprob);
  const float sign = opts.which == -1 ? -1.f : 1.f;
  std::vector<float> hval(val, val + nnz);
  if (sign < 0)
    for (auto& v : hval) v = -v;
  std::vector<int32_t> order, tp, tr0, trs;
  {
    int64_t r = 0, bo = 0, po = 0;
    for (int i = 0; i < nprob; ++i) {
      BProb& pr = b->hprob[i];
      pr.n = n[i];
      pr.p = p[i];
      pr.tmin = kTileMin;
      pr.pad = 0;
      pr.roff = r;
      pr.boff = bo;
      pr.ppoff = po;
      double mx = 0.0;
      for (int64_t k = 0; k < n[i]; ++k) {
        double s = 0.0;
        for (int64_t e = rowptr[r + k]; e < rowptr[r + k + 1]; ++e) s += fabs((double)hval[e]);
        mx = std::max(mx, s);
      }
      pr.anorm = (anorm && anorm[i] > 0.0) ? anorm[i] : (opts.anorm > 0.0 ? opts.anorm : mx);
      if (!(pr.anorm > 0.0)) pr.anorm = 1.0;
      r += n[i];
      bo += (int64_t)n[i] * p[i];
      po += (int64_t)p[i] * p[i];
    }
  }
  gsi_status s = batched_plan(nprob, n, p, std::vector<int32_t>(), 1 << 30, 1, order, tp, tr0, trs);
  if (s != GSI_OK) {
    delete b;
    return s;
  }
#define CK(expr)                \
  do {                          \
    s = (expr);                 \
    if (s != GSI_OK) goto fail; \
  } while (0)
  CK(cuda_status_ok(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking)));
  CK(balloc(b, (void**)&b->rowptr, (size_t)(rows + 1) * sizeof(int64_t)));
  CK(balloc(b, (void**)&b->colidx, (size_t)nnz * sizeof(int32_t)));
  CK(balloc(b, (void**)&b->val, (size_t)nnz * sizeof(float)));
  CK(balloc(b, (void**)&b->X0, (size_t)elems * sizeof(double)));
  CK(balloc(b, (void**)&b->X, (size_t)elems * sizeof(float2)));
  CK(balloc(b, (void**)&b->Y, (size_t)elems * sizeof(float2)));
  CK(balloc(b, (void**)&b->R[0], (size_t)elems * sizeof(float2)));
  CK(balloc(b, (void**)&b->R[1], (size_t)elems * sizeof(float2)));
  CK(balloc(b, (void**)&b->D, (size_t)elems * sizeof(float2)));
  CK(balloc(b, (void**)&b->W, (size_t)elems * sizeof(float2)));
  CK(balloc(b, (void**)&b->prob, (size_t)nprob * sizeof(BProb)));
  CK(balloc(b, (void**)&b->order, (size_t)nprob * sizeof(int32_t)));
  CK(balloc(b, (void**)&b->ptile, (size_t)nprob * sizeof(int2)));
  CK(balloc(b, (void**)&b->ntiles, sizeof(int32_t)));
  CK(balloc(b, (void**)&b->state, (size_t)nprob * sizeof(BState)));
  CK(balloc(b, (void**)&b->saved, (size_t)nprob * sizeof(int32_t)));
  CK(balloc(b, (void**)&b->Cm, (size_t)pp * sizeof(double)));
  CK(balloc(b, (void**)&b->Km, (size_t)pp * sizeof(double)));
  CK(balloc(b, (void**)&b->Mm, (size_t)pp * sizeof(double)));
  CK(balloc(b, (void**)&b->XDm, (size_t)pp * sizeof(double)));
  CK(balloc(b, (void**)&b->theta, (size_t)pp * sizeof(double)));
  CK(balloc(b, (void**)&b->G4, (size_t)NG * pp * sizeof(double)));
  CK(balloc(b, (void**)&b->counter, 3 * sizeof(int32_t)));
  CK(cuda_status_ok(cudaMallocHost((void**)&b->hcounter, 2 * sizeof(int32_t))));
  CK(cuda_status_ok(cudaMemcpy(b->rowptr, rowptr, (size_t)(rows + 1) * sizeof(int64_t),
                               cudaMemcpyHostToDevice)));
  CK(cuda_status_ok(cudaMemcpy(b->colidx, colidx, (size_t)nnz * sizeof(int32_t), cudaMemcpyHostToDevice)));
  CK(cuda_status_ok(cudaMemcpy(b->val, hval.data(), (size_t)nnz * sizeof(float), cudaMemcpyHostToDevice)));
  CK(cuda_status_ok(cudaMemcpy(b->X0, X0, (size_t)elems * sizeof(double), cudaMemcpyHostToDevice)));
  CK(cuda_status_ok(cudaMemcpy(b->prob, b->hprob.data(), (size_t)nprob * sizeof(BProb),
                               cudaMemcpyHostToDevice)));
  CK(cuda_status_ok(cudaMemcpy(b->order, order.data(), (size_t)nprob * sizeof(int32_t),
                               cudaMemcpyHostToDevice)));
  CK(cuda_status_ok(cudaMemset(b->Km, 0, (size_t)pp * sizeof(double))));
  {
    b->small_smem = sd_bytes(pmax);
    CK(cuda_status_ok(cudaFuncSetAttribute(b_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)b->small_smem)));
  }
  CK(set_tiles(b, 2048, 4, 2));
  CK(start(b));
  CK(cuda_status_ok(cudaStreamSynchronize(b->st)));
#undef CK
  *out = b;
  return GSI_OK;
fail:
  gsi_batched_destroy(b);
  return s;
}

gsi_status gsi_batched_set_tiles(gsi_batch* b, int32_t tile_max, int32_t ctas_per_sm,
                                 int32_t tiles_per_cta) {
  if (!b || tile_max < 32 || tile_max > 65536 || ctas_per_sm < 1 || ctas_per_sm > 32 ||
      tiles_per_cta < 1 || tiles_per_cta > 64)
    return GSI_ERR_ARG;
  GSI_TRY(set_tiles(b, tile_max, ctas_per_sm, tiles_per_cta));
  GSI_TRY(start(b));
  GSI_CUDA_TRY(cudaStreamSynchronize(b->st));
  return GSI_OK;
}

gsi_status gsi_batched_get_tiles(gsi_batch* b, int32_t* tile_max, int32_t* ctas_per_sm,
                                 int32_t* tiles_per_cta, int32_t* grid) {
  if (!b) return GSI_ERR_ARG;
  if (tile_max) *tile_max = b->tile_max;
  if (ctas_per_sm) *ctas_per_sm = b->ctas_per_sm;
  if (tiles_per_cta) *tiles_per_cta = b->tiles_per_cta;
  if (grid) *grid = b->grid;
  return GSI_OK;
}

gsi_status gsi_batched_last_plan(gsi_batch* b, int32_t* ntiles, int32_t* tile_prob,
                                 int32_t* tile_row0, int32_t* tile_rows, int32_t capacity) {
  if (!b || !ntiles) return GSI_ERR_ARG;
  int32_t nt = 0;
  GSI_CUDA_TRY(cudaStreamSynchronize(b->st));
  GSI_CUDA_TRY(cudaMemcpy(&nt, b->ntiles, sizeof(int32_t), cudaMemcpyDeviceToHost));
  *ntiles = nt;
  if (tile_prob || tile_row0 || tile_rows) {
    if (capacity < nt) return GSI_ERR_ARG;
    std::vector<BTile> ht(nt);
    GSI_CUDA_TRY(cudaMemcpy(ht.data(), b->tile, (size_t)nt * sizeof(BTile), cudaMemcpyDeviceToHost));
    for (int t = 0; t < nt; ++t) {
      if (tile_prob) tile_prob[t] = ht[t].prob;
      if (tile_row0) tile_row0[t] = ht[t].row0;
      if (tile_rows) tile_rows[t] = ht[t].rows;
    }
  }
  return GSI_OK;
}

gsi_status gsi_batched_reset(gsi_batch* b) {
  if (!b) return GSI_ERR_ARG;
  GSI_TRY(start(b));
  GSI_CUDA_TRY(cudaStreamSynchronize(b->st));
  return GSI_OK;
}

gsi_status gsi_batched_step(gsi_batch* b, int32_t npasses) {
  if (!b || npasses < 0) return GSI_ERR_ARG;
  for (int k = 0; k < npasses; ++k) GSI_TRY(launch_pass(b, b->st, 0));
  b->ritz_valid = false;
  GSI_TRY(read_state(b));
  return GSI_OK;
}

gsi_status gsi_batched_tune(gsi_batch* b, int32_t npasses, int32_t* tile_max, int32_t* ctas_per_sm,
                            int32_t* tiles_per_cta, double* ms_per_pass) {
  if (!b || npasses < 1) return GSI_ERR_ARG;
  static const int cand_rows[] = {256, 512, 1024, 2048, 4096};
  static const int cand_ctas[] = {2, 4, 8};
  static const int cand_tpc[] = {1, 2};
  cudaEvent_t e0, e1;
  GSI_CUDA_TRY(cudaEventCreate(&e0));
  GSI_CUDA_TRY(cudaEventCreate(&e1));
  double best = INFINITY;
  int br = b->tile_max, bc = b->ctas_per_sm, bt = b->tiles_per_cta;
  gsi_status s = GSI_OK;
  for (int tr : cand_rows) {
    for (int cc : cand_ctas) {
      for (int tc : cand_tpc) {
        s = set_tiles(b, tr, cc, tc);
        if (s == GSI_OK) s = start(b);
        if (s == GSI_OK) s = launch_pass(b, b->st, 0);  // warm-up pass
        if (s != GSI_OK) break;
        cudaEventRecord(e0, b->st);
        for (int k = 0; k < npasses && s == GSI_OK; ++k) s = launch_pass(b, b->st, 0);
        cudaEventRecord(e1, b->st);
        if (s != GSI_OK) break;
        cudaError_t ce = cudaEventSynchronize(e1);
        if (ce != cudaSuccess) {
          s = cuda_status(ce);
          break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double per = ms / npasses;
        if (per < best) {
          best = per;
          br = tr;
          bc = cc;
          bt = tc;
        }
      }
      if (s != GSI_OK) break;
    }
    if (s != GSI_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  GSI_TRY(s);
  GSI_TRY(set_tiles(b, br, bc, bt));
  GSI_TRY(start(b));
  GSI_CUDA_TRY(cudaStreamSynchronize(b->st));
  if (tile_max) *tile_max = br;
  if (ctas_per_sm) *ctas_per_sm = bc;
  if (tiles_per_cta) *tiles_per_cta = bt;
  if (ms_per_pass) *ms_per_pass = best;
  return GSI_OK;
}

gsi_status gsi_batched_solve(gsi_batch* b, int32_t use_graph, int32_t* passes) {
  if (!b) return GSI_ERR_ARG;
  const int bound = 2 * std::max(b->o.max_iters, 0) + 4;
  GSI_CUDA_TRY(cudaMemsetAsync(b->counter, 0, 3 * sizeof(int32_t), b->st));
  if (use_graph) {
    if (!b->gexec) GSI_TRY(build_graph(b));
    GSI_CUDA_TRY(cudaGraphLaunch(b->gexec, b->st));
    note_launch();
  } else {
    for (int k = 0; k < bound;) {
      for (int j = 0; j < 8 && k < bound; ++j, ++k) GSI_TRY(launch_pass(b, b->st, 0));
      GSI_CUDA_TRY(cudaMemcpyAsync(b->hcounter, b->counter, 2 * sizeof(int32_t),
                                   cudaMemcpyDeviceToHost, b->st));
      GSI_CUDA_TRY(cudaStreamSynchronize(b->st));
      if (b->hcounter[1] == 0) break;
    }
  }
  GSI_CUDA_TRY(cudaMemcpyAsync(b->hcounter, b->counter, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost,
                               b->st));
  GSI_TRY(read_state(b));
  b->ritz_valid = false;
  if (passes) *passes = b->hcounter[0];
  for (const BState& s : b->hstate)
    if (!s.converged) return GSI_ERR_NOCONV;
  return GSI_OK;
}

gsi_status gsi_batched_info(gsi_batch* b, int32_t i, gsi_info* info, int32_t* status) {
  if (!b || i < 0 || i >= b->nprob) return GSI_ERR_ARG;
  if ((int)b->hstate.size() != b->nprob) GSI_TRY(read_state(b));
  const BState& s = b->hstate[i];
  if (info) {
    info->iters = s.iters;
    info->matvecs = s.matvecs;
    info->restarts = s.restarts;
    info->brent_evals = s.evals;
    info->converged = s.converged;
    info->rel_residual = s.rel;
    info->rel_residual_inf = s.rel_inf;
    info->trace = (b->o.which == -1 ? -1.0 : 1.0) * s.trace;
    info->last_step = s.t;
  }
  if (status) *status = (s.flags & F_ACTIVE) ? -1 : s.status;
  return GSI_OK;
}

gsi_status gsi_batched_get_basis(gsi_batch* b, int32_t i, double* X, double* evals) {
  if (!b || i < 0 || i >= b->nprob) return GSI_ERR_ARG;
  const BProb& pr = b->hprob[i];
  const int64_t cnt = (int64_t)pr.n * pr.p;
  if (evals && !b->ritz_valid) {
    // Rayleigh-Ritz of every problem with an explicit AX: W = A X,
    // C' = X^T W, eig, W = X U (X itself is not changed)
    const BDev d = make_dev(b);
    const int g = b->grid, np = b->nprob;
    cudaStream_t s = b->st;
    b_mark_kernel<<<pgrid(np, 128), 128, 0, s>>>(d, 1, b->saved);
    GSI_LAUNCH_CHECK();
    b_plan_kernel<<<1, 1024, 0, s>>>(d, F_START);
    GSI_LAUNCH_CHECK();
    b_spmm_kernel<<<g, BT, 0, s>>>(d, F_START, 2);
    GSI_LAUNCH_CHECK();
    b_gram_kernel<1><<<g, BT, 0, s>>>(d, F_START, 2);
    GSI_LAUNCH_CHECK();
    b_reduce_kernel<<<rgrid(b, 1), 256, 0, s>>>(d, F_START, 1, 1, 1);
    GSI_LAUNCH_CHECK();
    b_small_kernel<<<np, BS, b->small_smem, s>>>(d, 2);
    GSI_LAUNCH_CHECK();
    b_retract_kernel<<<g, BT, 0, s>>>(d, 2);
    GSI_LAUNCH_CHECK();
    b_mark_kernel<<<pgrid(np, 128), 128, 0, s>>>(d, 0, b->saved);
    GSI_LAUNCH_CHECK();
    b->ritz_valid = true;
  }
  if (X) {
    const float2* src = (evals ? b->W : b->X) + pr.boff;
    double* tmp = nullptr;
    GSI_CUDA_TRY(cudaMallocAsync((void**)&tmp, (size_t)cnt * sizeof(double), b->st));
    gsi_status s = df_to_f64(cnt, src, tmp, b->st);
    if (s == GSI_OK)
      s = cuda_status_ok(cudaMemcpyAsync(X, tmp, (size_t)cnt * sizeof(double), cudaMemcpyDeviceToHost, b->st));
    cudaFreeAsync(tmp, b->st);
    GSI_TRY(s);
  }
  if (evals) {
    GSI_CUDA_TRY(cudaMemcpyAsync(evals, b->theta + pr.ppoff, (size_t)pr.p * sizeof(double),
                                 cudaMemcpyDeviceToHost, b->st));
  }
  GSI_CUDA_TRY(cudaStreamSynchronize(b->st));
  if (evals && b->o.which == -1)
    for (int k = 0; k < pr.p; ++k) evals[k] = -evals[k];
  return GSI_OK;
}

}  // extern "C"

extern "C" gsi_status gsi_batched_restart(gsi_batch* b, const double* X0, int32_t on_device) {
  if (!b || !X0) return GSI_ERR_ARG;
  GSI_CUDA_TRY(cudaMemcpyAsync(b->X0, X0, (size_t)b->elems * sizeof(double),
                               on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, b->st));
  GSI_TRY(start(b));
  GSI_CUDA_TRY(cudaStreamSynchronize(b->st));
  return GSI_OK;
}
