// Solver context and C entry points: Riemannian steepest descent (Alg. 2)
// and conjugate gradients (Alg. 4) with the exact line search of Alg. 3 and
// the one-matvec recursion of Eq. (save_matvec).
//
// One iteration (R = AX - XC is the residual, -grad phi; the step is
// X + tD with t >= 0):
//   C = X^T Y; R = Y - X C; stop if ||R||_F <= tol * anorm (explicit AX)
//   D = R (SD), or D = R + b (P - X K), K = X^T P, with the Polak-Ribiere b
//       (CG, restart to R when <D, R> <= 0 or every k_restart iterations)
//   W = A D
//   B = D^T D, Gam = D^T W, Z = D^T R (SD: Z = B), XX = X^T X
//   XD = X^T D = (I - XX)(C + b K)   (closed form, see below)
//   (t, M) from the p x p step; X <- (X + tD) M, Y <- (Y + tW) M
//   K_next = X_new^T D = M (XD + t B)  (CG, closed form)
// where M = S^{-1/2} with S = XX + t (XD + XD^T) + t^2 B, the Gram of X + tD,
// so that (X + tD) M is its polar factor (Eq. (Ynew)). S carries the measured
// departure of X from orthonormality (XX) and the tangency error it causes
// (XD), which keeps ||X^T X - I|| at rounding level.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <vector>

#include "blas_f64.cuh"
#include "df.cuh"
#include "oz.cuh"

namespace gsi {

static thread_local char g_last_error[256] = "";
static std::atomic<long long> g_launches{0};

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

void set_last_error(const char* msg) {
  snprintf(g_last_error, sizeof(g_last_error), "%s", msg);
}

gsi_status cuda_status(cudaError_t e) {
  set_last_error(cudaGetErrorString(e));
  if (e == cudaErrorMemoryAllocation) return GSI_ERR_OOM;
  return GSI_ERR_CUDA;
}

cudaError_t ensure_dyn_smem(const void* f, int bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, int> limit;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  int& cur = limit[{f, dev}];
  if (cur >= bytes) return cudaSuccess;
  e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}

int sm_count() {
  static int cached = 0;
  if (cached == 0) {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
      cached = v;
    else
      return 148;
  }
  return cached;
}

__global__ void scale_kernel(int64_t n, double s, double* x) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] *= s;
}

__global__ void symmetrize_kernel(int p, double* C) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= p * p) return;
  int i = e / p, j = e - i * p;
  if (i < j) {
    double v = 0.5 * (C[i * p + j] + C[j * p + i]);
    C[i * p + j] = v;
    C[j * p + i] = v;
  }
}

__global__ void csr_absmax_kernel(int64_t n, const int64_t* rowptr, const double* val,
                                  unsigned long long* out) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  double s = 0.0;
  for (int64_t k = rowptr[r]; k < rowptr[r + 1]; ++k) s += fabs(val[k]);
  // non-negative doubles order like their bit patterns
  atomicMax(out, (unsigned long long)__double_as_longlong(s));
}

}  // namespace gsi

using namespace gsi;

// Block element: float64 (precision GSI_PREC_F64) or df64 float2 (GSI_PREC_DF64);
// both are 8 bytes, so every n x p buffer has the same size in both modes.
struct gsi_ctx {
  cudaStream_t st = nullptr;
  int64_t n = 0, nnz = 0;
  int p = 0;
  gsi_opts o{};
  bool emu = true;
  bool mixed = false;  // GSI_PREC_MIXED: 3-digit operator apply until mixed_switch
  int nd = 7;          // digits per operand in the dense operator apply
  int fmt = GSI_CSR;
  double* Ad = nullptr;   // dense A, float64 (GSI_DENSE)
  float2* Adf = nullptr;  // dense A, df64
  float2* dense_ws = nullptr;
  int64_t* rowptr = nullptr;
  int32_t* colidx = nullptr;
  double* val = nullptr;    // float64 values (native mode and Rayleigh-Ritz)
  float2* vdf = nullptr;    // df64 values
  float2* dia_val = nullptr;  // stencil-shaped A: df64 values by row and diagonal
  DiaArgs dia{};              // its diagonals and shared-memory window
  bool use_dia = false;
  int C = 32;
  int64_t nchunks = 0;
  int64_t* perm = nullptr;
  int64_t* chunk_ptr = nullptr;
  int64_t* chunk_len = nullptr;
  int32_t* scol = nullptr;
  double* sval = nullptr;
  float2* sdf = nullptr;
  double anorm = 0.0;
  double sign = 1.0;
  void *X = nullptr, *Y = nullptr, *R = nullptr, *Rp = nullptr, *D = nullptr, *P = nullptr,
       *W = nullptr, *Xn = nullptr, *Yn = nullptr;
  double* pp = nullptr;  // p x p matrices
  double *Cm, *Bm, *Gm, *Zm, *XXm, *XDm, *Km, *Mm, *Gm2, *out, *dout;
  double *Tm, *Fm;  // p x p scratch of gsi_get_basis, which no iteration reads
  double* gram_ws = nullptr;
  float2* oz_gram_ws = nullptr;
  void* oz_rhs_ws = nullptr;
  float2* oz_parts = nullptr;
  float* oz_rinf = nullptr;  // per-block row-norm maxima of a fused residual product
  bool rinf_fused = false;   // the last block product also left max_r sum_j |R[r,j]| in dout[2]
  double* dots_ws = nullptr;
  double* small_ws = nullptr;
  // the eigenbasis of D^T D runs on a second stream while the other
  // line-search Grams run on st (one SM left to it); V and the diagonal pass
  // through eig_ws
  cudaStream_t st2 = nullptr;
  cudaEvent_t ev_b = nullptr, ev_e = nullptr;
  void* eig_ws = nullptr;
  int gram_reserve = 0;  // SMs the next Grams leave free
  double* host = nullptr;  // pinned readback buffer
  // LOBCG comparator: p x p workspace, masks of the kept columns of the
  // second and third basis blocks, and the eigensolver's scratch for 3p x 3p
  double* lob = nullptr;
  int* lob_mask = nullptr;
  double* lob_ws = nullptr;
  int* tmo = nullptr;      // pinned copy of the tensor-core kernels' timeout count
  int tmo_seen = 0;        // that count when this context last looked
  std::vector<void*> allocs;
  // iteration state
  int iters = 0, matvecs = 0, restarts = 0, last_evals = 0;
  bool y_fresh = true, have_prev = false, converged = false;
  double rr_prev = 0.0, res0_inf = -1.0, last_t = 0.0, rel = NAN, rel_inf = NAN;
  int64_t herm_n = 0;  // > 0: the realification of a complex Hermitian problem of this size
  // per-class timing (CUDA events on the context's stream)
  bool prof = false;
  struct Cls {
    long long launches = 0;
    double ms = 0.0, bytes = 0.0, flops = 0.0;
  } cls[GSI_K_COUNT];
  std::vector<cudaEvent_t> pool;
  struct Pending {
    int k;
    cudaEvent_t a, b;
  };
  std::vector<Pending> pending;
  cudaEvent_t cur = nullptr;
};

namespace {

gsi_status dev_alloc(gsi_ctx* c, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 16));
  if (e != cudaSuccess) return cuda_status(e);
  c->allocs.push_back(*p);
  return GSI_OK;
}

cudaEvent_t pool_get(gsi_ctx* c) {
  if (c->pool.empty()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
  }
  cudaEvent_t e = c->pool.back();
  c->pool.pop_back();
  return e;
}

void prof_begin(gsi_ctx* c) {
  if (!c->prof) return;
  c->cur = pool_get(c);
  cudaEventRecord(c->cur, c->st);
}

void prof_end(gsi_ctx* c, int k, double bytes, double flops) {
  if (!c->prof || !c->cur) return;
  cudaEvent_t e = pool_get(c);
  cudaEventRecord(e, c->st);
  c->pending.push_back({k, c->cur, e});
  c->cur = nullptr;
  c->cls[k].launches++;
  c->cls[k].bytes += bytes;
  c->cls[k].flops += flops;
}

// after a stream synchronisation: fold finished event pairs into the totals
void prof_harvest(gsi_ctx* c) {
  for (auto& pe : c->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, pe.a, pe.b) == cudaSuccess) c->cls[pe.k].ms += ms;
    c->pool.push_back(pe.a);
    c->pool.push_back(pe.b);
  }
  c->pending.clear();
}

// After a call's kernels: GSI_ERR_TIMEOUT if a bounded device wait of a
// tensor-core kernel ran out since the last look (such a kernel drains the
// tensor core, leaves non-finite outputs and counts the event), else s.
gsi_status timeout_check(gsi_ctx* c, gsi_status s) {
  if (!c->tmo) return s;
  if (oz_timeouts_async(c->tmo, c->st) != GSI_OK || cudaStreamSynchronize(c->st) != cudaSuccess) return s;
  if (*c->tmo != c->tmo_seen) {
    c->tmo_seen = *c->tmo;
    set_last_error("a bounded wait of a tensor-core kernel ran out");
    return GSI_ERR_TIMEOUT;
  }
  return s;
}

gsi_status readback(gsi_ctx* c, const double* src, int count) {
  GSI_CUDA_TRY(cudaMemcpyAsync(c->host, src, count * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  GSI_CUDA_TRY(cudaStreamSynchronize(c->st));
  prof_harvest(c);
  return GSI_OK;
}

double blk_bytes(gsi_ctx* c) { return 8.0 * (double)c->n * c->p; }

// ---- block operations, float64 or df64 ------------------------------------

// accurate: an explicit Y = A X (always 7-digit); otherwise the direction's
// apply W = A D, which the mixed mode computes with c->nd digits
gsi_status op_matvec(gsi_ctx* c, const void* in, void* outp, bool accurate = true) {
  c->matvecs++;
  prof_begin(c);
  gsi_status s;
  double bytes;
  if (c->fmt == GSI_DENSE) {
    bytes = 8.0 * (double)c->n * c->n + 2 * blk_bytes(c);
    s = c->emu ? oz_gram(c->n, (int)c->n, c->p, c->Adf, (const float2*)in, false, nullptr, c->dense_ws,
                         c->st, accurate ? 7 : c->nd, (float2*)outp)
               : dense_gemm(c->n, c->p, c->Ad, (const double*)in, (double*)outp, c->st);
    prof_end(c, GSI_K_SPMM, bytes, 2.0 * (double)c->n * c->n * c->p);
    return s;
  }
  if (c->fmt == GSI_SELL) {
    int64_t slots = c->nchunks * c->C;
    bytes = 12.0 * (double)c->nnz + 8.0 * slots + 2 * blk_bytes(c);
    s = c->emu ? df_spmm_sell(c->nchunks, c->C, c->perm, c->chunk_ptr, c->chunk_len, c->scol,
                              c->sdf, c->p, (const float2*)in, (float2*)outp, c->st)
               : spmm_sell(c->n, c->nchunks, c->C, c->perm, c->chunk_ptr, c->chunk_len, c->scol,
                           c->sval, c->p, (const double*)in, (double*)outp, c->st);
  } else if (c->use_dia && ((uintptr_t)in & 15) == 0 && ((uintptr_t)outp & 15) == 0) {
    bytes = 8.0 * (double)c->dia.nd * c->n + 2 * blk_bytes(c);
    DiaArgs a = c->dia;
    a.X = (const float2*)in;
    a.W = (float2*)outp;
    s = df_spmm_dia(a, c->st);
  } else {
    bytes = 12.0 * (double)c->nnz + 8.0 * (c->n + 1) + 2 * blk_bytes(c);
    s = c->emu ? df_spmm_csr(c->n, c->rowptr, c->colidx, c->vdf, c->p, (const float2*)in,
                             (float2*)outp, c->st)
               : spmm_csr(c->n, c->rowptr, c->colidx, c->val, c->p, (const double*)in,
                          (double*)outp, c->st);
  }
  prof_end(c, GSI_K_SPMM, bytes, 2.0 * c->nnz * c->p);
  return s;
}

gsi_status op_gram(gsi_ctx* c, const void* U, const void* V, bool sym, double* G) {
  prof_begin(c);
  gsi_status s;
  if (c->emu) {
    s = oz_gram(c->n, c->p, c->p, (const float2*)U, (const float2*)V, sym && U == V, G,
                c->oz_gram_ws, c->st, 7, nullptr, c->gram_reserve);
    if (s == GSI_OK && sym && U != V) {
      symmetrize_kernel<<<ceil_div(c->p * c->p, 256), 256, 0, c->st>>>(c->p, G);
      note_launch();
    }
  } else {
    s = gram(c->n, c->p, c->p, (const double*)U, (const double*)V, G, c->gram_ws, c->st);
    if (s == GSI_OK && sym) {
      symmetrize_kernel<<<ceil_div(c->p * c->p, 256), 256, 0, c->st>>>(c->p, G);
      note_launch();
    }
  }
  prof_end(c, GSI_K_GRAM, (U == V ? 1 : 2) * blk_bytes(c), 2.0 * c->n * c->p * c->p);
  return s;
}

// out = s0 U0 M0 (+ s1 U1 M1) + c0 E0 (+ c1 E1); optional dots (emu: fused;
// f64: separate pass) <out,out> -> dout[0], <out,dw> -> dout[1].
// row_inf: also max_r sum_j |out[r, j]| -> dout[2] where the product can form
// it (sets c->rinf_fused).
gsi_status op_blockmul(gsi_ctx* c, int nk, const void* U0, const double* M0, double s0,
                       const void* U1, const double* M1, double s1, int ne, const void* E0,
                       double c0, const void* E1, double c1, void* outp, bool dot_self,
                       const void* dw, bool row_inf = false) {
  prof_begin(c);
  gsi_status s;
  const bool want = dot_self || dw;
  c->rinf_fused = false;
  if (c->emu) {
    const float2* U[2] = {(const float2*)U0, (const float2*)(U1 ? U1 : U0)};
    const double* M[2] = {M0, M1 ? M1 : M0};
    double sc[2] = {s0, s1};
    const float2* E[2] = {(const float2*)E0, (const float2*)E1};
    float2 ce[2] = {df_from_double(c0), df_from_double(c1)};
    int np = 0;
    bool fused = false;
    s = oz_gemm(c->n, c->p, nk, U, M, sc, ne, E, ce, (float2*)outp, want ? c->oz_parts : nullptr,
                (const float2*)dw, dot_self, c->oz_rhs_ws, c->st, &np, 7,
                want && row_inf ? c->oz_rinf : nullptr, &fused);
    if (s == GSI_OK && want) s = df_sum_parts(np, c->oz_parts, c->dout, c->st, fused ? c->oz_rinf : nullptr);
    c->rinf_fused = s == GSI_OK && fused;
  } else {
    RowMulArgs a{};
    a.nk = nk;
    a.U[0] = (const double*)U0;
    a.M[0] = M0;
    a.s[0] = s0;
    a.U[1] = (const double*)U1;
    a.M[1] = M1;
    a.s[1] = s1;
    a.ne = ne;
    a.E[0] = (const double*)E0;
    a.c[0] = c0;
    a.E[1] = (const double*)E1;
    a.c[1] = c1;
    s = rowmul(c->n, c->p, a, (double*)outp, c->st);
    if (s == GSI_OK && want)
      s = dots(c->n, c->p, 2, (const double*)outp, (const double*)outp, (const double*)outp,
               (const double*)(dw ? dw : outp), nullptr, c->dout, c->dots_ws, c->st);
  }
  prof_end(c, GSI_K_BLOCKMUL, (nk + ne + 1) * blk_bytes(c), 2.0 * c->n * c->p * (double)nk * c->p);
  return s;
}

// max_r sum_j |R[r, j]| -> dout[2]
gsi_status op_rowinf(gsi_ctx* c, const void* Rb) {
  prof_begin(c);
  gsi_status s;
  if (c->emu)
    s = df_dots(c->n, c->p, nullptr, nullptr, nullptr, nullptr, (const float2*)Rb, c->dout,
                (float2*)c->dots_ws, c->st);
  else
    s = dots(c->n, c->p, 0, nullptr, nullptr, nullptr, nullptr, (const double*)Rb, c->dout,
             c->dots_ws, c->st);
  prof_end(c, GSI_K_REDUCE, blk_bytes(c), 0.0);
  return s;
}

gsi_status op_small(gsi_ctx* c, int mode, const double* B, const double* Zp) {
  prof_begin(c);
  gsi_status s = c->emu ? small_step_df(mode, c->p, c->Cm, B, c->Gm, Zp, c->XXm, c->XDm, c->Mm,
                                        c->out, c->small_ws, c->st, c->eig_ws)
                        : small_step(mode, c->p, c->Cm, B, c->Gm, Zp, c->XXm, c->XDm, c->Mm, c->out,
                                     c->small_ws, c->st);
  prof_end(c, GSI_K_SMALL, 0.0, 0.0);
  return s;
}

// X <- X M (M = (X^T X)^{-1/2}), twice
gsi_status orthonormalize(gsi_ctx* c) {
  for (int pass = 0; pass < 2; ++pass) {
    GSI_TRY(op_gram(c, c->X, c->X, true, c->Bm));
    GSI_TRY(op_small(c, 1, c->Bm, c->Bm));
    GSI_TRY(readback(c, c->out, 5));
    if (c->host[3] != 0.0) return GSI_ERR_BREAKDOWN;
    GSI_TRY(op_blockmul(c, 1, c->X, c->Mm, 1.0, nullptr, nullptr, 0.0, 0, nullptr, 0.0, nullptr,
                        0.0, c->Xn, false, nullptr));
    std::swap(c->X, c->Xn);
  }
  return GSI_OK;
}

// The stopped-on quantity: ||R||_F / anorm, or (stop_rule 1) the paper's
// table criterion ||R||_inf / ||R_0||_inf.
double crit(const gsi_ctx* c) { return c->o.stop_rule == 1 ? c->rel_inf : c->rel; }

// One iteration; returns GSI_OK and sets *stop when the stopping test holds.
gsi_status iterate(gsi_ctx* c, bool* stop) {
  const bool cg = c->o.method == GSI_CG;
  *stop = false;
  double rr = 0.0, rp = 0.0, rinf = 0.0;
  for (;;) {
    GSI_TRY(op_gram(c, c->X, c->Y, true, c->Cm));  // C = X^T A X, symmetric
    const bool want_rp = cg && c->have_prev;
    // R = Y - X C with <R,R>, <R,R_prev> and (where the product forms it)
    // max_r sum_j |R[r,j]|
    GSI_TRY(op_blockmul(c, 1, c->X, c->Cm, -1.0, nullptr, nullptr, 0.0, 1, c->Y, 1.0, nullptr, 0.0,
                        c->R, true, want_rp ? c->Rp : nullptr, true));
    const bool rinf_fused = c->rinf_fused;
    GSI_TRY(readback(c, c->dout, rinf_fused ? 3 : 2));
    rr = c->host[0];
    rp = want_rp ? c->host[1] : 0.0;
    if (rinf_fused) {
      rinf = c->host[2];
    } else {
      GSI_TRY(op_rowinf(c, c->R));
      GSI_TRY(readback(c, c->dout + 2, 1));
      rinf = c->host[0];
    }
    if (!isfinite(rr)) return GSI_ERR_NONFINITE;
    if (c->res0_inf < 0.0) c->res0_inf = rinf;
    c->rel = sqrt(rr) / c->anorm;
    c->rel_inf = c->res0_inf > 0.0 ? rinf / c->res0_inf : 0.0;
    if (c->mixed && c->nd != 7 && (c->rel <= c->o.mixed_switch || c->rel <= c->o.tol)) {
      // correction phase: 7-digit products from here on, with an explicit AX
      // and a fresh (gradient) direction
      c->nd = 7;
      GSI_TRY(op_matvec(c, c->X, c->Y));
      c->y_fresh = true;
      c->have_prev = false;
      continue;
    }
    if (crit(c) <= c->o.tol || c->iters >= c->o.max_iters) {
      if (!c->y_fresh) {  // the final residual is always taken with an explicit AX
        GSI_TRY(op_matvec(c, c->X, c->Y));
        c->y_fresh = true;
        continue;
      }
      c->converged = crit(c) <= c->o.tol;
      *stop = true;
      return GSI_OK;
    }
    break;
  }
  // search direction
  const void* Dp = c->R;
  bool restarted = false;
  double beta_used = 0.0;
  if (cg) {
    if (c->have_prev) {
      double b = (rr - rp) / c->rr_prev;
      // K = X^T P was carried over from the previous step in closed form
      // D = R + b P - X (b K), with <D, R>
      GSI_TRY(op_blockmul(c, 1, c->X, c->Km, -b, nullptr, nullptr, 0.0, 2, c->R, 1.0, c->P, b,
                          c->D, false, c->R));
      GSI_TRY(readback(c, c->dout + 1, 1));
      bool due = c->o.k_restart > 0 && c->iters % c->o.k_restart == 0;
      if (due || !(c->host[0] > 0.0)) restarted = true;
    }
    if (!c->have_prev || restarted) {
      GSI_CUDA_TRY(cudaMemcpyAsync(c->D, c->R, (size_t)blk_bytes(c), cudaMemcpyDeviceToDevice, c->st));
    }
    if (restarted) c->restarts++;
    Dp = c->D;
    beta_used = (c->have_prev && !restarted) ? (rr - rp) / c->rr_prev : 0.0;
  }
  GSI_TRY(op_matvec(c, Dp, c->W, false));
  GSI_TRY(op_gram(c, Dp, Dp, true, c->Bm));
  // the eigenbasis of B = D^T D on the second stream, alongside the Grams below
  const bool split = c->st2 != nullptr;
  if (split) {
    GSI_CUDA_TRY(cudaEventRecord(c->ev_b, c->st));
    GSI_CUDA_TRY(cudaStreamWaitEvent(c->st2, c->ev_b, 0));
    GSI_TRY(small_step_df(3, c->p, nullptr, c->Bm, nullptr, nullptr, nullptr, nullptr, nullptr, c->out,
                          c->small_ws, c->st2, c->eig_ws));
    GSI_CUDA_TRY(cudaEventRecord(c->ev_e, c->st2));
    c->gram_reserve = 1;
  }
  gsi_status gs = op_gram(c, Dp, c->W, true, c->Gm);
  const double* Zp = c->Bm;
  if (gs == GSI_OK && cg) {
    gs = op_gram(c, Dp, c->R, false, c->Zm);
    Zp = c->Zm;
  }
  if (gs == GSI_OK) gs = op_gram(c, c->X, c->X, true, c->XXm);
  c->gram_reserve = 0;
  if (split) GSI_CUDA_TRY(cudaStreamWaitEvent(c->st, c->ev_e, 0));
  GSI_TRY(gs);
  // X^T D in closed form from the measured X^T X: X^T R = (I - X^T X) C and
  // X^T P = K give X^T D = (I - X^T X)(C + b K) (b = 0 for SD and restarts)
  prof_begin(c);
  GSI_TRY(pp_axpby(c->p, 1.0, c->Cm, beta_used, beta_used != 0.0 ? c->Km : nullptr, c->Gm2, c->st));
  GSI_TRY(pp_gemm(c->p, -1.0, c->XXm, c->Gm2, 1.0, c->Gm2, c->XDm, c->st));
  prof_end(c, GSI_K_SMALL, 0.0, 0.0);
  GSI_TRY(op_small(c, split ? 4 : 0, c->Bm, Zp));
  GSI_TRY(readback(c, c->out, 5));
  const double t = c->host[0];
  c->last_t = t;
  c->last_evals = (int)c->host[2];
  if (c->host[3] != 0.0) return GSI_ERR_BREAKDOWN;
  if (!isfinite(t)) return GSI_ERR_NONFINITE;
  const double bmax = c->host[4];
  if (cg) {
    // next step's K = X_new^T D = M (X^T D + t D^T D)
    prof_begin(c);
    GSI_TRY(pp_axpby(c->p, 1.0, c->XDm, t, c->Bm, c->Gm2, c->st));
    GSI_TRY(pp_gemm(c->p, 1.0, c->Mm, c->Gm2, 0.0, nullptr, c->Km, c->st));
    prof_end(c, GSI_K_SMALL, 0.0, 0.0);
  }
  bool recompute = c->o.explicit_ax || t * sqrt(std::max(bmax, 0.0)) < 1e3 * 2.220446049250313e-16 ||
                   (c->o.recompute_every > 0 && (c->iters + 1) % c->o.recompute_every == 0);
  // X <- (X + tD) M, Y <- (Y + tW) M (Eq. (save_matvec)) or Y <- A X
  GSI_TRY(op_blockmul(c, 2, c->X, c->Mm, 1.0, Dp, c->Mm, t, 0, nullptr, 0.0, nullptr, 0.0, c->Xn,
                      false, nullptr));
  std::swap(c->X, c->Xn);
  if (recompute) {
    GSI_TRY(op_matvec(c, c->X, c->Y));
  } else {
    GSI_TRY(op_blockmul(c, 2, c->Y, c->Mm, 1.0, c->W, c->Mm, t, 0, nullptr, 0.0, nullptr, 0.0,
                        c->Yn, false, nullptr));
    std::swap(c->Y, c->Yn);
  }
  c->y_fresh = recompute;
  c->iters++;
  if (cg) {
    std::swap(c->D, c->P);
    std::swap(c->R, c->Rp);
  }
  c->rr_prev = rr;
  c->have_prev = true;
  return GSI_OK;
}

__global__ void diag_kernel(int p, const double* d, double* D) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= p * p) return;
  int i = e / p, j = e - i * p;
  D[e] = (i == j) ? d[i] : 0.0;
}

// out = a W + b Z + e Zp in the context's block type
gsi_status op_combine3(gsi_ctx* c, double a, const void* W, double b, const void* Z, double e,
                       const void* Zp, void* outp) {
  prof_begin(c);
  gsi_status s;
  const int64_t cnt = c->n * c->p;
  if (c->emu)
    s = df_combine3(cnt, df_from_double(a), (const float2*)W, df_from_double(b), (const float2*)Z,
                    df_from_double(e), (const float2*)Zp, (float2*)outp, c->st);
  else
    s = combine3(cnt, a, (const double*)W, b, (const double*)Z, e, (const double*)Zp, (double*)outp,
                 c->st);
  prof_end(c, GSI_K_REDUCE, (Zp ? 4 : 3) * blk_bytes(c), 0.0);
  return s;
}

// One iteration of Chebyshev-filtered subspace iteration (Alg. 1 with the
// filter C_d((t - c)/h) / C_d((lambda_1 - c)/h) of Eq. (optimal_poly)):
// Rayleigh-Ritz on span(X), residual test, Z = p_d(A) X by the three-term
// recurrence (sigma_{k+1} = 1/(2e - sigma_k), e = (lambda_1 - c)/h), then an
// orthonormal basis of span(Z).
gsi_status iterate_cheb(gsi_ctx* c, bool* stop) {
  const int p = c->p;
  *stop = false;
  // Rayleigh-Ritz with the fresh Y = A X
  GSI_TRY(op_gram(c, c->X, c->Y, true, c->Cm));
  prof_begin(c);
  if (c->emu) {
    GSI_TRY(small_step_df(2, p, nullptr, c->Cm, nullptr, nullptr, nullptr, c->XDm, c->Bm, c->out,
                          c->small_ws, c->st));
  } else {
    GSI_TRY(small_eig(p, c->Cm, c->XDm, c->Bm, c->small_ws, c->st));
  }
  diag_kernel<<<ceil_div(p * p, 256), 256, 0, c->st>>>(p, c->XDm, c->Gm);
  note_launch();
  prof_end(c, GSI_K_SMALL, 0.0, 0.0);
  GSI_TRY(op_blockmul(c, 1, c->X, c->Bm, 1.0, nullptr, nullptr, 0.0, 0, nullptr, 0.0, nullptr, 0.0,
                      c->Xn, false, nullptr));
  std::swap(c->X, c->Xn);
  GSI_TRY(op_blockmul(c, 1, c->Y, c->Bm, 1.0, nullptr, nullptr, 0.0, 0, nullptr, 0.0, nullptr, 0.0,
                      c->Yn, false, nullptr));
  std::swap(c->Y, c->Yn);
  // R = Y - X diag(theta), ||R||_F
  GSI_TRY(op_blockmul(c, 1, c->X, c->Gm, -1.0, nullptr, nullptr, 0.0, 1, c->Y, 1.0, nullptr, 0.0,
                      c->R, true, nullptr));
  GSI_TRY(readback(c, c->dout, 1));
  const double rr = c->host[0];
  GSI_TRY(op_rowinf(c, c->R));
  GSI_TRY(readback(c, c->dout + 2, 1));
  const double rinf = c->host[0];
  if (!isfinite(rr)) return GSI_ERR_NONFINITE;
  if (c->res0_inf < 0.0) c->res0_inf = rinf;
  c->rel = sqrt(rr) / c->anorm;
  if (c->o.cheb_guard > 0) {
    // guard vectors: only the p - guard largest Ritz pairs enter the test,
    // from the diagonal of R^T R (column norms) and theta
    GSI_TRY(op_gram(c, c->R, c->R, true, c->Fm));
    GSI_TRY(readback(c, c->Fm, p * p));
    std::vector<double> cn(p);
    for (int i = 0; i < p; ++i) cn[i] = c->host[i * p + i];
    GSI_TRY(readback(c, c->XDm, p));
    std::vector<int> ord(p);
    for (int i = 0; i < p; ++i) ord[i] = i;
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return c->host[a] > c->host[b]; });
    double rw = 0.0;
    for (int i = 0; i < p - c->o.cheb_guard; ++i) rw += cn[ord[i]];
    c->rel = sqrt(rw) / c->anorm;
  }
  c->rel_inf = c->res0_inf > 0.0 ? rinf / c->res0_inf : 0.0;
  // the Ritz basis is kept in C for fill_info: C <- diag(theta)
  GSI_CUDA_TRY(cudaMemcpyAsync(c->Cm, c->Gm, (size_t)p * p * sizeof(double),
                               cudaMemcpyDeviceToDevice, c->st));
  if (crit(c) <= c->o.tol || c->iters >= c->o.max_iters) {
    c->converged = crit(c) <= c->o.tol;
    *stop = true;
    return GSI_OK;
  }
  // filter: Z_1 = (sigma_1 / h)(A - cI) X, Z_{k+1} = (2 sigma_{k+1} / h)(A - cI) Z_k - sigma_k sigma_{k+1} Z_{k-1}
  double lo = c->o.cheb_lo, hi = c->o.cheb_hi, scale = c->o.cheb_scale;
  if (c->o.cheb_adaptive) {
    // Ritz-based bounds: the unwanted interval [cheb_lo, theta_min], scaled at
    // theta_max (the Ritz values of this step's Rayleigh-Ritz, in XDm)
    GSI_TRY(readback(c, c->XDm, p));
    hi = INFINITY;
    scale = -INFINITY;
    for (int i = 0; i < p; ++i) {
      hi = std::min(hi, c->host[i]);
      scale = std::max(scale, c->host[i]);
    }
    if (!(hi > lo)) return GSI_ERR_ARG;
  }
  const double cc = 0.5 * (hi + lo), hh = 0.5 * (hi - lo);
  const double e = (scale - cc) / hh;
  double sigma = 1.0 / e;
  void* bufs[4] = {c->X, c->D, c->P, c->R};
  int ip = 0, ic = 1;
  GSI_TRY(op_matvec(c, bufs[ip], c->W));
  GSI_TRY(op_combine3(c, sigma / hh, c->W, -cc * sigma / hh, bufs[ip], 0.0, nullptr, bufs[ic]));
  for (int k = 1; k < c->o.cheb_degree; ++k) {
    const double sn = 1.0 / (2.0 * e - sigma);
    int nb = 0;  // a buffer holding neither Z_{k-1} nor Z_k
    while (nb == ip || nb == ic) ++nb;
    GSI_TRY(op_matvec(c, bufs[ic], c->W));
    GSI_TRY(op_combine3(c, 2.0 * sn / hh, c->W, -2.0 * sn * cc / hh, bufs[ic], -sigma * sn, bufs[ip],
                        bufs[nb]));
    ip = ic;
    ic = nb;
    sigma = sn;
  }
  // the filtered block becomes X (buffers are only re-labelled)
  c->X = bufs[ic];
  c->D = bufs[(ic + 1) % 4];
  c->P = bufs[(ic + 2) % 4];
  c->R = bufs[(ic + 3) % 4];
  GSI_TRY(orthonormalize(c));
  GSI_TRY(op_matvec(c, c->X, c->Y));
  c->y_fresh = true;
  c->iters++;
  return GSI_OK;
}

// ---- LOBCG comparator (Sec. 6.4, "Comparison to LOBCG") ------------------

constexpr double LOBCG_RANK_TOL = 1e-7;  // kept singular values, relative to a block's largest

// p x p slots of the LOBCG workspace
struct LobWs {
  double *K1, *K2, *S, *U, *M2, *M3, *H12, *H13, *H22, *H23, *H33, *V1, *V2, *V3, *H, *th;
};
LobWs lob_ws(gsi_ctx* c) {
  const size_t q = (size_t)c->p * c->p;
  double* L = c->lob;
  return {L, L + q, L + 2 * q, L + 3 * q, L + 12 * q, L + 13 * q, L + 14 * q, L + 15 * q, L + 16 * q,
          L + 17 * q, L + 18 * q, L + 19 * q, L + 20 * q, L + 21 * q, L + 22 * q, L + 31 * q};
}
size_t lob_doubles(int p) { return (size_t)31 * p * p + 3 * (size_t)p + 64; }

// One basis block of V_k in place of *B: projected off Q1 (and Q2) twice;
// from the eigendecomposition of its Gram B^T B = U diag(th) U^T,
// B U_r diag(th_r)^(-1/2) over th_i > tol^2 th_0 (dropped columns zero,
// mask 0); then Q <- Q (Q^T Q)^(-1/2) on the kept columns.
gsi_status lob_block(gsi_ctx* c, void** B, const void* Q1, const void* Q2, double* M, int* mask) {
  const int p = c->p;
  LobWs w = lob_ws(c);
  for (int pass = 0; pass < 2; ++pass) {
    GSI_TRY(op_gram(c, Q1, *B, false, w.K1));
    if (Q2) GSI_TRY(op_gram(c, Q2, *B, false, w.K2));
    GSI_TRY(op_blockmul(c, Q2 ? 2 : 1, Q1, w.K1, -1.0, Q2, Q2 ? w.K2 : nullptr, -1.0, 1, *B, 1.0, nullptr, 0.0,
                        *B, false, nullptr));
  }
  GSI_TRY(op_gram(c, *B, *B, true, w.S));
  prof_begin(c);
  GSI_TRY(small_eig(p, w.S, w.th, w.U, c->lob_ws, c->st));
  GSI_TRY(lobcg_coef(p, w.th, w.U, LOBCG_RANK_TOL * LOBCG_RANK_TOL, M, mask, c->st));
  prof_end(c, GSI_K_SMALL, 0.0, 0.0);
  GSI_TRY(op_blockmul(c, 1, *B, M, 1.0, nullptr, nullptr, 0.0, 0, nullptr, 0.0, nullptr, 0.0, c->Yn, false,
                      nullptr));
  std::swap(*B, c->Yn);
  GSI_TRY(op_gram(c, *B, *B, true, w.S));
  prof_begin(c);
  GSI_TRY(lobcg_mask_gram(p, w.S, mask, c->st));
  prof_end(c, GSI_K_SMALL, 0.0, 0.0);
  GSI_TRY(op_small(c, 1, w.S, w.S));  // Mm = S^(-1/2)
  GSI_TRY(readback(c, c->out, 5));
  if (c->host[3] != 0.0) return GSI_ERR_BREAKDOWN;
  GSI_TRY(op_blockmul(c, 1, *B, c->Mm, 1.0, nullptr, nullptr, 0.0, 0, nullptr, 0.0, nullptr, 0.0, c->Yn, false,
                      nullptr));
  std::swap(*B, c->Yn);
  return GSI_OK;
}

// One LOBCG iteration (the comparator of Sec. 6.4, in its LOBCG(+) form):
// the Rayleigh-Ritz procedure on V_k = span(X_k, G_k, P_k) (Eq.
// (def_Vk_LOBPCG)), G_k = A X_k - X_k C_k and P_k the part of X_k outside
// span(X_{k-1}) (Knyazev's block, which the paper's footnote puts in place of
// X_{k-1}; same V_k). Buffers: Q1 = X (AQ1 = Y, explicit every iteration),
// Q2 in R (AQ2 in W), Q3 in D (AQ3 in Rp), P in P. Q^T A Q is formed from
// its six p x p blocks (explicit products with A Q, the paper's LOBCG(+));
// its top p eigenvectors give X_{k+1} = Q1 V1 + Q2 V2 + Q3 V3 and
// P_{k+1} = Q2 V2 + Q3 V3.
gsi_status iterate_lobcg(gsi_ctx* c, bool* stop) {
  const int p = c->p;
  *stop = false;
  LobWs w = lob_ws(c);
  GSI_TRY(op_gram(c, c->X, c->Y, true, c->Cm));
  GSI_TRY(op_blockmul(c, 1, c->X, c->Cm, -1.0, nullptr, nullptr, 0.0, 1, c->Y, 1.0, nullptr, 0.0, c->R, true,
                      nullptr, true));
  const bool rinf_fused = c->rinf_fused;
  GSI_TRY(readback(c, c->dout, rinf_fused ? 3 : 2));
  const double rr = c->host[0];
  double rinf = rinf_fused ? c->host[2] : 0.0;
  if (!rinf_fused) {
    GSI_TRY(op_rowinf(c, c->R));
    GSI_TRY(readback(c, c->dout + 2, 1));
    rinf = c->host[0];
  }
  if (!isfinite(rr)) return GSI_ERR_NONFINITE;
  if (c->res0_inf < 0.0) c->res0_inf = rinf;
  c->rel = sqrt(rr) / c->anorm;
  c->rel_inf = c->res0_inf > 0.0 ? rinf / c->res0_inf : 0.0;
  if (crit(c) <= c->o.tol || c->iters >= c->o.max_iters) {
    c->converged = crit(c) <= c->o.tol;
    *stop = true;
    return GSI_OK;
  }
  const bool prev = c->have_prev;
  GSI_TRY(lob_block(c, &c->R, c->X, nullptr, w.M2, c->lob_mask));
  GSI_TRY(op_matvec(c, c->R, c->W));
  if (prev) {
    GSI_CUDA_TRY(cudaMemcpyAsync(c->D, c->P, (size_t)blk_bytes(c), cudaMemcpyDeviceToDevice, c->st));
    GSI_TRY(lob_block(c, &c->D, c->X, c->R, w.M3, c->lob_mask + p));
    GSI_TRY(op_matvec(c, c->D, c->Rp));
  }
  GSI_TRY(op_gram(c, c->X, c->W, false, w.H12));
  GSI_TRY(op_gram(c, c->R, c->W, true, w.H22));
  if (prev) {
    GSI_TRY(op_gram(c, c->X, c->Rp, false, w.H13));
    GSI_TRY(op_gram(c, c->R, c->Rp, false, w.H23));
    GSI_TRY(op_gram(c, c->D, c->Rp, true, w.H33));
  }
  const int nb = prev ? 3 : 2;
  prof_begin(c);
  GSI_TRY(lobcg_assemble(p, nb, c->Cm, w.H12, w.H13, w.H22, w.H23, w.H33, c->lob_mask, c->lob_mask + p,
                         -(10.0 * c->anorm + 1.0), w.H, c->st));
  GSI_TRY(small_eig(nb * p, w.H, w.th, w.U, c->lob_ws, c->st));
  GSI_TRY(lobcg_split(p, nb, w.U, w.V1, w.V2, w.V3, c->st));
  prof_end(c, GSI_K_SMALL, 0.0, 0.0);
  GSI_TRY(op_blockmul(c, prev ? 2 : 1, c->R, w.V2, 1.0, prev ? c->D : nullptr, prev ? w.V3 : nullptr, 1.0, 0,
                      nullptr, 0.0, nullptr, 0.0, c->Yn, false, nullptr));
  GSI_TRY(op_blockmul(c, 1, c->X, w.V1, 1.0, nullptr, nullptr, 0.0, 1, c->Yn, 1.0, nullptr, 0.0, c->Xn, false,
                      nullptr));
  std::swap(c->X, c->Xn);
  std::swap(c->P, c->Yn);
  GSI_TRY(op_matvec(c, c->X, c->Y));
  c->y_fresh = true;
  c->have_prev = true;
  c->iters++;
  return GSI_OK;
}

gsi_status iterate_any(gsi_ctx* c, bool* stop) {
  if (c->o.method == GSI_CHEB) return iterate_cheb(c, stop);
  if (c->o.method == GSI_LOBCG) return iterate_lobcg(c, stop);
  return iterate(c, stop);
}

void fill_info(gsi_ctx* c, gsi_info* info) {
  if (!info) return;
  info->iters = c->iters;
  info->matvecs = c->matvecs;
  info->restarts = c->restarts;
  info->brent_evals = c->last_evals;
  info->converged = c->converged ? 1 : 0;
  info->rel_residual = c->rel;
  info->rel_residual_inf = c->rel_inf;
  info->last_step = c->last_t;
  double tr = 0.0;
  if (cudaMemcpyAsync(c->host, c->Cm, (size_t)c->p * c->p * sizeof(double),
                      cudaMemcpyDeviceToHost, c->st) == cudaSuccess &&
      cudaStreamSynchronize(c->st) == cudaSuccess) {
    for (int i = 0; i < c->p; ++i) tr += c->host[i * c->p + i];
  }
  // the realified objective is twice the complex one
  info->trace = c->sign * tr * (c->herm_n > 0 ? 0.5 : 1.0);
}

// the current X as a start block: orthonormalise it, Y = A X, clear the
// iteration state and the counters
gsi_status restart_state(gsi_ctx* c) {
  c->iters = c->matvecs = c->restarts = c->last_evals = 0;
  c->nd = c->mixed ? 3 : 7;
  c->y_fresh = true;
  c->have_prev = c->converged = false;
  c->rr_prev = 0.0;
  c->res0_inf = -1.0;
  c->last_t = 0.0;
  c->rel = c->rel_inf = NAN;
  GSI_TRY(orthonormalize(c));
  GSI_TRY(op_matvec(c, c->X, c->Y));
  GSI_CUDA_TRY(cudaStreamSynchronize(c->st));
  prof_harvest(c);
  return GSI_OK;
}

// load X0 (float64, host or device), orthonormalise, Y = A X, clear the state
gsi_status start(gsi_ctx* c, const double* X0, int on_device) {
  const size_t blk = (size_t)blk_bytes(c);
  cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (c->emu) {
    GSI_CUDA_TRY(cudaMemcpyAsync(c->W, X0, blk, kind, c->st));  // float64 staging in W
    GSI_TRY(df_from_f64(c->n * c->p, (const double*)c->W, (float2*)c->X, c->st));
  } else {
    GSI_CUDA_TRY(cudaMemcpyAsync(c->X, X0, blk, kind, c->st));
  }
  return restart_state(c);
}

// (re)allocate a device buffer of the context: the old one (if any) is freed
// and dropped from the context's list
gsi_status realloc_dev(gsi_ctx* c, void** p, size_t bytes) {
  if (*p) {
    auto it = std::find(c->allocs.begin(), c->allocs.end(), *p);
    if (it != c->allocs.end()) c->allocs.erase(it);
    cudaFree(*p);
    *p = nullptr;
  }
  return dev_alloc(c, p, bytes);
}

// Stencil-shaped CSR operators (every nonzero on one of at most DIA_MAXD
// diagonals, p even <= 64, df64 mode): the diagonal layout for the staged
// SpMM, used when GSI_SPMM_DIA=1 in the environment at creation. Not the
// default: at 128^3 it measured slower than the CSR kernel at every p
// (p = 64: 1.59 against 1.02 ms), bound by one CTA per SM and far-diagonal
// rows that leave L2 before their reuse.
gsi_status setup_dia(gsi_ctx* c, const gsi_matrix* A) {
  c->use_dia = false;
  const char* env = getenv("GSI_SPMM_DIA");
  if (!c->emu || c->fmt != GSI_CSR || (c->p & 1) || c->p > 64 || !(env && env[0] == '1')) return GSI_OK;
  const int64_t n = c->n, nnz = c->nnz;
  cudaMemcpyKind kind = A->on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
  std::vector<int64_t> rp(n + 1);
  std::vector<int32_t> ci(nnz);
  GSI_CUDA_TRY(cudaMemcpy(rp.data(), A->rowptr, (n + 1) * sizeof(int64_t), kind));
  GSI_CUDA_TRY(cudaMemcpy(ci.data(), A->colidx, nnz * sizeof(int32_t), kind));
  int32_t nd = 0;
  int64_t offs[DIA_MAXD];
  GSI_TRY(gsi_csr_to_dia(n, rp.data(), ci.data(), nullptr, DIA_MAXD, &nd, offs, nullptr));
  if (nd < 1) return GSI_OK;
  DiaArgs a{};
  a.n = n;
  a.p = c->p;
  a.nd = nd;
  for (int d = 0; d < nd; ++d) a.off[d] = (int)offs[d];
  if (!dia_plan(c->p, nd, a.off, &a.q, &a.near_mask, a.far_d, &a.nfar)) return GSI_OK;
  std::vector<double> hv(nnz), dv((size_t)n * nd);
  GSI_CUDA_TRY(cudaMemcpy(hv.data(), A->val, nnz * sizeof(double), kind));
  GSI_TRY(gsi_csr_to_dia(n, rp.data(), ci.data(), hv.data(), DIA_MAXD, &nd, offs, dv.data()));
  std::vector<float2> df(dv.size());
  for (size_t e = 0; e < dv.size(); ++e) df[e] = df_from_double(c->sign * dv[e]);
  GSI_TRY(realloc_dev(c, (void**)&c->dia_val, df.size() * sizeof(float2)));
  GSI_CUDA_TRY(cudaMemcpyAsync(c->dia_val, df.data(), df.size() * sizeof(float2), cudaMemcpyHostToDevice, c->st));
  GSI_CUDA_TRY(cudaStreamSynchronize(c->st));
  a.val = c->dia_val;
  c->dia = a;
  c->use_dia = true;
  return GSI_OK;
}

// Copy the operator A into the context's device memory (sign applied for
// which = -1), with its df64 copy and, for GSI_SELL, its SELL-C-sigma layout.
// Buffers are (re)allocated when missing or when A's sizes differ from the
// last operator's; c->n and c->fmt are already set.
gsi_status upload_operator(gsi_ctx* c, const gsi_matrix* A) {
  const int64_t n = c->n;
  const int p = c->p;
  cudaMemcpyKind kind = A->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (c->fmt == GSI_DENSE) {
    const size_t nn = (size_t)n * n;
    if (!c->Ad) GSI_TRY(dev_alloc(c, (void**)&c->Ad, nn * sizeof(double)));
    GSI_CUDA_TRY(cudaMemcpyAsync(c->Ad, A->val, nn * sizeof(double), kind, c->st));
    if (c->sign < 0) {
      scale_kernel<<<ceil_div((int64_t)nn, 256), 256, 0, c->st>>>((int64_t)nn, -1.0, c->Ad);
      note_launch();
      GSI_CUDA_TRY(cudaGetLastError());
    }
    if (c->emu) {
      if (!c->Adf) GSI_TRY(dev_alloc(c, (void**)&c->Adf, nn * sizeof(float2)));
      GSI_TRY(df_from_f64((int64_t)nn, c->Ad, c->Adf, c->st));
      if (!c->dense_ws) GSI_TRY(dev_alloc(c, (void**)&c->dense_ws, oz_gram_scratch_bytes(n, (int)n, p, false)));
    }
    return GSI_OK;
  }
  const bool grow = !c->val || A->nnz != c->nnz;
  c->nnz = A->nnz;
  if (!c->rowptr) GSI_TRY(dev_alloc(c, (void**)&c->rowptr, (n + 1) * sizeof(int64_t)));
  if (grow) {
    GSI_TRY(realloc_dev(c, (void**)&c->colidx, c->nnz * sizeof(int32_t)));
    GSI_TRY(realloc_dev(c, (void**)&c->val, c->nnz * sizeof(double)));
    if (c->emu) GSI_TRY(realloc_dev(c, (void**)&c->vdf, c->nnz * sizeof(float2)));
  }
  GSI_CUDA_TRY(cudaMemcpyAsync(c->rowptr, A->rowptr, (n + 1) * sizeof(int64_t), kind, c->st));
  GSI_CUDA_TRY(cudaMemcpyAsync(c->colidx, A->colidx, c->nnz * sizeof(int32_t), kind, c->st));
  GSI_CUDA_TRY(cudaMemcpyAsync(c->val, A->val, c->nnz * sizeof(double), kind, c->st));
  if (c->sign < 0 && c->nnz > 0) {
    scale_kernel<<<ceil_div(c->nnz, 256), 256, 0, c->st>>>(c->nnz, -1.0, c->val);
    note_launch();
    GSI_CUDA_TRY(cudaGetLastError());
  }
  if (c->emu) GSI_TRY(df_from_f64(c->nnz, c->val, c->vdf, c->st));
  GSI_TRY(setup_dia(c, A));
  if (c->fmt == GSI_SELL) {
    c->C = A->sell_C > 0 ? A->sell_C : 32;
    int sigma = A->sell_sigma > 0 ? A->sell_sigma : 32;
    std::vector<int64_t> hrp(n + 1);
    std::vector<int32_t> hci(c->nnz);
    std::vector<double> hv(c->nnz);
    GSI_CUDA_TRY(cudaMemcpyAsync(hrp.data(), c->rowptr, (n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, c->st));
    GSI_CUDA_TRY(cudaMemcpyAsync(hci.data(), c->colidx, c->nnz * sizeof(int32_t), cudaMemcpyDeviceToHost, c->st));
    GSI_CUDA_TRY(cudaMemcpyAsync(hv.data(), c->val, c->nnz * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    GSI_CUDA_TRY(cudaStreamSynchronize(c->st));
    int64_t nch = 0, total = 0;
    GSI_TRY(gsi_sell_size(n, hrp.data(), c->C, sigma, &nch, &total));
    std::vector<int64_t> perm(nch * c->C), cptr(nch + 1), clen(nch);
    std::vector<int32_t> scol(total);
    std::vector<double> sval(total);
    GSI_TRY(gsi_csr_to_sell(n, hrp.data(), hci.data(), hv.data(), c->C, sigma, perm.data(), cptr.data(),
                            clen.data(), scol.data(), sval.data()));
    c->nchunks = nch;
    GSI_TRY(realloc_dev(c, (void**)&c->perm, perm.size() * sizeof(int64_t)));
    GSI_TRY(realloc_dev(c, (void**)&c->chunk_ptr, cptr.size() * sizeof(int64_t)));
    GSI_TRY(realloc_dev(c, (void**)&c->chunk_len, clen.size() * sizeof(int64_t)));
    GSI_TRY(realloc_dev(c, (void**)&c->scol, scol.size() * sizeof(int32_t)));
    GSI_TRY(realloc_dev(c, (void**)&c->sval, sval.size() * sizeof(double)));
    GSI_CUDA_TRY(cudaMemcpyAsync(c->perm, perm.data(), perm.size() * 8, cudaMemcpyHostToDevice, c->st));
    GSI_CUDA_TRY(cudaMemcpyAsync(c->chunk_ptr, cptr.data(), cptr.size() * 8, cudaMemcpyHostToDevice, c->st));
    GSI_CUDA_TRY(cudaMemcpyAsync(c->chunk_len, clen.data(), clen.size() * 8, cudaMemcpyHostToDevice, c->st));
    GSI_CUDA_TRY(cudaMemcpyAsync(c->scol, scol.data(), scol.size() * 4, cudaMemcpyHostToDevice, c->st));
    GSI_CUDA_TRY(cudaMemcpyAsync(c->sval, sval.data(), sval.size() * 8, cudaMemcpyHostToDevice, c->st));
    if (c->emu) {
      GSI_TRY(realloc_dev(c, (void**)&c->sdf, sval.size() * sizeof(float2)));
      GSI_TRY(df_from_f64((int64_t)sval.size(), c->sval, c->sdf, c->st));
    }
    GSI_CUDA_TRY(cudaStreamSynchronize(c->st));
  }
  return GSI_OK;
}

// c->anorm: the given bound, else ||A||_inf of the context's operator
gsi_status set_anorm(gsi_ctx* c, double anorm) {
  if (anorm > 0) {
    c->anorm = anorm;
    return GSI_OK;
  }
  unsigned long long* d_mx = (unsigned long long*)c->dout;
  GSI_CUDA_TRY(cudaMemsetAsync(d_mx, 0, 8, c->st));
  if (c->fmt == GSI_DENSE) {
    GSI_TRY(dense_absmax(c->n, c->Ad, d_mx, c->st));
  } else {
    csr_absmax_kernel<<<ceil_div(c->n, 256), 256, 0, c->st>>>(c->n, c->rowptr, c->val, d_mx);
    note_launch();
    GSI_CUDA_TRY(cudaGetLastError());
  }
  GSI_TRY(readback(c, c->dout, 1));
  c->anorm = c->host[0];
  if (!(c->anorm > 0)) c->anorm = 1.0;
  return GSI_OK;
}

}  // namespace

extern "C" {

gsi_status gsi_default_opts(gsi_opts* o) {
  if (!o) return GSI_ERR_ARG;
  o->method = GSI_SD;
  o->which = 1;
  o->tol = 1e-8;
  o->anorm = 0.0;
  o->max_iters = 10000;
  o->k_restart = 0;
  o->recompute_every = 50;
  o->explicit_ax = 0;
  o->precision = GSI_PREC_DF64;
  o->cheb_degree = 8;
  o->cheb_lo = 0.0;
  o->cheb_hi = 0.0;
  o->cheb_scale = 0.0;
  o->mixed_switch = 1e-5;
  o->stop_rule = 0;
  o->cheb_adaptive = 0;
  o->cheb_guard = 0;
  return GSI_OK;
}

const char* gsi_status_str(gsi_status s) {
  switch (s) {
    case GSI_OK: return "ok";
    case GSI_ERR_ARG: return "invalid argument";
    case GSI_ERR_CUDA: return "CUDA error";
    case GSI_ERR_OOM: return "out of device memory";
    case GSI_ERR_NOCONV: return "not converged within max_iters";
    case GSI_ERR_BREAKDOWN: return "breakdown of a p x p factorisation";
    case GSI_ERR_NONFINITE: return "non-finite value";
    case GSI_ERR_TIMEOUT: return "device wait timed out";
  }
  return "unknown status";
}

const char* gsi_last_error(void) { return g_last_error; }

gsi_status gsi_destroy(gsi_ctx* c) {
  if (!c) return GSI_ERR_ARG;
  if (c->st) cudaStreamSynchronize(c->st);
  if (c->st2) {
    cudaStreamSynchronize(c->st2);
    cudaStreamDestroy(c->st2);
  }
  if (c->ev_b) cudaEventDestroy(c->ev_b);
  if (c->ev_e) cudaEventDestroy(c->ev_e);
  prof_harvest(c);
  for (cudaEvent_t e : c->pool) cudaEventDestroy(e);
  for (void* p : c->allocs) cudaFree(p);
  if (c->host) cudaFreeHost(c->host);
  if (c->tmo) cudaFreeHost(c->tmo);
  delete c;
  return GSI_OK;
}

gsi_status gsi_create(const gsi_matrix* A, int32_t p, const double* X0, int32_t X0_on_device,
                      const gsi_opts* o, void* stream, gsi_ctx** out) {
  if (!A || !X0 || !out || !A->val) return GSI_ERR_ARG;
  if (A->fmt != GSI_CSR && A->fmt != GSI_SELL && A->fmt != GSI_DENSE) return GSI_ERR_ARG;
  if (A->fmt != GSI_DENSE && (!A->rowptr || !A->colidx)) return GSI_ERR_ARG;
  if (p < 1 || p > 128 || A->n < 2 * (int64_t)p || (A->fmt != GSI_DENSE && A->nnz < 0))
    return GSI_ERR_ARG;
  gsi_opts opts;
  gsi_default_opts(&opts);
  if (o) opts = *o;
  if (opts.method == GSI_CHEB && !opts.cheb_adaptive &&
      (opts.cheb_degree < 1 || !(opts.cheb_hi > opts.cheb_lo) || !(opts.cheb_scale > opts.cheb_hi)))
    return GSI_ERR_ARG;
  if (opts.method == GSI_CHEB && (opts.cheb_degree < 1 || opts.cheb_guard < 0 || opts.cheb_guard >= p))
    return GSI_ERR_ARG;
  if (opts.method == GSI_LOBCG && p > 64) return GSI_ERR_ARG;
  if ((opts.method != GSI_SD && opts.method != GSI_CG && opts.method != GSI_CHEB && opts.method != GSI_LOBCG) ||
      (opts.which != 1 && opts.which != -1) ||
      opts.max_iters < 0 || !(opts.tol >= 0.0) || (opts.stop_rule != 0 && opts.stop_rule != 1) ||
      (opts.precision != GSI_PREC_DF64 && opts.precision != GSI_PREC_F64 &&
       opts.precision != GSI_PREC_MIXED))
    return GSI_ERR_ARG;
  gsi_ctx* c = new gsi_ctx();
  *out = nullptr;
  c->st = (cudaStream_t)stream;
  c->n = A->n;
  c->nnz = A->nnz;
  c->p = p;
  c->o = opts;
  c->emu = opts.precision != GSI_PREC_F64;
  c->mixed = opts.precision == GSI_PREC_MIXED;
  c->nd = c->mixed ? 3 : 7;
  c->fmt = A->fmt;
  c->sign = opts.which == -1 ? -1.0 : 1.0;
  const int64_t n = c->n;
  const size_t blk = (size_t)n * p * 8;
  gsi_status s = GSI_OK;
#define CK(expr)                \
  do {                          \
    s = (expr);                 \
    if (s != GSI_OK) goto fail; \
  } while (0)
  if (c->fmt == GSI_DENSE) c->nnz = 0;
  CK(upload_operator(c, A));
  {
    void* bufs[9];
    for (int i = 0; i < 9; ++i) CK(dev_alloc(c, &bufs[i], blk));
    c->X = bufs[0]; c->Y = bufs[1]; c->R = bufs[2]; c->Rp = bufs[3];
    c->D = bufs[4]; c->P = bufs[5]; c->W = bufs[6]; c->Xn = bufs[7]; c->Yn = bufs[8];
    const size_t q = (size_t)p * p;
    CK(dev_alloc(c, (void**)&c->pp, (11 * q + 64) * sizeof(double)));
    c->Cm = c->pp; c->Bm = c->pp + q; c->Gm = c->pp + 2 * q; c->Zm = c->pp + 3 * q;
    c->XXm = c->pp + 4 * q; c->XDm = c->pp + 5 * q; c->Km = c->pp + 6 * q; c->Mm = c->pp + 7 * q;
    c->Gm2 = c->pp + 8 * q;
    c->Tm = c->pp + 9 * q;
    c->Fm = c->pp + 10 * q;
    c->out = c->pp + 11 * q;
    c->dout = c->out + 16;
    if (c->emu) {
      CK(dev_alloc(c, (void**)&c->oz_gram_ws, oz_gram_scratch_bytes(n, p, p, false)));
      CK(dev_alloc(c, &c->oz_rhs_ws, oz_rhs_bytes(p, 2)));
      CK(dev_alloc(c, (void**)&c->oz_parts, (size_t)oz_gemm_max_parts(p) * 2 * sizeof(float2)));
      CK(dev_alloc(c, (void**)&c->oz_rinf, (size_t)oz_gemm_max_parts(p) * sizeof(float)));
      CK(dev_alloc(c, (void**)&c->dots_ws, (size_t)df_dots_blocks(n * p) * 3 * sizeof(float2)));
    } else {
      CK(dev_alloc(c, (void**)&c->gram_ws, gram_scratch_doubles(n, p, p) * sizeof(double)));
      CK(dev_alloc(c, (void**)&c->dots_ws, (size_t)dots_blocks(n) * 3 * sizeof(double)));
    }
    CK(dev_alloc(c, (void**)&c->small_ws, std::max(small_scratch_doubles(p) * sizeof(double),
                                                   small_df_scratch_bytes(p))));
    if (c->emu) {
      CK(dev_alloc(c, &c->eig_ws, (size_t)(q + p) * sizeof(float2)));
      CK(cuda_status_ok(cudaStreamCreateWithFlags(&c->st2, cudaStreamNonBlocking)));
      CK(cuda_status_ok(cudaEventCreateWithFlags(&c->ev_b, cudaEventDisableTiming)));
      CK(cuda_status_ok(cudaEventCreateWithFlags(&c->ev_e, cudaEventDisableTiming)));
    }
    if (opts.method == GSI_LOBCG) {
      CK(dev_alloc(c, (void**)&c->lob, lob_doubles(p) * sizeof(double)));
      CK(dev_alloc(c, (void**)&c->lob_mask, 2 * (size_t)p * sizeof(int)));
      CK(dev_alloc(c, (void**)&c->lob_ws, small_scratch_doubles(3 * p) * sizeof(double)));
    }
    CK(cuda_status_ok(cudaMallocHost((void**)&c->host, std::max<size_t>(q, 64) * sizeof(double))));
    CK(cuda_status_ok(cudaMallocHost((void**)&c->tmo, 64)));
    CK(oz_timeouts_async(c->tmo, c->st));
    CK(cuda_status_ok(cudaStreamSynchronize(c->st)));
    c->tmo_seen = *c->tmo;
    CK(set_anorm(c, opts.anorm));
    CK(timeout_check(c, start(c, X0, X0_on_device)));
  }
#undef CK
  *out = c;
  return GSI_OK;
fail:
  gsi_destroy(c);
  return s;
}

gsi_status gsi_reset(gsi_ctx* c, const double* X0, int32_t X0_on_device) {
  if (!c || !X0) return GSI_ERR_ARG;
  return timeout_check(c, start(c, X0, X0_on_device));
}

gsi_status gsi_set_operator(gsi_ctx* c, const gsi_matrix* A, double anorm) {
  if (!c || !A || !A->val || A->fmt != c->fmt || A->n != c->n) return GSI_ERR_ARG;
  if (A->fmt != GSI_DENSE && (!A->rowptr || !A->colidx || A->nnz < 0)) return GSI_ERR_ARG;
  GSI_TRY(upload_operator(c, A));
  GSI_TRY(set_anorm(c, anorm > 0 ? anorm : c->o.anorm));
  return timeout_check(c, restart_state(c));
}

gsi_status gsi_step(gsi_ctx* c, int32_t nsteps, gsi_info* info) {
  if (!c || nsteps < 0) return GSI_ERR_ARG;
  for (int i = 0; i < nsteps; ++i) {
    bool stop = false;
    gsi_status s = iterate_any(c, &stop);
    if (s != GSI_OK) return timeout_check(c, s);
    if (stop) break;
  }
  fill_info(c, info);
  return timeout_check(c, GSI_OK);
}

gsi_status gsi_solve(gsi_ctx* c, gsi_info* info) {
  if (!c) return GSI_ERR_ARG;
  for (;;) {
    bool stop = false;
    gsi_status s = iterate_any(c, &stop);
    if (s != GSI_OK) return timeout_check(c, s);
    if (stop) break;
  }
  fill_info(c, info);
  return timeout_check(c, c->converged ? GSI_OK : GSI_ERR_NOCONV);
}

gsi_status gsi_set_wait_limit(int32_t polls) { return oz_set_wait_limit(polls); }

gsi_status gsi_device_timeouts(int64_t* count) {
  if (!count) return GSI_ERR_ARG;
  int* h = nullptr;
  GSI_CUDA_TRY(cudaMallocHost((void**)&h, sizeof(int)));
  gsi_status s = oz_timeouts_async(h, 0);
  cudaError_t e = cudaStreamSynchronize(0);
  if (s == GSI_OK && e != cudaSuccess) s = cuda_status(e);
  if (s == GSI_OK) *count = *h;
  cudaFreeHost(h);
  return s;
}

gsi_status gsi_create_hermitian(const gsi_zmatrix* A, int32_t p, const double* X0, int32_t X0_on_device,
                                const gsi_opts* o, void* stream, gsi_ctx** out) {
  if (!A || !X0 || !out || !A->rowptr || !A->colidx || !A->val || p < 1 || p > 64 || A->n < 1 ||
      A->n < 2 * (int64_t)p || A->nnz < 0)
    return GSI_ERR_ARG;
  if (o && o->method != GSI_SD && o->method != GSI_CG) return GSI_ERR_ARG;
  const int64_t n = A->n, nnz = A->nnz;
  std::vector<int64_t> rp(n + 1);
  std::vector<int32_t> ci(nnz);
  std::vector<double> va(2 * nnz), x0(2 * (size_t)n * p);
  cudaMemcpyKind kA = A->on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
  cudaMemcpyKind kX = X0_on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
  GSI_CUDA_TRY(cudaMemcpy(rp.data(), A->rowptr, (n + 1) * sizeof(int64_t), kA));
  GSI_CUDA_TRY(cudaMemcpy(ci.data(), A->colidx, nnz * sizeof(int32_t), kA));
  GSI_CUDA_TRY(cudaMemcpy(va.data(), A->val, 2 * nnz * sizeof(double), kA));
  GSI_CUDA_TRY(cudaMemcpy(x0.data(), X0, x0.size() * sizeof(double), kX));
  if (rp[0] != 0 || rp[n] != nnz) return GSI_ERR_ARG;
  for (int64_t r = 0; r < n; ++r)
    if (rp[r + 1] < rp[r]) return GSI_ERR_ARG;
  // [[Ar, -Ai], [Ai, Ar]] (2n x 2n), exact zeros dropped except the diagonal
  std::vector<int64_t> hrp(2 * n + 1, 0);
  std::vector<int32_t> hci;
  std::vector<double> hva;
  hci.reserve(4 * nnz);
  hva.reserve(4 * nnz);
  for (int half = 0; half < 2; ++half)
    for (int64_t r = 0; r < n; ++r) {
      const int64_t R = half * n + r;
      for (int part = 0; part < 2; ++part)  // column block: Re part (cols < n), then Im part
        for (int64_t k = rp[r]; k < rp[r + 1]; ++k) {
          const int32_t col = ci[k];
          if (col < 0 || col >= n) return GSI_ERR_ARG;
          const double re = va[2 * k], im = va[2 * k + 1];
          // half 0: row r of [Ar, -Ai]; half 1: row r of [Ai, Ar]
          const double v = half == 0 ? (part == 0 ? re : -im) : (part == 0 ? im : re);
          const int64_t C = part * n + col;
          if (v != 0.0 || C == R) {
            hci.push_back((int32_t)C);
            hva.push_back(v);
          }
        }
      hrp[R + 1] = (int64_t)hci.size();
    }
  if (2 * n > INT32_MAX) return GSI_ERR_ARG;
  // [[X0r, -X0i], [X0i, X0r]] (2n x 2p, row-major)
  std::vector<double> hx(4 * (size_t)n * p);
  for (int64_t r = 0; r < n; ++r)
    for (int j = 0; j < p; ++j) {
      const double re = x0[2 * ((size_t)r * p + j)], im = x0[2 * ((size_t)r * p + j) + 1];
      hx[(size_t)r * 2 * p + j] = re;
      hx[(size_t)r * 2 * p + p + j] = -im;
      hx[(size_t)(n + r) * 2 * p + j] = im;
      hx[(size_t)(n + r) * 2 * p + p + j] = re;
    }
  gsi_opts opts;
  gsi_default_opts(&opts);
  if (o) opts = *o;
  // ||R^||_F = sqrt(2) ||R||_F: the bound scaled alike keeps the test on the complex residual
  if (opts.anorm > 0) opts.anorm *= sqrt(2.0);
  gsi_matrix m{};
  m.fmt = GSI_CSR;
  m.n = 2 * n;
  m.nnz = (int64_t)hci.size();
  m.rowptr = hrp.data();
  m.colidx = hci.data();
  m.val = hva.data();
  m.on_device = 0;
  GSI_TRY(gsi_create(&m, 2 * p, hx.data(), 0, &opts, stream, out));
  (*out)->herm_n = n;
  return GSI_OK;
}

gsi_status gsi_get_basis_hermitian(gsi_ctx* c, double* X, double* evals, int32_t to_device) {
  if (!c || c->herm_n <= 0) return GSI_ERR_ARG;
  const int64_t n = c->herm_n;
  const int p = c->p / 2;
  if (evals) {
    std::vector<double> ev(2 * (size_t)p);
    GSI_TRY(gsi_get_basis(c, nullptr, ev.data(), 0));
    std::vector<double> e(p);
    for (int i = 0; i < p; ++i) e[i] = ev[2 * i];  // each complex Ritz value appears twice
    if (to_device) {
      GSI_CUDA_TRY(cudaMemcpy(evals, e.data(), p * sizeof(double), cudaMemcpyHostToDevice));
    } else {
      memcpy(evals, e.data(), p * sizeof(double));
    }
  }
  if (X) {
    std::vector<double> xr(4 * (size_t)n * p), xz(2 * (size_t)n * p);
    GSI_TRY(gsi_get_basis(c, xr.data(), nullptr, 0));
    for (int64_t r = 0; r < n; ++r)
      for (int j = 0; j < p; ++j) {
        xz[2 * ((size_t)r * p + j)] = xr[(size_t)r * 2 * p + j];
        xz[2 * ((size_t)r * p + j) + 1] = xr[(size_t)(n + r) * 2 * p + j];
      }
    if (to_device) {
      GSI_CUDA_TRY(cudaMemcpy(X, xz.data(), xz.size() * sizeof(double), cudaMemcpyHostToDevice));
    } else {
      memcpy(X, xz.data(), xz.size() * sizeof(double));
    }
  }
  return GSI_OK;
}

gsi_status gsi_state_ptrs(gsi_ctx* c, void** X, void** Y) {
  if (!c) return GSI_ERR_ARG;
  if (X) *X = c->X;
  if (Y) *Y = c->Y;
  return GSI_OK;
}

gsi_status gsi_get_basis(gsi_ctx* c, double* X, double* evals, int32_t to_device) {
  if (!c) return GSI_ERR_ARG;
  const int p = c->p;
  const size_t blk = (size_t)blk_bytes(c);
  cudaMemcpyKind kind = to_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  const void* src = c->X;
  if (evals) {
    // Rayleigh-Ritz with an explicit AX: theta in Tm, U in Gm2; W and Yn are
    // scratch. Only buffers that no later iteration reads are touched (not K
    // of the CG transport).
    GSI_TRY(op_matvec(c, c->X, c->W));
    c->matvecs--;  // not part of the iteration count
    GSI_TRY(op_gram(c, c->X, c->W, true, c->Fm));
    GSI_TRY(small_eig(p, c->Fm, c->Tm, c->Gm2, c->small_ws, c->st));
    if (X) {
      GSI_TRY(op_blockmul(c, 1, c->X, c->Gm2, 1.0, nullptr, nullptr, 0.0, 0, nullptr, 0.0, nullptr,
                          0.0, c->Yn, false, nullptr));
      src = c->Yn;
    }
  }
  if (X) {
    if (c->emu) {
      GSI_TRY(df_to_f64(c->n * p, (const float2*)src, (double*)c->W, c->st));
      src = c->W;
    }
    GSI_CUDA_TRY(cudaMemcpyAsync(X, src, blk, kind, c->st));
  }
  if (evals) {
    GSI_CUDA_TRY(cudaMemcpyAsync(c->host, c->Tm, p * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  }
  GSI_CUDA_TRY(cudaStreamSynchronize(c->st));
  prof_harvest(c);
  if (evals) {
    std::vector<double> ev(p);
    for (int i = 0; i < p; ++i) ev[i] = c->sign * c->host[i];
    if (to_device) {
      GSI_CUDA_TRY(cudaMemcpy(evals, ev.data(), p * sizeof(double), cudaMemcpyHostToDevice));
    } else {
      memcpy(evals, ev.data(), p * sizeof(double));
    }
  }
  return GSI_OK;
}

gsi_status gsi_profile_enable(gsi_ctx* c, int32_t on) {
  if (!c) return GSI_ERR_ARG;
  GSI_CUDA_TRY(cudaStreamSynchronize(c->st));
  prof_harvest(c);
  c->prof = on != 0;
  for (auto& k : c->cls) k = gsi_ctx::Cls{};
  return GSI_OK;
}

gsi_status gsi_profile_read(gsi_ctx* c, int32_t k, int64_t* launches, double* total_ms,
                            double* alg_bytes, double* alg_flops) {
  if (!c || k < 0 || k >= GSI_K_COUNT) return GSI_ERR_ARG;
  GSI_CUDA_TRY(cudaStreamSynchronize(c->st));
  prof_harvest(c);
  if (launches) *launches = c->cls[k].launches;
  if (total_ms) *total_ms = c->cls[k].ms;
  if (alg_bytes) *alg_bytes = c->cls[k].bytes;
  if (alg_flops) *alg_flops = c->cls[k].flops;
  return GSI_OK;
}

int64_t gsi_launch_count(void) { return (int64_t)g_launches.load(); }

}  // extern "C"
