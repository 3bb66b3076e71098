// Solver context and C entry points: Riemannian steepest descent (Alg. 2)
// and conjugate gradients (Alg. 4) with the exact line search of Alg. 3 and
// the one-matvec recursion of Eq. (save_matvec).
//
// One iteration (R = AX - XC is the residual, -grad phi; the step is
// X + tD with t >= 0):
//   C = X^T Y; R = Y - X C; stop if ||R||_F <= tol * anorm (explicit AX)
//   D = R (SD), or D = R + b (P - X (X^T P)) with the Polak-Ribiere b (CG,
//       restart to R when <D, R> <= 0 or every k_restart iterations)
//   W = A D
//   B = D^T D, Gam = D^T W, Z = D^T R (SD: Z = B), XX = X^T X, XD = X^T D
//   (t, M) from the p x p step; X <- (X + tD) M, Y <- (Y + tW) M
// where M = S^{-1/2} with S = XX + t (XD + XD^T) + t^2 B, the measured Gram
// of X + tD, so that (X + tD) M is its polar factor (Eq. (Ynew)).
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <vector>

#include "blas_f64.cuh"

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

struct gsi_ctx {
  cudaStream_t st = nullptr;
  int64_t n = 0, nnz = 0;
  int p = 0;
  gsi_opts o{};
  int fmt = GSI_CSR;
  int64_t* rowptr = nullptr;
  int32_t* colidx = nullptr;
  double* val = nullptr;
  int C = 32;
  int64_t nchunks = 0;
  int64_t* perm = nullptr;
  int64_t* chunk_ptr = nullptr;
  int64_t* chunk_len = nullptr;
  int32_t* scol = nullptr;
  double* sval = nullptr;
  double anorm = 0.0;
  double sign = 1.0;
  double *X = nullptr, *Y = nullptr, *R = nullptr, *Rp = nullptr, *D = nullptr, *P = nullptr,
         *W = nullptr;
  double* pp = nullptr;  // p x p matrices
  double *Cm, *Bm, *Gm, *Zm, *XXm, *XDm, *Km, *Mm, *out, *dout;
  double* gram_ws = nullptr;
  double* dots_ws = nullptr;
  double* small_ws = nullptr;
  double* host = nullptr;  // pinned readback buffer
  std::vector<void*> allocs;
  // iteration state
  int iters = 0, matvecs = 0, restarts = 0, last_evals = 0;
  bool y_fresh = true, have_prev = false, converged = false;
  double rr_prev = 0.0, res0_inf = -1.0, last_t = 0.0, rel = NAN, rel_inf = NAN;
};

namespace {

gsi_status dev_alloc(gsi_ctx* c, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 16));
  if (e != cudaSuccess) return cuda_status(e);
  c->allocs.push_back(*p);
  return GSI_OK;
}

gsi_status matvec(gsi_ctx* c, const double* in, double* outp) {
  c->matvecs++;
  if (c->fmt == GSI_SELL)
    return spmm_sell(c->n, c->nchunks, c->C, c->perm, c->chunk_ptr, c->chunk_len, c->scol,
                     c->sval, c->p, in, outp, c->st);
  return spmm_csr(c->n, c->rowptr, c->colidx, c->val, c->p, in, outp, c->st);
}

gsi_status G(gsi_ctx* c, const double* U, const double* V, double* out) {
  return gram(c->n, c->p, c->p, U, V, out, c->gram_ws, c->st);
}

gsi_status readback(gsi_ctx* c, const double* src, int count) {
  GSI_CUDA_TRY(cudaMemcpyAsync(c->host, src, count * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  GSI_CUDA_TRY(cudaStreamSynchronize(c->st));
  return GSI_OK;
}

// X <- X M (in place), M = (X^T X)^{-1/2}.
gsi_status orthonormalize(gsi_ctx* c) {
  for (int pass = 0; pass < 2; ++pass) {
    GSI_TRY(G(c, c->X, c->X, c->Bm));
    GSI_TRY(small_step(1, c->p, nullptr, c->Bm, nullptr, nullptr, nullptr, nullptr, c->Mm, c->out,
                       c->small_ws, c->st));
    GSI_TRY(readback(c, c->out, 5));
    if (c->host[3] != 0.0) return GSI_ERR_BREAKDOWN;
    RowMulArgs a{};
    a.nk = 1;
    a.U[0] = c->X;
    a.M[0] = c->Mm;
    a.s[0] = 1.0;
    GSI_TRY(rowmul(c->n, c->p, a, c->X, c->st));
  }
  return GSI_OK;
}

// One iteration; returns GSI_OK and sets *stop when the stopping test holds.
gsi_status iterate(gsi_ctx* c, bool* stop) {
  const int p = c->p;
  const int64_t n = c->n;
  const bool cg = c->o.method == GSI_CG;
  *stop = false;
  double rr = 0.0, rp = 0.0, rinf = 0.0;
  for (;;) {
    GSI_TRY(G(c, c->X, c->Y, c->Cm));
    symmetrize_kernel<<<ceil_div(p * p, 256), 256, 0, c->st>>>(p, c->Cm);
    GSI_LAUNCH_CHECK();
    RowMulArgs a{};
    a.nk = 1;
    a.U[0] = c->X;
    a.M[0] = c->Cm;
    a.s[0] = -1.0;
    a.ne = 1;
    a.E[0] = c->Y;
    a.c[0] = 1.0;
    GSI_TRY(rowmul(n, p, a, c->R, c->st));
    bool want_rp = cg && c->have_prev;
    GSI_TRY(dots(n, p, want_rp ? 2 : 1, c->R, c->R, c->R, c->Rp, c->R, c->dout, c->dots_ws, c->st));
    GSI_TRY(readback(c, c->dout, 3));
    rr = c->host[0];
    rp = c->host[1];
    rinf = c->host[2];
    if (!isfinite(rr)) return GSI_ERR_NONFINITE;
    if (c->res0_inf < 0.0) c->res0_inf = rinf;
    c->rel = sqrt(rr) / c->anorm;
    c->rel_inf = c->res0_inf > 0.0 ? rinf / c->res0_inf : 0.0;
    if (c->rel <= c->o.tol || c->iters >= c->o.max_iters) {
      if (!c->y_fresh) {  // the final residual is always taken with an explicit AX
        GSI_TRY(matvec(c, c->X, c->Y));
        c->y_fresh = true;
        continue;
      }
      c->converged = c->rel <= c->o.tol;
      *stop = true;
      return GSI_OK;
    }
    break;
  }
  // search direction
  const double* Dp = c->R;
  bool restarted = false;
  if (cg) {
    if (c->have_prev) {
      double b = (rr - rp) / c->rr_prev;
      GSI_TRY(G(c, c->X, c->P, c->Km));
      RowMulArgs a{};
      a.nk = 1;
      a.U[0] = c->X;
      a.M[0] = c->Km;
      a.s[0] = -b;
      a.ne = 2;
      a.E[0] = c->R;
      a.c[0] = 1.0;
      a.E[1] = c->P;
      a.c[1] = b;
      GSI_TRY(rowmul(n, p, a, c->D, c->st));
      GSI_TRY(dots(n, p, 1, c->D, c->R, nullptr, nullptr, nullptr, c->dout, c->dots_ws, c->st));
      GSI_TRY(readback(c, c->dout, 1));
      bool due = c->o.k_restart > 0 && c->iters % c->o.k_restart == 0;
      if (due || !(c->host[0] > 0.0)) restarted = true;
    }
    if (!c->have_prev || restarted) {
      GSI_CUDA_TRY(cudaMemcpyAsync(c->D, c->R, (size_t)n * p * sizeof(double),
                                   cudaMemcpyDeviceToDevice, c->st));
    }
    if (restarted) c->restarts++;
    Dp = c->D;
  }
  GSI_TRY(matvec(c, Dp, c->W));
  GSI_TRY(G(c, Dp, Dp, c->Bm));
  GSI_TRY(G(c, Dp, c->W, c->Gm));
  const double* Zp = c->Bm;
  if (cg) {
    GSI_TRY(G(c, Dp, c->R, c->Zm));
    Zp = c->Zm;
  }
  GSI_TRY(G(c, c->X, c->X, c->XXm));
  GSI_TRY(G(c, c->X, Dp, c->XDm));
  GSI_TRY(small_step(0, p, c->Cm, c->Bm, c->Gm, Zp, c->XXm, c->XDm, c->Mm, c->out, c->small_ws,
                     c->st));
  GSI_TRY(readback(c, c->out, 5));
  const double t = c->host[0];
  c->last_t = t;
  c->last_evals = (int)c->host[2];
  if (c->host[3] != 0.0) return GSI_ERR_BREAKDOWN;
  if (!isfinite(t)) return GSI_ERR_NONFINITE;
  const double bmax = c->host[4];
  bool recompute = c->o.explicit_ax || t * sqrt(std::max(bmax, 0.0)) < 1e3 * 2.220446049250313e-16 ||
                   (c->o.recompute_every > 0 && (c->iters + 1) % c->o.recompute_every == 0);
  {
    RowMulArgs a{};
    a.nk = 2;
    a.U[0] = c->X;
    a.M[0] = c->Mm;
    a.s[0] = 1.0;
    a.U[1] = Dp;
    a.M[1] = c->Mm;
    a.s[1] = t;
    GSI_TRY(rowmul(n, p, a, c->X, c->st));
  }
  if (recompute) {
    GSI_TRY(matvec(c, c->X, c->Y));
  } else {
    RowMulArgs a{};
    a.nk = 2;
    a.U[0] = c->Y;
    a.M[0] = c->Mm;
    a.s[0] = 1.0;
    a.U[1] = c->W;
    a.M[1] = c->Mm;
    a.s[1] = t;
    GSI_TRY(rowmul(n, p, a, c->Y, c->st));
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
  info->trace = c->sign * tr;
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
  for (void* p : c->allocs) cudaFree(p);
  if (c->host) cudaFreeHost(c->host);
  delete c;
  return GSI_OK;
}

gsi_status gsi_create(const gsi_matrix* A, int32_t p, const double* X0, int32_t X0_on_device,
                      const gsi_opts* o, void* stream, gsi_ctx** out) {
  if (!A || !X0 || !out || !A->rowptr || !A->colidx || !A->val) return GSI_ERR_ARG;
  if (p < 1 || p > 128 || A->n < 2 * (int64_t)p || A->nnz < 0) return GSI_ERR_ARG;
  if (A->fmt != GSI_CSR && A->fmt != GSI_SELL) return GSI_ERR_ARG;
  gsi_opts opts;
  gsi_default_opts(&opts);
  if (o) opts = *o;
  if ((opts.method != GSI_SD && opts.method != GSI_CG) || (opts.which != 1 && opts.which != -1) ||
      opts.max_iters < 0 || !(opts.tol >= 0.0))
    return GSI_ERR_ARG;
  gsi_ctx* c = new gsi_ctx();
  *out = nullptr;
  c->st = (cudaStream_t)stream;
  c->n = A->n;
  c->nnz = A->nnz;
  c->p = p;
  c->o = opts;
  c->fmt = A->fmt;
  c->sign = opts.which == -1 ? -1.0 : 1.0;
  const int64_t n = c->n;
  const size_t blk = (size_t)n * p * sizeof(double);
  gsi_status s = GSI_OK;
#define CK(expr)               \
  do {                         \
    s = (expr);                \
    if (s != GSI_OK) goto fail; \
  } while (0)
  {
    cudaMemcpyKind kind = A->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CK(dev_alloc(c, (void**)&c->rowptr, (n + 1) * sizeof(int64_t)));
    CK(dev_alloc(c, (void**)&c->colidx, c->nnz * sizeof(int32_t)));
    CK(dev_alloc(c, (void**)&c->val, c->nnz * sizeof(double)));
    CK(cuda_status_ok(cudaMemcpyAsync(c->rowptr, A->rowptr, (n + 1) * sizeof(int64_t), kind, c->st)));
    CK(cuda_status_ok(cudaMemcpyAsync(c->colidx, A->colidx, c->nnz * sizeof(int32_t), kind, c->st)));
    CK(cuda_status_ok(cudaMemcpyAsync(c->val, A->val, c->nnz * sizeof(double), kind, c->st)));
    if (c->sign < 0 && c->nnz > 0) {
      scale_kernel<<<ceil_div(c->nnz, 256), 256, 0, c->st>>>(c->nnz, -1.0, c->val);
      note_launch();
      CK(cuda_status_ok(cudaGetLastError()));
    }
    if (c->fmt == GSI_SELL) {
      c->C = A->sell_C > 0 ? A->sell_C : 32;
      int sigma = A->sell_sigma > 0 ? A->sell_sigma : 32;
      std::vector<int64_t> hrp(n + 1);
      std::vector<int32_t> hci(c->nnz);
      std::vector<double> hv(c->nnz);
      CK(cuda_status_ok(cudaMemcpyAsync(hrp.data(), c->rowptr, (n + 1) * sizeof(int64_t),
                                        cudaMemcpyDeviceToHost, c->st)));
      CK(cuda_status_ok(cudaMemcpyAsync(hci.data(), c->colidx, c->nnz * sizeof(int32_t),
                                        cudaMemcpyDeviceToHost, c->st)));
      CK(cuda_status_ok(cudaMemcpyAsync(hv.data(), c->val, c->nnz * sizeof(double),
                                        cudaMemcpyDeviceToHost, c->st)));
      CK(cuda_status_ok(cudaStreamSynchronize(c->st)));
      int64_t nch = 0, total = 0;
      CK(gsi_sell_size(n, hrp.data(), c->C, sigma, &nch, &total));
      std::vector<int64_t> perm(nch * c->C), cptr(nch + 1), clen(nch);
      std::vector<int32_t> scol(total);
      std::vector<double> sval(total);
      CK(gsi_csr_to_sell(n, hrp.data(), hci.data(), hv.data(), c->C, sigma, perm.data(), cptr.data(),
                         clen.data(), scol.data(), sval.data()));
      c->nchunks = nch;
      CK(dev_alloc(c, (void**)&c->perm, perm.size() * sizeof(int64_t)));
      CK(dev_alloc(c, (void**)&c->chunk_ptr, cptr.size() * sizeof(int64_t)));
      CK(dev_alloc(c, (void**)&c->chunk_len, clen.size() * sizeof(int64_t)));
      CK(dev_alloc(c, (void**)&c->scol, scol.size() * sizeof(int32_t)));
      CK(dev_alloc(c, (void**)&c->sval, sval.size() * sizeof(double)));
      CK(cuda_status_ok(cudaMemcpyAsync(c->perm, perm.data(), perm.size() * 8, cudaMemcpyHostToDevice, c->st)));
      CK(cuda_status_ok(cudaMemcpyAsync(c->chunk_ptr, cptr.data(), cptr.size() * 8, cudaMemcpyHostToDevice, c->st)));
      CK(cuda_status_ok(cudaMemcpyAsync(c->chunk_len, clen.data(), clen.size() * 8, cudaMemcpyHostToDevice, c->st)));
      CK(cuda_status_ok(cudaMemcpyAsync(c->scol, scol.data(), scol.size() * 4, cudaMemcpyHostToDevice, c->st)));
      CK(cuda_status_ok(cudaMemcpyAsync(c->sval, sval.data(), sval.size() * 8, cudaMemcpyHostToDevice, c->st)));
      CK(cuda_status_ok(cudaStreamSynchronize(c->st)));
    }
    double* bufs[7];
    for (int i = 0; i < 7; ++i) CK(dev_alloc(c, (void**)&bufs[i], blk));
    c->X = bufs[0]; c->Y = bufs[1]; c->R = bufs[2]; c->Rp = bufs[3];
    c->D = bufs[4]; c->P = bufs[5]; c->W = bufs[6];
    const size_t q = (size_t)p * p;
    CK(dev_alloc(c, (void**)&c->pp, (8 * q + 64) * sizeof(double)));
    c->Cm = c->pp; c->Bm = c->pp + q; c->Gm = c->pp + 2 * q; c->Zm = c->pp + 3 * q;
    c->XXm = c->pp + 4 * q; c->XDm = c->pp + 5 * q; c->Km = c->pp + 6 * q; c->Mm = c->pp + 7 * q;
    c->out = c->pp + 8 * q;
    c->dout = c->out + 16;
    CK(dev_alloc(c, (void**)&c->gram_ws, gram_scratch_doubles(n, p, p) * sizeof(double)));
    CK(dev_alloc(c, (void**)&c->dots_ws, (size_t)dots_blocks(n) * 3 * sizeof(double)));
    CK(dev_alloc(c, (void**)&c->small_ws, small_scratch_doubles(p) * sizeof(double)));
    CK(cuda_status_ok(cudaMallocHost((void**)&c->host, std::max<size_t>(q, 64) * sizeof(double))));
    // anorm
    if (opts.anorm > 0) {
      c->anorm = opts.anorm;
    } else {
      unsigned long long* d_mx = (unsigned long long*)c->dout;
      CK(cuda_status_ok(cudaMemsetAsync(d_mx, 0, 8, c->st)));
      csr_absmax_kernel<<<ceil_div(n, 256), 256, 0, c->st>>>(n, c->rowptr, c->val, d_mx);
      note_launch();
      CK(cuda_status_ok(cudaGetLastError()));
      CK(readback(c, c->dout, 1));
      c->anorm = c->host[0];
      if (!(c->anorm > 0)) c->anorm = 1.0;
    }
    CK(cuda_status_ok(cudaMemcpyAsync(c->X, X0, blk,
                                      X0_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                      c->st)));
    CK(orthonormalize(c));
    CK(matvec(c, c->X, c->Y));
    CK(cuda_status_ok(cudaStreamSynchronize(c->st)));
  }
#undef CK
  *out = c;
  return GSI_OK;
fail:
  gsi_destroy(c);
  return s;
}

gsi_status gsi_step(gsi_ctx* c, int32_t nsteps, gsi_info* info) {
  if (!c || nsteps < 0) return GSI_ERR_ARG;
  for (int i = 0; i < nsteps; ++i) {
    bool stop = false;
    GSI_TRY(iterate(c, &stop));
    if (stop) break;
  }
  fill_info(c, info);
  return GSI_OK;
}

gsi_status gsi_solve(gsi_ctx* c, gsi_info* info) {
  if (!c) return GSI_ERR_ARG;
  for (;;) {
    bool stop = false;
    GSI_TRY(iterate(c, &stop));
    if (stop) break;
  }
  fill_info(c, info);
  return c->converged ? GSI_OK : GSI_ERR_NOCONV;
}

gsi_status gsi_state_ptrs(gsi_ctx* c, double** X, double** Y) {
  if (!c) return GSI_ERR_ARG;
  if (X) *X = c->X;
  if (Y) *Y = c->Y;
  return GSI_OK;
}

gsi_status gsi_get_basis(gsi_ctx* c, double* X, double* evals, int32_t to_device) {
  if (!c) return GSI_ERR_ARG;
  const int p = c->p;
  const size_t blk = (size_t)c->n * p * sizeof(double);
  cudaMemcpyKind kind = to_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (!evals) {
    if (X) GSI_CUDA_TRY(cudaMemcpyAsync(X, c->X, blk, kind, c->st));
    GSI_CUDA_TRY(cudaStreamSynchronize(c->st));
    return GSI_OK;
  }
  // Rayleigh-Ritz with an explicit AX (W is scratch here): theta in XDm, U in Bm
  GSI_TRY(spmm_csr(c->n, c->rowptr, c->colidx, c->val, p, c->X, c->W, c->st));
  GSI_TRY(G(c, c->X, c->W, c->Km));
  double* U = c->Bm;
  GSI_TRY(small_eig(p, c->Km, c->XDm, U, c->small_ws, c->st));
  if (X) {
    RowMulArgs a{};
    a.nk = 1;
    a.U[0] = c->X;
    a.M[0] = U;
    a.s[0] = 1.0;
    GSI_TRY(rowmul(c->n, p, a, c->W, c->st));
    GSI_CUDA_TRY(cudaMemcpyAsync(X, c->W, blk, kind, c->st));
  }
  GSI_CUDA_TRY(cudaMemcpyAsync(c->host, c->XDm, p * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  GSI_CUDA_TRY(cudaStreamSynchronize(c->st));
  std::vector<double> ev(p);
  for (int i = 0; i < p; ++i) ev[i] = c->sign * c->host[i];
  if (to_device) {
    GSI_CUDA_TRY(cudaMemcpy(evals, ev.data(), p * sizeof(double), cudaMemcpyHostToDevice));
  } else {
    memcpy(evals, ev.data(), p * sizeof(double));
  }
  return GSI_OK;
}

}  // extern "C"
