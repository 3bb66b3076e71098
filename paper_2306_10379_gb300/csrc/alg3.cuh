// The exact line search of Alg. 3 in float64 (one thread): the model
// phi(t) of Eq. (phi_P), its derivative of Eq. (deriv_P), the bracket of
// Eqs. (derv1)/(derv2) and Brent-Dekker root finding on phi'.
#pragma once
#include <math.h>

namespace gsi {

#ifndef GSI_DEPS_DEFINED
#define GSI_DEPS_DEFINED
constexpr double ALG3_EPS = 2.220446049250313e-16;
#endif

// phi'(t) of Eq. (deriv_P), summed over i ascending.
__device__ inline double dphi(double t, int p, const double* al, const double* be, const double* ga,
                       const double* ze) {
  double s = 0.0;
  for (int i = 0; i < p; ++i) {
    double num = ze[i] + (ga[i] - al[i] * be[i]) * t - be[i] * ze[i] * t * t;
    double den = 1.0 + be[i] * t * t;
    s += num / (den * den);
  }
  return -s;
}

__device__ inline double phi_model(double t, int p, const double* al, const double* be,
                            const double* ga, const double* ze) {
  double s = 0.0;
  for (int i = 0; i < p; ++i) s += (al[i] + 2.0 * ze[i] * t + ga[i] * t * t) / (1.0 + be[i] * t * t);
  return -0.5 * s;
}

// Brent-Dekker zero of phi' on [a, b] with phi'(a) phi'(b) <= 0 (R. P. Brent,
// Algorithms for Minimization without Derivatives, 1973, ch. 4): inverse
// quadratic / secant steps kept inside the bracket, bisection otherwise;
// stops when the bracket is below 2 eps |b|. Returns the root; *ev counts
// evaluations.
__device__ inline double brent(double a, double b, double fa, double fb, int p, const double* al,
                        const double* be, const double* ga, const double* ze, int* ev) {
  if (fa == 0.0) return a;
  if (fb == 0.0) return b;
  double c = a, fc = fa, d = b - a, e = d;
  for (int it = 0; it < 100; ++it) {
    if ((fb > 0.0 && fc > 0.0) || (fb < 0.0 && fc < 0.0)) {
      c = a;
      fc = fa;
      d = e = b - a;
    }
    if (fabs(fc) < fabs(fb)) {
      a = b; b = c; c = a;
      fa = fb; fb = fc; fc = fa;
    }
    double tol = 2.0 * ALG3_EPS * fabs(b) + 1e-300;
    double m = 0.5 * (c - b);
    if (fabs(m) <= tol || fb == 0.0) break;
    if (fabs(e) >= tol && fabs(fa) > fabs(fb)) {
      double s = fb / fa, P, Q;
      if (a == c) {
        P = 2.0 * m * s;
        Q = 1.0 - s;
      } else {
        double q = fa / fc, r = fb / fc;
        P = s * (2.0 * m * q * (q - r) - (b - a) * (r - 1.0));
        Q = (q - 1.0) * (r - 1.0) * (s - 1.0);
      }
      if (P > 0.0) Q = -Q; else P = -P;
      if (2.0 * P < fmin(3.0 * m * Q - fabs(tol * Q), fabs(e * Q))) {
        e = d;
        d = P / Q;
      } else {
        d = m;
        e = m;
      }
    } else {
      d = m;
      e = m;
    }
    a = b;
    fa = fb;
    b = (fabs(d) > tol) ? b + d : b + copysign(tol, m);
    fb = dphi(b, p, al, be, ga, ze);
    ++*ev;
  }
  return b;
}

// Alg. 3 generalised to zeta (Sec. 5.2). Bracket-eligible branches have
// beta_i > eps * sum(beta) and zeta_i > 0; xi_i from Eq. (derv1) (delta < 0)
// or Eq. (derv2) (delta >= 0) with zeta in the CG places. The step is the
// first minimiser of the model past xi_min: the right end is doubled from
// xi_min (capped at xi_max) until phi' >= 0, then Brent.
__device__ inline double get_mu(int p, const double* al, const double* be, const double* ga,
                         const double* ze, int* ev) {
  double sb = 0.0;
  for (int i = 0; i < p; ++i) sb += be[i];
  double xmin = INFINITY, xmax = -INFINITY;
  int cnt = 0;
  for (int i = 0; i < p; ++i) {
    double b = be[i], z = ze[i];
    if (!(b > ALG3_EPS * sb) || !(z > 0.0)) continue;
    double d = ga[i] - al[i] * b;
    double disc = sqrt(d * d + 4.0 * b * z * z);
    double xi = (d < 0.0) ? 2.0 * z / (-d + disc) : (d + disc) / (2.0 * b * z);
    xmin = fmin(xmin, xi);
    xmax = fmax(xmax, xi);
    ++cnt;
  }
  *ev = 0;
  if (cnt == 0) return 0.0;
  double fa = dphi(xmin, p, al, be, ga, ze);
  ++*ev;
  double lo, flo, hi, fhi;
  if (fa > 0.0) {
    lo = 0.0;
    flo = dphi(0.0, p, al, be, ga, ze);
    ++*ev;
    if (flo >= 0.0) return 0.0;
    hi = xmin;
    fhi = fa;
  } else {
    lo = flo = hi = fhi = 0.0;
    lo = xmin; flo = fa; hi = xmin; fhi = fa;
    int k = 0;
    while (fhi < 0.0) {
      if (k >= 64) return hi;
      double nxt = 2.0 * hi;
      if (hi < xmax) nxt = fmin(nxt, xmax);
      lo = hi;
      flo = fhi;
      hi = nxt;
      fhi = dphi(hi, p, al, be, ga, ze);
      ++*ev;
      ++k;
    }
  }
  return brent(lo, hi, flo, fhi, p, al, be, ga, ze, ev);
}



// ---- warp-cooperative variants: every lane of one warp runs the same
// control flow; phi and phi' are summed over the lanes (lane j takes terms
// j, j+32, ...), then reduced in a fixed butterfly order.
__device__ inline double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  // lanes may differ in the last bit (different summation orders): take lane
  // 0's value so that every lane follows the same control flow
  return __shfl_sync(0xffffffffu, v, 0);
}

__device__ inline double dphi_warp(double t, int p, const double* al, const double* be,
                                   const double* ga, const double* ze) {
  double s = 0.0;
  for (int i = threadIdx.x & 31; i < p; i += 32) {
    double num = ze[i] + (ga[i] - al[i] * be[i]) * t - be[i] * ze[i] * t * t;
    double den = 1.0 + be[i] * t * t;
    s += num / (den * den);
  }
  return -warp_sum(s);
}

__device__ inline double phi_model_warp(double t, int p, const double* al, const double* be,
                                        const double* ga, const double* ze) {
  double s = 0.0;
  for (int i = threadIdx.x & 31; i < p; i += 32)
    s += (al[i] + 2.0 * ze[i] * t + ga[i] * t * t) / (1.0 + be[i] * t * t);
  return -0.5 * warp_sum(s);
}
// Brent-Dekker zero of phi' on [a, b] with phi'(a) phi'(b) <= 0 (R. P. Brent,
// Algorithms for Minimization without Derivatives, 1973, ch. 4): inverse
// quadratic / secant steps kept inside the bracket, bisection otherwise;
// stops when the bracket is below 2 eps |b|. Returns the root; *ev counts
// evaluations.
__device__ inline double brent_warp(double a, double b, double fa, double fb, int p, const double* al,
                        const double* be, const double* ga, const double* ze, int* ev) {
  if (fa == 0.0) return a;
  if (fb == 0.0) return b;
  double c = a, fc = fa, d = b - a, e = d;
  for (int it = 0; it < 100; ++it) {
    if ((fb > 0.0 && fc > 0.0) || (fb < 0.0 && fc < 0.0)) {
      c = a;
      fc = fa;
      d = e = b - a;
    }
    if (fabs(fc) < fabs(fb)) {
      a = b; b = c; c = a;
      fa = fb; fb = fc; fc = fa;
    }
    double tol = 2.0 * ALG3_EPS * fabs(b) + 1e-300;
    double m = 0.5 * (c - b);
    if (fabs(m) <= tol || fb == 0.0) break;
    if (fabs(e) >= tol && fabs(fa) > fabs(fb)) {
      double s = fb / fa, P, Q;
      if (a == c) {
        P = 2.0 * m * s;
        Q = 1.0 - s;
      } else {
        double q = fa / fc, r = fb / fc;
        P = s * (2.0 * m * q * (q - r) - (b - a) * (r - 1.0));
        Q = (q - 1.0) * (r - 1.0) * (s - 1.0);
      }
      if (P > 0.0) Q = -Q; else P = -P;
      if (2.0 * P < fmin(3.0 * m * Q - fabs(tol * Q), fabs(e * Q))) {
        e = d;
        d = P / Q;
      } else {
        d = m;
        e = m;
      }
    } else {
      d = m;
      e = m;
    }
    a = b;
    fa = fb;
    b = (fabs(d) > tol) ? b + d : b + copysign(tol, m);
    fb = dphi_warp(b, p, al, be, ga, ze);
    ++*ev;
  }
  return b;
}

// Alg. 3 generalised to zeta (Sec. 5.2). Bracket-eligible branches have
// beta_i > eps * sum(beta) and zeta_i > 0; xi_i from Eq. (derv1) (delta < 0)
// or Eq. (derv2) (delta >= 0) with zeta in the CG places. The step is the
// first minimiser of the model past xi_min: the right end is doubled from
// xi_min (capped at xi_max) until phi' >= 0, then Brent.
__device__ inline double get_mu_warp(int p, const double* al, const double* be, const double* ga,
                         const double* ze, int* ev) {
  double sb = 0.0;  // summed in index order by lane 0, then broadcast
  if ((threadIdx.x & 31) == 0)
    for (int i = 0; i < p; ++i) sb += be[i];
  sb = __shfl_sync(0xffffffffu, sb, 0);
  // the xi_i over the lanes (lane j takes j, j + 32, ...); min, max and
  // count are exact, so every lane ends with the same values
  double xmin = INFINITY, xmax = -INFINITY;
  int cnt = 0;
  for (int i = threadIdx.x & 31; i < p; i += 32) {
    double b = be[i], z = ze[i];
    if (!(b > ALG3_EPS * sb) || !(z > 0.0)) continue;
    double d = ga[i] - al[i] * b;
    double disc = sqrt(d * d + 4.0 * b * z * z);
    double xi = (d < 0.0) ? 2.0 * z / (-d + disc) : (d + disc) / (2.0 * b * z);
    xmin = fmin(xmin, xi);
    xmax = fmax(xmax, xi);
    ++cnt;
  }
  for (int o = 16; o > 0; o >>= 1) {
    xmin = fmin(xmin, __shfl_xor_sync(0xffffffffu, xmin, o));
    xmax = fmax(xmax, __shfl_xor_sync(0xffffffffu, xmax, o));
    cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  }
  *ev = 0;
  if (cnt == 0) return 0.0;
  double fa = dphi_warp(xmin, p, al, be, ga, ze);
  ++*ev;
  double lo, flo, hi, fhi;
  if (fa > 0.0) {
    lo = 0.0;
    flo = dphi_warp(0.0, p, al, be, ga, ze);
    ++*ev;
    if (flo >= 0.0) return 0.0;
    hi = xmin;
    fhi = fa;
  } else {
    lo = flo = hi = fhi = 0.0;
    lo = xmin; flo = fa; hi = xmin; fhi = fa;
    int k = 0;
    while (fhi < 0.0) {
      if (k >= 64) return hi;
      double nxt = 2.0 * hi;
      if (hi < xmax) nxt = fmin(nxt, xmax);
      lo = hi;
      flo = fhi;
      hi = nxt;
      fhi = dphi_warp(hi, p, al, be, ga, ze);
      ++*ev;
      ++k;
    }
  }
  return brent_warp(lo, hi, flo, fhi, p, al, be, ga, ze, ev);
}


}  // namespace gsi
