"""CPU FP64 oracle for gradient-type subspace iteration (Alimisis, Saad &
Vandereycken, arXiv 2306.10379).

TEST INFRASTRUCTURE ONLY. Only the test-suite, the smoke check and the
CPU-baseline leg of the benchmark may import this module. The CUDA library
never calls it, shares no code with it, and must fail loudly rather than fall
back to it.

Plain, slow and direct: numpy / scipy.sparse library products serve as the
matrix products, numpy.linalg.eigh as the small symmetric eigensolver, and
everything else is written out in the order of the paper's algorithms. All
arithmetic is float64.

Sign convention. The paper writes G = grad phi = -(AX - XC) and steps
X - mu*G (Sec. 3, Eq. (gradPhi), Alg. 2). Here R = AX - XC (the residual,
= -G) and the step is X + t*D with t >= 0; the iterates are identical. With
this sign zeta_i = (V^T D^T A X V)_ii = (V^T D^T R V)_ii for tangent D (the
paper's D_zeta of Eq. (CG_linesearch_D) after the sign flip), and
zeta = beta for steepest descent (Eqs. (GTAY)-(GTG)).

Readings of points the paper leaves open:
  * stopping test ||R||_F / ||A||_2 <= tol, checked every iteration, or, as
    an option, the paper's table criterion ||R_k||_inf / ||R_0||_inf <= tol
    (largest row sum of |R|, Table "Comparison of LOBCG and Riemannian CG");
  * Brent-Dekker root finding on phi'(t) with tolerance 2 eps |t|, at most
    100 evaluations;
  * branches with beta_i <= eps * sum(beta) and, for CG, the concave branches
    (zeta_i <= 0) are left out of the bracket but kept in phi';
  * the step is the first minimiser of the model past xi_min: the bracket's
    right end is found by doubling from xi_min (capped at xi_max), lo <- 0
    when phi'(xi_min) > 0;
  * CG: first iteration and restarts use P = R; plain Polak-Ribiere beta;
    restart when <P, R> <= 0 or every k_restart iterations (0 = never);
  * zeta is taken from D^T R, and the polar factor from the measured Gram of
    X + tD (both equal the paper's expressions in exact arithmetic);
  * AX is recomputed explicitly when t*sqrt(beta_max) < 1e3*eps, every
    `recompute_every` iterations, and before the final residual;
  * LOBCG (the comparator of Sec. 6.4): X_{k-1} is replaced by the momentum
    block P_k of Knyazev's method (the part of X_k outside span(X_{k-1}); the
    paper's footnote says a better-conditioned block replaces X_{k-1} without
    naming it), which spans the same V_k; the basis of span(X_k, G_k, P_k) is
    built block by block from Gram matrices (the paper's implementation
    orthonormalises by Cholesky) with rank truncation at 1e-7 of each block's
    largest singular value; the Rayleigh-Ritz matrix Q^T A Q is formed
    explicitly (the paper's LOBCG(+));
  * complex Hermitian A (the footnote to Eq. (phi)): the same steps in
    complex arithmetic, inner products by their real part, the line-search
    coefficients the real diagonals of V^H {C, Gamma, Z} V;
  * subspace tracking (the slowly varying operators of Sec. 1): each operator
    of a sequence is solved from the previous one's final iterate, which the
    solve orthonormalises again like any start block; the CG state (direction,
    previous residual) starts afresh for every operator.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

EPS = np.finfo(np.float64).eps


# ---------------------------------------------------------------------------
# Operator and block products (Sec. 6.1, "Efficient matvecs")
# ---------------------------------------------------------------------------

def csr_operator(n, rowptr, colidx, val):
    """scipy CSR matrix from plain CSR arrays."""
    return sp.csr_matrix((np.asarray(val, np.float64), np.asarray(colidx, np.int64),
                          np.asarray(rowptr, np.int64)), shape=(n, n))


def spmm(A, X):
    """Block matvec W = A X (one per iteration in the paper's accounting)."""
    return np.asarray(A @ X)


def gram(U, V):
    """Tall-skinny Gram product U^T V (p x p)."""
    return U.T @ V


def residual(X, Y, C):
    """R = AX - XC with Y = AX and C = X^T A X (Eq. (gradPhi), sign flipped)."""
    return Y - X @ C


def anorm_inf(A):
    """||A||_inf = max absolute row sum, an upper bound of ||A||_2."""
    return float(np.max(np.asarray(abs(A).sum(axis=1)).ravel()))


# ---------------------------------------------------------------------------
# Line search (Sec. 3.1 Eqs. (Gdec)-(xii), Sec. 5.2 Eqs. (phi_P)-(deriv_P),
# Sec. 6.1 Eqs. (derv1)-(derv2), Alg. 3)
# ---------------------------------------------------------------------------

def ls_coefficients(C, B, Gamma, Z):
    """Diagonalise B = D^T D = V diag(beta) V^T (Eq. (Gdec)) and return
    alpha = diag(V^T C V), beta, gamma = diag(V^T Gamma V),
    zeta = diag(V^T Z V) (Eqs. (diags), (CG_linesearch_D)), and V."""
    Bs = 0.5 * (B + B.T)
    beta, V = np.linalg.eigh(Bs)
    beta = np.maximum(beta, 0.0)
    alpha = np.einsum("ki,kl,li->i", V, C, V)
    gamma = np.einsum("ki,kl,li->i", V, Gamma, V)
    zeta = np.einsum("ki,kl,li->i", V, Z, V)
    return alpha, beta, gamma, zeta, V


def phi_model(t, alpha, beta, gamma, zeta):
    """phi(X(t)) = -1/2 sum (alpha_i + 2 zeta_i t + gamma_i t^2)/(1 + beta_i t^2),
    Eq. (phi_P) (Eq. (phinew) when zeta = beta)."""
    return -0.5 * float(np.sum((alpha + 2.0 * zeta * t + gamma * t * t) / (1.0 + beta * t * t)))


def dphi_model(t, alpha, beta, gamma, zeta):
    """phi'(t) = -sum (zeta_i + (gamma_i - alpha_i beta_i) t - beta_i zeta_i t^2)
    / (1 + beta_i t^2)^2, Eq. (deriv_P) (Eq. (dqnew) when zeta = beta).
    The sum runs over i in ascending order."""
    num = zeta + (gamma - alpha * beta) * t - beta * zeta * t * t
    den = (1.0 + beta * t * t) ** 2
    return -float(np.sum(num / den))


def branch_roots(alpha, beta, gamma, zeta):
    """Positive root xi_i of each bracket-eligible branch numerator
    zeta_i + delta_i t - beta_i zeta_i t^2, delta_i = gamma_i - alpha_i beta_i,
    in the cancellation-free forms of Eqs. (derv1) (delta_i < 0) and (derv2)
    (delta_i >= 0), written with zeta_i in place of beta_i where the CG
    generalisation puts it. Eligible: beta_i > eps*sum(beta) and zeta_i > 0
    (concave branches are ignored for the bracket, Sec. 5.2)."""
    sb = float(np.sum(beta))
    xs = []
    for a, b, g, z in zip(alpha, beta, gamma, zeta):
        if not (b > EPS * sb) or not (z > 0.0):
            continue
        d = g - a * b
        disc = math.sqrt(d * d + 4.0 * b * z * z)
        if d < 0.0:
            xs.append(2.0 * z / (-d + disc))
        else:
            xs.append((d + disc) / (2.0 * b * z))
    return np.array(xs)


def brent_zero(f, a, b, fa, fb, maxeval=100):
    """Dekker-Brent safeguarded root finder (R. P. Brent, Algorithms for
    Minimization without Derivatives, 1973, ch. 4), for f(a) f(b) <= 0.

    Keeps a bracket [b, c] with f(b) f(c) <= 0 and |f(b)| <= |f(c)|, tries
    inverse quadratic interpolation (secant with two points) and accepts it
    only while it stays inside the bracket and shrinks fast enough; otherwise
    bisects. Stops when the bracket half-width is below 2 eps |b| (+ tiny).
    Returns (root, evaluations)."""
    evals = 0
    if fa == 0.0:
        return a, evals
    if fb == 0.0:
        return b, evals
    c, fc = a, fa
    e = d = b - a
    while evals < maxeval:
        if (fb > 0.0 and fc > 0.0) or (fb < 0.0 and fc < 0.0):
            c, fc = a, fa
            e = d = b - a
        if abs(fc) < abs(fb):
            a, b, c = b, c, b
            fa, fb, fc = fb, fc, fb
        tol = 2.0 * EPS * abs(b) + 1e-300
        m = 0.5 * (c - b)
        if abs(m) <= tol or fb == 0.0:
            break
        if abs(e) >= tol and abs(fa) > abs(fb):
            s = fb / fa
            if a == c:
                pq_p = 2.0 * m * s
                pq_q = 1.0 - s
            else:
                q = fa / fc
                r = fb / fc
                pq_p = s * (2.0 * m * q * (q - r) - (b - a) * (r - 1.0))
                pq_q = (q - 1.0) * (r - 1.0) * (s - 1.0)
            if pq_p > 0:
                pq_q = -pq_q
            else:
                pq_p = -pq_p
            if 2.0 * pq_p < min(3.0 * m * pq_q - abs(tol * pq_q), abs(e * pq_q)):
                e, d = d, pq_p / pq_q
            else:
                d = e = m
        else:
            d = e = m
        a, fa = b, fb
        b = b + d if abs(d) > tol else b + math.copysign(tol, m)
        fb = f(b)
        evals += 1
    return b, evals


def get_mu(alpha, beta, gamma, zeta, max_doublings=64):
    """Alg. 3 (Get_Mu), generalised to zeta for CG (Sec. 5.2).

    phi' < 0 on [0, xi_min] (every eligible branch still descends), so the
    search starts at xi_min. The bracket's right end is found by doubling from
    xi_min (capped at xi_max on the first pass) until phi' >= 0, and Brent then
    finds the root of phi' in [lo, hi]: the first local minimiser of the
    model past xi_min. A branch whose beta_i sits at rounding level has no
    relative accuracy and can put a spurious root of phi' far beyond the main
    minimum; stopping at the first sign change keeps the step where the model
    is accurate. If phi'(xi_min) > 0 (possible for CG) the search runs on
    [0, xi_min]; if phi'(0) >= 0 the direction is not a descent direction and
    t = 0. Returns (t, evaluations, lo, hi)."""
    xs = branch_roots(alpha, beta, gamma, zeta)
    if xs.size == 0:
        return 0.0, 0, 0.0, 0.0
    f = lambda t: dphi_model(t, alpha, beta, gamma, zeta)
    xmin, xmax = float(xs.min()), float(xs.max())
    fa = f(xmin)
    evals = 1
    if fa > 0.0:
        lo, flo = 0.0, f(0.0)
        evals += 1
        if flo >= 0.0:
            return 0.0, evals, 0.0, xmin
        hi, fhi = xmin, fa
    else:
        lo, flo = xmin, fa
        hi, fhi = xmin, fa
        k = 0
        while fhi < 0.0:
            if k >= max_doublings:
                return hi, evals, lo, hi
            nxt = 2.0 * hi
            if hi < xmax:
                nxt = min(nxt, xmax)
            lo, flo = hi, fhi
            hi = nxt
            fhi = f(hi)
            evals += 1
            k += 1
    t, ev = brent_zero(f, lo, hi, flo, fhi)
    return t, evals + ev, lo, hi


def polar_factor_matrix(V, beta, t):
    """M = V (I + t^2 D_beta)^{-1/2} V^T, so that (X + tD) M is the polar
    factor of X + tD (Eqs. (Psi3), (Ynew), (Xnew_P))."""
    d = 1.0 / np.sqrt(1.0 + t * t * beta)
    return (V * d) @ V.T


def inverse_sqrt(S):
    """S^{-1/2} of a symmetric positive definite p x p matrix (eigh).

    The retraction uses M = (Z^T Z)^{-1/2} with Z = X + tD and the Gram
    Z^T Z measured, so that Z M is the polar factor of Z (Eq. (Ynew)). In
    exact arithmetic Z^T Z = I + t^2 D^T D and M = V D_t^{-1} V^T; in floating
    point the measured Gram keeps X orthonormal, while the analytic form lets
    ||X^T X - I|| grow by about |1 - 2 t lambda| per step (the residual
    R = Y - XC is tangent only up to (X^T X - I) C)."""
    s, U = np.linalg.eigh(0.5 * (S + S.T))
    return (U / np.sqrt(s)) @ U.T


# ---------------------------------------------------------------------------
# Start block, Rayleigh-Ritz, diagnostics
# ---------------------------------------------------------------------------

def orthonormalize(X0):
    """Polar orthonormalisation X0 (X0^T X0)^{-1/2}, applied twice (the second
    pass removes the rounding left by the first), via eigh of the Gram."""
    X = np.array(X0, dtype=np.float64)
    for _ in range(2):
        s, U = np.linalg.eigh(X.T @ X)
        X = X @ ((U / np.sqrt(s)) @ U.T)
    return X


def rayleigh_ritz(X, Y):
    """Ritz pairs of span(X) with Y = AX: C = X^T Y = U diag(theta) U^T,
    Ritz vectors XU, values theta in descending order (Eq. (rr1))."""
    C = X.T @ Y
    theta, U = np.linalg.eigh(0.5 * (C + C.T))
    order = np.argsort(theta)[::-1]
    return theta[order], X @ U[:, order], U[:, order]


def principal_angles(X, U):
    """Principal angles between span(X) and span(U), both orthonormal: the
    cosines are the singular values of X^T U."""
    s = np.linalg.svd(X.T @ U, compute_uv=False)
    return np.arccos(np.clip(s, -1.0, 1.0))


# ---------------------------------------------------------------------------
# Riemannian steepest descent (Alg. 2) and conjugate gradients (Alg. 4)
# ---------------------------------------------------------------------------

@dataclass
class Options:
    method: str = "sd"              # "sd" (Alg. 2) or "cg" (Alg. 4)
    tol: float = 1e-8               # on ||R||_F / anorm
    anorm: float = 0.0              # 0 -> ||A||_inf
    max_iters: int = 10000
    k_restart: int = 0              # 0 = never
    recompute_every: int = 50
    explicit_ax: bool = False       # RCG(+): explicit AX every iteration
    stop_rule: str = "fro"          # "fro": ||R||_F / anorm; "inf": ||R_k||_inf / ||R_0||_inf


@dataclass
class IterRecord:
    k: int
    t: float
    phi: float
    res_f: float
    res_inf: float
    evals: int
    restarted: bool


@dataclass
class Result:
    X: np.ndarray
    Y: np.ndarray
    iters: int
    matvecs: int
    converged: bool
    rel_residual: float
    restarts: int
    history: list = field(default_factory=list)


def solve(A, X0, opts: Options, record=False, callback=None):
    """Run Alg. 2 (opts.method == "sd") or Alg. 4 ("cg") from X0.

    Per iteration k (all quantities float64):
      R = Y - X C, C = X^T Y                          (Eq. (gradPhi))
      stop if ||R||_F <= tol * anorm
      D = R (SD); CG: D = R + beta_PR (P - X (X^T P)) (Eq. (Pnew) with the
          projection transport), restart to D = R when <D, R> <= 0 or every
          k_restart iterations
      W = A D                                          (the one block matvec)
      B = D^T D, Gamma = D^T W, Z = D^T R (= D^T A X for tangent D, the
          identity used in Sec. 5.2; Z = B for SD by Eqs. (GTAY)-(GTG)). D^T Y
          itself would carry (D^T X) C, a rounding-level term that swamps
          <D, R> once ||R|| < sqrt(eps) ||A||
      t = Get_Mu(alpha, beta, gamma, zeta)             (Alg. 3)
      M = (Z^T Z)^{-1/2}, Z = X + tD, the polar factor  (Eq. (Ynew), Eq. (Xnew_P))
      X <- Z M,  Y <- (Y + tW) M                       (Eq. (save_matvec))
    """
    n, p = X0.shape
    anorm = opts.anorm if opts.anorm > 0 else anorm_inf(A)
    X = orthonormalize(X0)
    Y = spmm(A, X)
    matvecs = 1
    P = None
    R_prev = None
    rr_prev = None
    restarts = 0
    history = []
    res0_inf = None
    converged = False
    y_fresh = True
    k = 0
    rel = float("nan")
    while True:
        C = gram(X, Y)
        C = 0.5 * (C + C.T)
        R = residual(X, Y, C)
        rr = float(np.sum(R * R))
        rel = math.sqrt(rr) / anorm
        res_inf = float(np.max(np.sum(np.abs(R), axis=1)))
        if res0_inf is None:
            res0_inf = res_inf
        crit = rel if opts.stop_rule == "fro" else res_inf / res0_inf
        if crit <= opts.tol or k >= opts.max_iters:
            if not y_fresh:
                # the final residual is always taken with an explicit AX
                Y = spmm(A, X)
                matvecs += 1
                y_fresh = True
                continue
            converged = crit <= opts.tol
            break
        restarted = False
        if opts.method == "sd" or P is None:
            D = R
        else:
            beta_pr = (rr - float(np.sum(R * R_prev))) / rr_prev
            Kp = gram(X, P)
            D = R + beta_pr * (P - X @ Kp)
            due = opts.k_restart > 0 and k % opts.k_restart == 0
            if due or float(np.sum(D * R)) <= 0.0:
                D = R
                restarted = True
        if restarted:
            restarts += 1
        W = spmm(A, D)
        matvecs += 1
        B = gram(D, D)
        Gam = gram(D, W)
        Z = B if opts.method == "sd" else gram(D, R)
        alpha, beta, gamma, zeta, V = ls_coefficients(C, B, 0.5 * (Gam + Gam.T), Z)
        t, evals, _, _ = get_mu(alpha, beta, gamma, zeta)
        Zt = X + t * D
        M = inverse_sqrt(gram(Zt, Zt))
        X = Zt @ M
        recompute = (opts.explicit_ax or t * math.sqrt(max(beta.max(), 0.0)) < 1e3 * EPS
                     or (opts.recompute_every > 0 and (k + 1) % opts.recompute_every == 0))
        if recompute:
            Y = spmm(A, X)
            matvecs += 1
        else:
            Y = (Y + t * W) @ M
        y_fresh = recompute
        if record:
            history.append(IterRecord(k, t, phi_model(t, alpha, beta, gamma, zeta),
                                      math.sqrt(rr), res_inf / res0_inf, evals, restarted))
        if callback is not None:
            callback(k, X, Y, t)
        P, R_prev, rr_prev = D, R, rr
        k += 1
    return Result(X, Y, k, matvecs, converged, rel, restarts, history)


def solve_hermitian(A, X0, opts: Options):
    """Alg. 2 / Alg. 4 for a complex Hermitian A (the paper's footnote to
    Eq. (phi): minimise -1/2 Re tr(X^H A X) over X^H X = I), in complex128,
    step for step as solve(): transposes become conjugate transposes, inner
    products take their real part (Re <U, V> = Re tr(U^H V)), B = D^H D is
    diagonalised by a unitary V and alpha, beta, gamma, zeta are the real
    diagonals Re diag(V^H {C, Gamma, Z} V) of Hermitian (C, Gamma) or
    general (Z = D^H R) matrices; Get_Mu, the polar retraction and the AX
    recursion are unchanged. A: scipy sparse or dense complex, Hermitian;
    X0: complex n x p."""
    def herm(M):
        return 0.5 * (M + M.conj().T)

    def inv_sqrt_h(S):
        s, U = np.linalg.eigh(herm(S))
        return (U / np.sqrt(s)) @ U.conj().T

    def rdot(U, V):
        return float(np.real(np.vdot(U, V)))

    n, p = X0.shape
    anorm = opts.anorm if opts.anorm > 0 else float(abs(A).sum(axis=1).max())
    X = np.array(X0, dtype=np.complex128)
    for _ in range(2):
        X = X @ inv_sqrt_h(X.conj().T @ X)
    Y = A @ X
    matvecs = 1
    P = R_prev = rr_prev = None
    restarts = 0
    y_fresh = True
    k = 0
    rel = float("nan")
    while True:
        C = herm(X.conj().T @ Y)
        R = Y - X @ C
        rr = rdot(R, R)
        rel = math.sqrt(rr) / anorm
        if rel <= opts.tol or k >= opts.max_iters:
            if not y_fresh:
                Y = A @ X
                matvecs += 1
                y_fresh = True
                continue
            break
        restarted = False
        if opts.method == "sd" or P is None:
            D = R
        else:
            beta_pr = (rr - rdot(R, R_prev)) / rr_prev
            D = R + beta_pr * (P - X @ (X.conj().T @ P))
            due = opts.k_restart > 0 and k % opts.k_restart == 0
            if due or rdot(D, R) <= 0.0:
                D = R
                restarted = True
        restarts += int(restarted)
        W = A @ D
        matvecs += 1
        B = D.conj().T @ D
        Gam = herm(D.conj().T @ W)
        Z = B if opts.method == "sd" else D.conj().T @ R
        beta, V = np.linalg.eigh(herm(B))
        beta = np.maximum(beta, 0.0)
        alpha = np.real(np.einsum("ki,kl,li->i", V.conj(), C, V))
        gamma = np.real(np.einsum("ki,kl,li->i", V.conj(), Gam, V))
        zeta = np.real(np.einsum("ki,kl,li->i", V.conj(), Z, V))
        t, _, _, _ = get_mu(alpha, beta, gamma, zeta)
        Zt = X + t * D
        M = inv_sqrt_h(Zt.conj().T @ Zt)
        X = Zt @ M
        recompute = (opts.explicit_ax or t * math.sqrt(max(beta.max(), 0.0)) < 1e3 * EPS
                     or (opts.recompute_every > 0 and (k + 1) % opts.recompute_every == 0))
        if recompute:
            Y = A @ X
            matvecs += 1
        else:
            Y = (Y + t * W) @ M
        y_fresh = recompute
        P, R_prev, rr_prev = D, R, rr
        k += 1
    return Result(X, Y, k, matvecs, rel <= opts.tol, rel, restarts)


def track(mats, X0, opts: Options, anorms=None):
    """Subspace tracking over a sequence of operators A_0, A_1, ... (Sec. 1:
    eigenspaces of slowly varying matrices, as in self-consistent-field
    iterations): A_0 is solved from X0, every later A_k from the final
    iterate X of A_{k-1}. Returns the list of Results."""
    out = []
    X = X0
    for k, A in enumerate(mats):
        o = opts if anorms is None else Options(**{**opts.__dict__, "anorm": float(anorms[k])})
        r = solve(A, X, o)
        out.append(r)
        X = r.X
    return out


# ---------------------------------------------------------------------------
# LOBCG comparator (Sec. 6.4, "Comparison to LOBCG"; Knyazev 2001)
# ---------------------------------------------------------------------------

LOBCG_RANK_TOL = 1e-7


def block_basis(blocks, rank_tol=LOBCG_RANK_TOL):
    """Orthonormal basis of the column span of the blocks, built block by
    block as the paper's implementation does it, by orthonormalisations of
    Gram matrices (Sec. 6.4: three per iteration, by Cholesky): each block B
    is projected off the basis so far (twice); with its Gram
    S = B^T B = U diag(s) U^T (eigenvalues descending), B U_r diag(s_r)^(-1/2)
    over the eigenvalues s_i > rank_tol^2 s_1 spans what is left of B (its
    singular values above rank_tol times the largest), and a second pass
    Q <- Q (Q^T Q)^(-1/2) restores orthonormality to rounding level. A Gram
    resolves singular values down to about sqrt(eps) of the largest, hence
    rank_tol = 1e-7. Returns (Q, widths)."""
    Q = np.zeros((blocks[0].shape[0], 0))
    widths = []
    for B in blocks:
        for _ in range(2):
            B = B - Q @ (Q.T @ B)
        s, U = np.linalg.eigh(B.T @ B)
        s, U = s[::-1], U[:, ::-1]
        keep = s > rank_tol ** 2 * s[0] if s[0] > 0.0 else np.zeros(s.size, bool)
        Qb = B @ (U[:, keep] / np.sqrt(s[keep]))
        if Qb.shape[1]:
            Qb = Qb @ inverse_sqrt(Qb.T @ Qb)
        Q = np.hstack([Q, Qb])
        widths.append(Qb.shape[1])
    return Q, widths


def lobcg_step(A, X, W=None):
    """One LOBCG step: the Rayleigh-Ritz procedure for A on
    V_k = span(X_k, G_k, W) (Eq. (def_Vk_LOBPCG)), G_k = A X_k - X_k C_k the
    gradient direction and W the momentum block: X_{k-1} itself, or -- the
    better-conditioned block the paper's footnote to that equation refers to
    (Knyazev 2001) -- P_k, the part of X_k outside span(X_{k-1}) from the
    previous step; both give the same V_k. The next iterate is the Ritz
    vectors of the p largest Ritz values (the maximisation of the partial
    trace; the minimum problem runs on -A as in Sec. 2.1). Returns
    (X_{k+1}, P_{k+1}), P_{k+1} = X_{k+1} minus its component in span(X_k)."""
    Y = spmm(A, X)
    C = gram(X, Y)
    G = Y - X @ (0.5 * (C + C.T))
    Q, widths = block_basis([X, G] + ([W] if W is not None else []))
    H = gram(Q, spmm(A, Q))
    w, V = np.linalg.eigh(0.5 * (H + H.T))
    V = V[:, np.argsort(w)[::-1][:X.shape[1]]]
    w1 = widths[0]
    return Q @ V, Q[:, w1:] @ V[w1:, :]


def lobcg_solve(A, X0, tol=1e-8, anorm=0.0, max_iters=10000, record=False, stop_rule="fro"):
    """LOBCG from the orthonormalised X0: (X_{k+1}, P_{k+1}) =
    lobcg_step(A, X_k, P_k) (no momentum block in the first step), with the
    stopping tests of solve(): ||A X_k - X_k C_k||_F <= tol * anorm, or
    (stop_rule "inf") ||R_k||_inf / ||R_0||_inf <= tol. record: the Result's
    history holds each iterate X_k (k >= 1)."""
    anorm = anorm if anorm > 0 else anorm_inf(A)
    X = orthonormalize(X0)
    P = None
    k = 0
    hist = []
    res0_inf = None
    while True:
        Y = spmm(A, X)
        C = gram(X, Y)
        R = residual(X, Y, 0.5 * (C + C.T))
        rel = math.sqrt(float(np.sum(R * R))) / anorm
        res_inf = float(np.max(np.sum(np.abs(R), axis=1)))
        if res0_inf is None:
            res0_inf = res_inf
        crit = rel if stop_rule == "fro" else res_inf / res0_inf
        if crit <= tol or k >= max_iters:
            break
        X, P = lobcg_step(A, X, P)
        if record:
            hist.append(X.copy())
        k += 1
    return Result(X, Y, k, k + 1, crit <= tol, rel, 0, hist)


# ---------------------------------------------------------------------------
# Chebyshev-filtered subspace iteration (Alg. 1 with Eq. (optimal_poly))
# ---------------------------------------------------------------------------

def chebyshev_filter(A, X, degree, c, h, scale_at):
    """Z = C_d((A - cI)/h) X / C_d((scale_at - c)/h) by the three-term
    recurrence T_{k+1} = 2 s T_k - T_{k-1}, s = (A - cI)/h, with each step
    divided by the running scale ratio so the top of the spectrum stays O(1)
    (the scaling at lambda_1 of Sec. 2.2)."""
    e = (scale_at - c) / h
    sigma = 1.0 / e
    Z_prev = X
    Z = (spmm(A, X) - c * X) * (sigma / h)
    for _ in range(1, degree):
        sigma_next = 1.0 / (2.0 * e - sigma)
        Z_next = (2.0 * sigma_next / h) * (spmm(A, Z) - c * Z) - (sigma * sigma_next) * Z_prev
        Z_prev, Z, sigma = Z, Z_next, sigma_next
    return Z


def chebyshev_si(A, X0, degree, lam_p1, lam_n, lam_1, tol=1e-8, anorm=0.0, max_outer=10000,
                 adaptive=False, guard=0):
    """Alg. 1 with p_k = C_d((t - c)/h), c = (lam_{p+1} + lam_n)/2,
    h = (lam_{p+1} - lam_n)/2, scaled at lam_1 (Eq. (optimal_poly)); an
    orthonormalisation and Rayleigh-Ritz after every `degree` matvecs.
    lam_p1 may be any estimate of the unwanted interval's upper end, e.g.
    lam_{p+k} (the remark after Eq. (optimal_poly)). adaptive: the bounds
    follow the Ritz values of each Rayleigh-Ritz step instead (the practice
    the paper notes in Sec. 6.2): upper end of the unwanted interval the
    smallest Ritz value of the block, scaling point the largest, lam_n kept
    as the given lower bound of the spectrum. guard: the trailing Ritz pairs
    (smallest Ritz values) left out of the stopping test -- guard vectors,
    which keep the filter's upper end below the wanted eigenvalues.
    Returns (X, theta, outer iterations, matvecs, rel residual)."""
    anorm = anorm if anorm > 0 else anorm_inf(A)
    c = 0.5 * (lam_p1 + lam_n)
    h = 0.5 * (lam_p1 - lam_n)
    X = orthonormalize(X0)
    matvecs = 0
    rel = float("nan")
    for outer in range(max_outer + 1):
        Y = spmm(A, X)
        matvecs += 1
        theta, Xr, U = rayleigh_ritz(X, Y)
        Yr = Y @ U
        R = Yr - Xr * theta
        rel = float(np.linalg.norm(R[:, :R.shape[1] - guard])) / anorm
        X = Xr
        if rel <= tol or outer == max_outer:
            return X, theta, outer, matvecs, rel
        if adaptive:
            hi, lam_1 = float(np.min(theta)), float(np.max(theta))
            c, h = 0.5 * (hi + lam_n), 0.5 * (hi - lam_n)
        Z = chebyshev_filter(A, X, degree, c, h, lam_1)
        matvecs += degree
        Q, _ = np.linalg.qr(Z)
        X = Q
    return X, theta, max_outer, matvecs, rel


# ---------------------------------------------------------------------------
# SELL-C-sigma (sliced ELLPACK) layout of a CSR matrix
# ---------------------------------------------------------------------------

def sell_c_sigma(n, rowptr, colidx, val, C=32, sigma=32):
    """Sliced ELLPACK with chunk height C and sorting window sigma.

    Within each window of sigma consecutive rows, rows are ordered by nnz
    descending, ties by ascending row index. Consecutive groups of C permuted
    rows form a chunk whose width is its longest row; chunk storage is
    column-major (entry j of the C rows, then entry j+1, ...). Padding slots
    hold the row's own index as column and 0.0 as value; rows past n in the
    last chunk are padding rows with perm = -1.
    Returns (perm, chunk_ptr, chunk_len, sell_col, sell_val):
    perm[k] = original row at permuted position k."""
    rowptr = np.asarray(rowptr, np.int64)
    lens = np.diff(rowptr)
    perm = []
    for w0 in range(0, n, sigma):
        rows = list(range(w0, min(n, w0 + sigma)))
        rows.sort(key=lambda r: (-int(lens[r]), r))
        perm.extend(rows)
    nchunks = (n + C - 1) // C
    perm = perm + [-1] * (nchunks * C - n)
    chunk_len = np.zeros(nchunks, np.int64)
    for ch in range(nchunks):
        rows = [r for r in perm[ch * C:(ch + 1) * C] if r >= 0]
        chunk_len[ch] = max(int(lens[r]) for r in rows)
    chunk_ptr = np.zeros(nchunks + 1, np.int64)
    chunk_ptr[1:] = np.cumsum(chunk_len * C)
    scol = np.zeros(int(chunk_ptr[-1]), np.int32)
    sval = np.zeros(int(chunk_ptr[-1]), np.float64)
    for ch in range(nchunks):
        base = int(chunk_ptr[ch])
        for lane in range(C):
            r = perm[ch * C + lane]
            for j in range(int(chunk_len[ch])):
                slot = base + j * C + lane
                if r >= 0 and j < lens[r]:
                    scol[slot] = colidx[rowptr[r] + j]
                    sval[slot] = val[rowptr[r] + j]
                else:
                    scol[slot] = max(r, 0) if r >= 0 else 0
                    sval[slot] = 0.0
    return np.array(perm, np.int64), chunk_ptr, chunk_len, scol, sval


# ---------------------------------------------------------------------------
# Batches of independent problems. The paper solves one problem at a time;
# a batch is just that method applied to each problem (Sec. 2.1 problem
# statement per A_i), and the GPU's work tables are plain integer
# bookkeeping with the definition written out here.
# ---------------------------------------------------------------------------

def batched_plan(n, p, tile_max, target_tiles, active=None):
    """Problem order (descending p, then descending n, then ascending index)
    and the tile table of one pass over the problems with active[i] (all
    when active is None): with S their total rows and T = ceil(S /
    target_tiles), problem i is cut into tiles of
    T_i = min(tile_max, max(64, T)) consecutive rows, the last
    one ragged. Returns (order, tiles), tiles a list of (problem, first row,
    rows)."""
    order = sorted(range(len(n)), key=lambda i: (-int(p[i]), -int(n[i]), i))
    on = [True] * len(n) if active is None else [bool(a) for a in active]
    S = sum(int(n[i]) for i in range(len(n)) if on[i])
    T = -(-S // int(target_tiles)) if S > 0 else 1
    tiles = []
    for i in order:
        if not on[i]:
            continue
        Ti = min(int(tile_max), max(64, T))
        r = 0
        while r < int(n[i]):
            tiles.append((i, r, min(Ti, int(n[i]) - r)))
            r += Ti
    return order, tiles


def batched_solve(mats, X0s, opts: Options, anorms=None, callback=None):
    """solve() on every problem of a batch, independently. mats[i] is a
    scipy sparse matrix, X0s[i] its start block; anorms[i] (optional) the
    norm of the stopping test. callback(i, k, X, Y, t) as in solve()."""
    out = []
    for i, (A, X0) in enumerate(zip(mats, X0s)):
        o = Options(**{**opts.__dict__})
        if anorms is not None:
            o.anorm = float(anorms[i])
        cb = None if callback is None else (lambda k, X, Y, t, i=i: callback(i, k, X, Y, t))
        out.append(solve(A, X0, o, callback=cb))
    return out


# ---------------------------------------------------------------------------
# Learned warm start. The paper motivates warm starts from related problems
# (Sec. 1, subspace iteration reused across a sequence of operators) but
# prints no network; what follows is the plain definition of each piece:
# a coarse basis C (m x p on an nc x nc grid) mapped to the fine grid by
# bilinear prolongation P, a multilayer perceptron producing C from the 16
# field coefficients, the subspace loss of span(P C) against the plain
# method's converged basis U, its gradient, and the Adam update.
# ---------------------------------------------------------------------------

def prolongation_1d(nc, nf):
    """P1 (nf x nc): hat-function interpolation from nc interior coarse nodes
    at (a+1)/(nc+1) to nf interior fine nodes at (i+1)/(nf+1) on [0, 1] with
    zero boundary values."""
    xf = (np.arange(nf) + 1.0) / (nf + 1)
    xc = (np.arange(nc) + 1.0) / (nc + 1)
    return np.maximum(0.0, 1.0 - np.abs(xf[:, None] - xc[None, :]) * (nc + 1))


def prolongation(nc, nf):
    """Bilinear prolongation P = P1 (x) P1 (nf^2 x nc^2, scipy CSR), fine node
    (i, j) at row i + nf j, coarse node (a, b) at column a + nc b (the
    ordering of the 5-point operators)."""
    P1 = sp.csr_matrix(prolongation_1d(nc, nf))
    return sp.kron(P1, P1, format="csr")


def bf16_round(x):
    """float32(x) rounded to bfloat16 (nearest, ties to even), as float64."""
    f = np.ascontiguousarray(np.asarray(x, np.float64).astype(np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def mlp_init(din, hidden, dout, seed):
    """The network's seeded initial weights (a seeded input, shared with the
    library's callers: paper_2306_10379_gb300.inputs.mlp_init)."""
    from paper_2306_10379_gb300.inputs import mlp_init as _init
    return _init(din, hidden, dout, seed)


def mlp_forward(prm, x, bf16=True):
    """out = W3 r(W2 r(W1 x + b1) + b2) + b3 for a batch x (B x din), r = ReLU.
    With bf16, every product's operands are rounded to bfloat16 (weights and
    the layer inputs); sums and biases in float64. Returns (out, cache)."""
    q = bf16_round if bf16 else (lambda a: np.asarray(a, np.float64))
    a0 = q(x)
    z1 = a0 @ q(prm["W1"]).T + prm["b1"]
    h1 = np.maximum(z1, 0.0)
    a1 = q(h1)
    z2 = a1 @ q(prm["W2"]).T + prm["b2"]
    h2 = np.maximum(z2, 0.0)
    a2 = q(h2)
    out = a2 @ q(prm["W3"]).T + prm["b3"]
    return out, (a0, z1, a1, z2, a2)


def mlp_backward(prm, cache, dout, bf16=True):
    """Gradients of sum(out * dout) w.r.t. the parameters (backpropagation
    through the three layers; with bf16 the products' operands -- the
    incoming gradient, weights and layer inputs -- rounded to bfloat16)."""
    q = bf16_round if bf16 else (lambda a: np.asarray(a, np.float64))
    a0, z1, a1, z2, a2 = cache
    g3 = q(dout)
    grads = {"W3": g3.T @ a2, "b3": np.asarray(dout, np.float64).sum(0)}
    d2 = (g3 @ q(prm["W3"])) * (z2 > 0)
    g2 = q(d2)
    grads["W2"] = g2.T @ a1
    grads["b2"] = d2.sum(0)
    d1 = (g2 @ q(prm["W2"])) * (z1 > 0)
    g1 = q(d1)
    grads["W1"] = g1.T @ a0
    grads["b1"] = d1.sum(0)
    return grads


def warm_loss_grad(C, S, Bt):
    """Subspace loss of one sample and its gradient w.r.t. the coarse basis C
    (m x p): with X = P C, N = X^T X = C^T S C (S = P^T P), Bt = P^T U (U the
    plain method's orthonormal n x p basis), Q = C^T Bt Bt^T C,
        L = p - tr(N^{-1} Q) = sum of sin^2 of the principal angles between
            span(X) and span(U),
        dL/dC = -2 [Bt (Bt^T C) N^{-1} - S C N^{-1} Q N^{-1}]."""
    C = np.asarray(C, np.float64)
    p = C.shape[1]
    SC = S @ C
    N = C.T @ SC
    G = Bt.T @ C
    Q = G.T @ G
    Ni = np.linalg.inv(N)
    L = p - float(np.trace(Ni @ Q))
    dC = -2.0 * (Bt @ (G @ Ni) - SC @ (Ni @ Q @ Ni))
    return L, dC


def adam_step(w, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015) at step t >= 1; returns (w, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v
