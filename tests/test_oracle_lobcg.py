"""Pins of the oracle's LOBCG comparator (Sec. 6.4, comparison to LOBCG) against
facts that do not depend on it: App. A's containment of the Riemannian CG
iterate in the LOBCG subspace and the resulting bound on phi, the p = 1 case
(one Rayleigh-Ritz step on span(x, g) is the exact steepest-descent step),
and convergence to the closed-form spectrum of FD Laplacians."""
import numpy as np

from oracle import gsi_oracle as O
from paper_2306_10379_gb300 import inputs as I


def _op(dims):
    A = I.fd_laplacian(dims)
    return A, O.csr_operator(A.n, A.rowptr, A.colidx, A.val), I.laplacian_eigenvalues(dims)


def _trace(S, X):
    return float(np.trace(X.T @ (S @ X)))


def test_rcg_iterate_lies_in_the_lobcg_subspace():
    """App. A: X_{k+1} of Riemannian CG lies in span(X_k, G_k, X_{k-1}), so the
    LOBCG step from the same (X_k, X_{k-1}) reaches at least its partial trace
    (phi(X_LOBCG) <= phi(X_RCG))."""
    A, S, lam = _op((16, 15))
    p = 4
    traj = []
    O.solve(S, I.start_block(A.n, p, I.SEED_BASE + 3), O.Options(method="cg", tol=0.0, max_iters=8,
                                                                 anorm=lam[0]),
            callback=lambda k, X, Y, t: traj.append(X.copy()))
    for k in (2, 4, 6):
        Xm1, Xk, Xk1 = traj[k - 1], traj[k], traj[k + 1]
        Y = S @ Xk
        C = Xk.T @ Y
        G = Y - Xk @ (0.5 * (C + C.T))
        Q, _ = O.block_basis([Xk, G, Xm1])
        assert np.max(np.abs(Q.T @ Q - np.eye(Q.shape[1]))) < 1e-12
        assert np.linalg.norm(Xk1 - Q @ (Q.T @ Xk1)) <= 1e-10 * np.linalg.norm(Xk1), k
        Xl, _ = O.lobcg_step(S, Xk, Xm1)
        assert np.max(np.abs(Xl.T @ Xl - np.eye(p))) < 1e-12
        assert _trace(S, Xl) >= _trace(S, Xk1) - 1e-12 * abs(_trace(S, Xk1)), k


def test_lobcg_first_step_for_p1_is_the_exact_sd_step():
    """p = 1 without a previous iterate: Rayleigh-Ritz on span(x, g) gives the
    maximiser of the Rayleigh quotient over that plane, which the exact line
    search of Alg. 2 / Alg. 3 also finds."""
    A, S, lam = _op((13, 11))
    x0 = I.start_block(A.n, 1, I.SEED_BASE + 5)
    traj = []
    O.solve(S, x0, O.Options(method="sd", tol=0.0, max_iters=1, anorm=lam[0]),
            callback=lambda k, X, Y, t: traj.append(X.copy()))
    xl, _ = O.lobcg_step(S, O.orthonormalize(x0))
    assert abs(abs(float(xl[:, 0] @ traj[0][:, 0])) - 1.0) < 1e-12


def test_lobcg_converges_to_the_closed_form_spectrum():
    """2D 20 x 18 Laplacian, p = 6: residual 1e-8 relative, Ritz values within
    the quadratic bound of the closed form, an orthonormal basis; and, as the
    paper reports for FD matrices, fewer iterations than Riemannian CG from the
    same start."""
    dims, p = (20, 18), 6
    A, S, lam = _op(dims)
    X0 = I.start_block(A.n, p, I.SEED_BASE + 9)
    res = O.lobcg_solve(S, X0, tol=1e-8, anorm=lam[0])
    assert res.converged
    X = res.X
    assert np.max(np.abs(X.T @ X - np.eye(p))) < 1e-12
    theta = np.sort(np.linalg.eigvalsh(X.T @ (S @ X)))[::-1]
    gap = lam[p - 1] - lam[p]
    assert np.max(np.abs(theta - lam[:p])) <= 2 * (1e-8 * lam[0]) ** 2 / gap + 1e-12 * lam[0]
    rcg = O.solve(S, X0, O.Options(method="cg", tol=1e-8, anorm=lam[0]))
    assert rcg.converged and res.iters < rcg.iters


def test_momentum_block_spans_the_same_subspace_as_the_previous_iterate():
    """The footnote's replacement of X_{k-1}: with P_k the part of X_k outside
    span(X_{k-1}), span(X_k, G_k, P_k) = span(X_k, G_k, X_{k-1}) (V_1 of X_k
    in the basis of the previous step is invertible), so a step from either
    gives the same next iterate (as a subspace and as Ritz values)."""
    dims, p = (16, 15), 5
    A, S, lam = _op(dims)
    X = O.orthonormalize(I.start_block(A.n, p, I.SEED_BASE + 4))
    Xm1, P = None, None
    for k in range(4):
        Xn, Pn = O.lobcg_step(S, X, P)
        if k >= 1:
            Y = S @ X
            G = Y - X @ (X.T @ Y)
            Qa, _ = O.block_basis([X, G, P])
            Qb, _ = O.block_basis([X, G, Xm1])
            assert Qa.shape[1] == Qb.shape[1] == 3 * p
            assert np.linalg.norm(Qb - Qa @ (Qa.T @ Qb), 2) < 1e-10  # sine of the largest angle
            Xa, _ = O.lobcg_step(S, X, Xm1)
            assert np.linalg.norm(Xa - Xn @ (Xn.T @ Xa), 2) < 1e-10
            assert abs(_trace(S, Xa) - _trace(S, Xn)) < 1e-12 * abs(_trace(S, Xn))
        Xm1, X, P = X, Xn, Pn
