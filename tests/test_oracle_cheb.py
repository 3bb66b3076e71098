"""Pins of the oracle's filter variants (Sec. 2.3 and Sec. 6.2): the Ritz-based
adaptive bounds converge to the closed-form spectrum, and the remark after
Eq. (optimal_poly) -- ending the unwanted interval at lambda_{p+k}, k > 1,
instead of lambda_{p+1} can converge faster -- holds on an FD Laplacian."""
import numpy as np

from oracle import gsi_oracle as O
from paper_2306_10379_gb300 import inputs as I


def _problem(dims):
    A = I.fd_laplacian(dims)
    return A, I.laplacian_eigenvalues(dims), O.csr_operator(A.n, A.rowptr, A.colidx, A.val)


def test_adaptive_bounds_converge_to_the_closed_form():
    """Ritz-based bounds on [0, theta_min] (0 lies below the Laplacian's
    spectrum) with 3 guard vectors: the 6 wanted Ritz pairs reach the
    tolerance and match the closed form; without guard vectors the filter's
    upper end theta_min sits at lambda_p, which it then no longer separates
    from lambda_{p+1}, and the p-th pair stalls."""
    dims, p, g, d = (20, 18), 9, 3, 8
    A, lam, S = _problem(dims)
    assert lam[-1] > 0.0
    X0 = I.start_block(A.n, p, 7)
    X, th, outer, mv, rel = O.chebyshev_si(S, X0, d, 0.0, 0.0, 0.0, tol=1e-9, anorm=lam[0], adaptive=True,
                                           guard=g)
    assert rel <= 1e-9 and outer < 100
    assert np.max(np.abs(th[:p - g] - lam[:p - g])) < 1e-11 * lam[0]
    assert np.max(np.abs(X.T @ X - np.eye(p))) < 1e-13
    _, th0, outer0, _, rel0 = O.chebyshev_si(S, I.start_block(A.n, p - g, 7), d, 0.0, 0.0, 0.0, tol=1e-9,
                                             anorm=lam[0], adaptive=True, max_outer=3 * outer)
    assert rel0 > 1e-9


def test_interval_end_lambda_p_plus_k_remark():
    """Fixed bounds [lambda_n, lambda_{p+k}] with the exact spectrum: k = 2
    needs fewer outer iterations than k = 1 here (25 against 32)."""
    dims, p, d = (20, 18), 6, 8
    A, lam, S = _problem(dims)
    X0 = I.start_block(A.n, p, 7)
    outs = {}
    for k in (1, 2):
        _, th, outer, _, rel = O.chebyshev_si(S, X0, d, lam[p + k - 1], lam[-1], lam[0], tol=1e-8, anorm=lam[0])
        assert rel <= 1e-8
        assert np.max(np.abs(np.sort(th)[::-1] - lam[:p])) < 1e-10 * lam[0]
        outs[k] = outer
    assert outs[2] < outs[1]
