"""Chebyshev-filtered subspace iteration (Alg. 1 with the filter of Eq.
(optimal_poly)), the paper's comparator, against the oracle: the Ritz values
after k filter steps, the converged spectrum and the iteration counts."""
import numpy as np
import pytest

from oracle import gsi_oracle as O
from paper_2306_10379_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gsi():
    from paper_2306_10379_gb300 import build, gsi as g
    build.build()
    return g


def _problem(dims, p):
    A = I.fd_laplacian(dims)
    lam = I.laplacian_eigenvalues(dims)
    S = O.csr_operator(A.n, A.rowptr, A.colidx, A.val)
    return A, lam, S


@pytest.mark.parametrize("precision", ["df64", "f64"])
def test_cheb_steps_match_oracle(gsi, precision):
    dims, p, d = (20, 18), 6, 8
    A, lam, S = _problem(dims, p)
    X0 = I.start_block(A.n, p, 7)
    with gsi.Solver(A, p, X0, method="cheb", tol=1e-12, anorm=lam[0], precision=precision,
                    cheb_degree=d, cheb_interval=(lam[-1], lam[p]), cheb_scale=lam[0]) as s:
        for k in range(1, 4):
            s.step(1)
            _, ev = s.basis()
            _, th, outer, mv, rel = O.chebyshev_si(S, X0, d, lam[p], lam[-1], lam[0], tol=0.0,
                                                  anorm=lam[0], max_outer=k)
            assert outer == k
            assert np.max(np.abs(ev - th) / np.abs(th)) < 1e-10, k


@pytest.mark.parametrize("precision", ["df64", "f64"])
def test_cheb_converges_like_oracle(gsi, precision):
    dims, p, d = (16, 16), 6, 8
    A, lam, S = _problem(dims, p)
    X0 = I.start_block(A.n, p, 9)
    with gsi.Solver(A, p, X0, method="cheb", tol=1e-9, anorm=lam[0], precision=precision,
                    cheb_degree=d, cheb_interval=(lam[-1], lam[p]), cheb_scale=lam[0]) as s:
        info = s.solve()
        X, ev = s.basis()
    _, th, outer, mv, rel = O.chebyshev_si(S, X0, d, lam[p], lam[-1], lam[0], tol=1e-9, anorm=lam[0])
    assert info["converged"] == 1
    assert abs(info["iters"] - outer) <= 1
    assert info["matvecs"] == 1 + info["iters"] * (d + 1)
    assert np.max(np.abs(ev - lam[:p])) < 1e-11 * lam[0]
    R = S @ X - X * ev
    assert np.linalg.norm(R) / lam[0] <= 1.01e-9


def test_cheb_rejects_bad_interval(gsi):
    A, lam, S = _problem((10, 10), 3)
    with pytest.raises(gsi.GsiError):
        gsi.Solver(A, 3, I.start_block(A.n, 3, 1), method="cheb", cheb_interval=(1.0, 0.5),
                   cheb_scale=2.0)


@pytest.mark.parametrize("precision", ["df64", "f64"])
def test_cheb_adaptive_matches_oracle(gsi, precision):
    """Ritz-based bounds (unwanted interval [0, theta_min], scaled at
    theta_max) with 3 guard vectors: Ritz values after each of the first 4
    filter steps against the oracle's adaptive run, then the outer iteration
    count and convergence of the 6 wanted pairs to the closed form."""
    dims, p, g, d = (20, 18), 9, 3, 8
    A, lam, S = _problem(dims, p)
    X0 = I.start_block(A.n, p, 7)
    with gsi.Solver(A, p, X0, method="cheb", tol=1e-9, anorm=lam[0], precision=precision, cheb_degree=d,
                    cheb_interval=(0.0, 0.0), cheb_adaptive=True, cheb_guard=g) as s:
        for k in range(1, 5):
            s.step(1)
            _, ev = s.basis()
            _, th, outer, _, _ = O.chebyshev_si(S, X0, d, 0.0, 0.0, 0.0, tol=0.0, anorm=lam[0], max_outer=k,
                                                adaptive=True, guard=g)
            assert np.max(np.abs(ev - th) / np.abs(th)) < 1e-10, k
        info = s.solve()
        _, ev = s.basis()
    _, th, outer, _, _ = O.chebyshev_si(S, X0, d, 0.0, 0.0, 0.0, tol=1e-9, anorm=lam[0], adaptive=True, guard=g)
    assert info["converged"] == 1
    assert abs(info["iters"] - outer) <= 1
    assert np.max(np.abs(ev[:p - g] - lam[:p - g])) < 1e-11 * lam[0]
