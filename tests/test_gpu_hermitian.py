"""Complex Hermitian A (the footnote to Eq. (phi)) through
gsi_create_hermitian against the oracle's complex128 solve_hermitian and the
closed-form spectrum of a twisted (magnetic) torus Laplacian."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import gsi_oracle as O
from paper_2306_10379_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _zop(A):
    return sp.csr_matrix((A.val, A.colidx, A.rowptr), shape=(A.n, A.n))


@pytest.mark.parametrize("precision", ["df64", "f64"])
@pytest.mark.parametrize("method", ["sd", "cg"])
def test_trajectory_matches_complex_oracle(torch_cuda, method, precision):
    """First 10 iterates equal the oracle's complex iterates to 1e-10 (the
    realification carries the iterate itself, not only its span)."""
    from paper_2306_10379_gb300 import gsi
    dims, th, p = (16, 14), (0.9, 2.3), 6
    A = I.twisted_torus_laplacian(dims, th)
    lam = I.twisted_torus_eigenvalues(dims, th)
    S = _zop(A)
    X0 = I.complex_start_block(A.n, p, 3)
    traj = []
    for k in range(1, 11):
        traj.append(O.solve_hermitian(S, X0, O.Options(method=method, tol=1e-8, anorm=lam[0], max_iters=k)).X)
    with gsi.HermitianSolver(A, p, X0, method=method, tol=1e-8, anorm=lam[0], precision=precision) as s:
        for k in range(10):
            s.step(1)
            X, _ = s.basis(evals=False)
            assert np.max(np.abs(X - traj[k])) <= 1e-10, k


@pytest.mark.parametrize("precision", ["df64", "f64"])
def test_solve_closed_form_and_oracle(torch_cuda, precision):
    """CG to 1e-8: complex orthonormality (to the rounding drift of the
    realification's structure), Ritz values within the quadratic
    residual bound of the closed form, the subspace within Davis-Kahan of the
    exact one, iteration count within 2% of the complex oracle's; the
    smallest eigenvalues via which = -1."""
    from paper_2306_10379_gb300 import gsi
    dims, th, p = (16, 14), (0.9, 2.3), 6
    A = I.twisted_torus_laplacian(dims, th)
    lam = I.twisted_torus_eigenvalues(dims, th)
    S = _zop(A)
    X0 = I.complex_start_block(A.n, p, 3)
    ref = O.solve_hermitian(S, X0, O.Options(method="cg", tol=1e-8, anorm=lam[0]))
    with gsi.HermitianSolver(A, p, X0, method="cg", tol=1e-8, anorm=lam[0], precision=precision) as s:
        info = s.solve()
        X, ev = s.basis()
    assert info["converged"] == 1 and ref.converged
    assert abs(info["iters"] - ref.iters) <= max(2, 0.02 * ref.iters), (info["iters"], ref.iters)
    # the realified iterate is orthonormal to rounding (5e-13); its complex
    # structure [[Xr, -Xi], [Xi, Xr]] only up to a rounding drift, which the
    # extracted complex basis carries (about 4e-12 after a df64 solve)
    assert np.max(np.abs(X.conj().T @ X - np.eye(p))) < 2e-11
    gap = lam[p - 1] - lam[p]
    assert np.max(np.abs(ev - lam[:p])) <= 2 * (1e-8 * lam[0]) ** 2 / gap + 1e-12 * lam[0]
    Ad = S.toarray()
    w, U = np.linalg.eigh(Ad)
    Uex = U[:, ::-1][:, :p]
    R = Ad @ X - X @ (X.conj().T @ Ad @ X)
    sin = np.linalg.norm(X - Uex @ (Uex.conj().T @ X), 2)
    assert sin <= 2 * np.linalg.norm(R) / gap + 1e-12
    assert abs(info["trace"] - np.sum(lam[:p])) < 1e-7 * lam[0]
    with gsi.HermitianSolver(A, p, X0, method="cg", which=-1, tol=1e-8, anorm=lam[0], precision=precision) as s:
        assert s.solve()["converged"] == 1
        _, ev = s.basis()
    assert np.max(np.abs(ev - lam[::-1][:p])) < 1e-9 * lam[0]
