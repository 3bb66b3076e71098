"""Subspace tracking through gsi_set_operator (a sequence of slowly varying
operators, each solved from the previous final iterate; Sec. 1) against the
oracle's track() and the dense eigendecompositions."""
import numpy as np
import pytest

from oracle import gsi_oracle as O
from paper_2306_10379_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["df64", "f64"])
def test_tracking_matches_oracle(torch_cuda, precision):
    from paper_2306_10379_gb300 import gsi
    dims, p, K, eps = (20, 18), 6, 4, 0.05
    seq = I.drifting_laplacians(dims, K, eps)
    lam = I.laplacian_eigenvalues(dims)
    anorm = lam[0] + K * eps
    X0 = I.start_block(seq[0].n, p, 12)
    mats = [O.csr_operator(A.n, A.rowptr, A.colidx, A.val) for A in seq]
    ref = O.track(mats, X0, O.Options(method="cg", tol=1e-8, anorm=anorm))
    with gsi.Solver(seq[0], p, X0, method="cg", tol=1e-8, anorm=anorm, precision=precision) as s:
        for k, A in enumerate(seq):
            if k > 0:
                s.set_operator(A)
            info = s.solve()
            X, ev = s.basis()
            assert info["converged"] == 1
            assert abs(info["iters"] - ref[k].iters) <= max(2, 0.02 * ref[k].iters), (k, info["iters"], ref[k].iters)
            Ad = mats[k].toarray()
            w, U = np.linalg.eigh(Ad)
            assert np.max(np.abs(ev - w[::-1][:p])) < 1e-10 * anorm
            R = Ad @ X - X * ev
            gap = w[-p] - w[-p - 1]
            assert O.principal_angles(X, U[:, -p:]).max() <= 2 * np.linalg.norm(R) / gap + 1e-12
    assert all(ref[k].iters < ref[0].iters for k in range(1, K))


def test_identical_operator_needs_no_iteration(torch_cuda):
    from paper_2306_10379_gb300 import gsi
    dims, p = (20, 18), 6
    A = I.fd_laplacian(dims)
    lam = I.laplacian_eigenvalues(dims)
    with gsi.Solver(A, p, I.start_block(A.n, p, 11), method="cg", tol=1e-8, anorm=lam[0]) as s:
        assert s.solve()["iters"] > 50
        X1, _ = s.basis(evals=False)
        s.set_operator(A)
        info = s.solve()
        X2, _ = s.basis(evals=False)
    assert info["converged"] == 1 and info["iters"] == 0
    # sine of the largest principal angle (arccos of the cosines would read an
    # orthonormality error d as an angle of sqrt(2 d))
    assert np.linalg.norm(X2 - X1 @ (X1.T @ X2), 2) < 1e-12


@pytest.mark.parametrize("fmt", ["csr", "sell"])
def test_set_operator_with_other_sparsity(torch_cuda, fmt):
    """An operator with another number of nonzeros (buffers reallocated, the
    SELL layout rebuilt): the solve from the carried basis finds its own
    dominant subspace."""
    from paper_2306_10379_gb300 import gsi
    n, p = 2000, 8
    A0 = I.er_laplacian(n, 5)
    A1 = I.er_laplacian(n, 6, mean_degree=10)
    assert A0.nnz != A1.nnz
    with gsi.Solver(A0, p, I.start_block(n, p, 3), method="cg", tol=1e-8, fmt=fmt) as s:
        assert s.solve()["converged"] == 1
        s.set_operator(A1)
        info = s.solve()
        X, ev = s.basis()
    Ad = O.csr_operator(A1.n, A1.rowptr, A1.colidx, A1.val).toarray()
    w = np.linalg.eigvalsh(Ad)
    assert info["converged"] == 1
    assert np.max(np.abs(ev - w[::-1][:p])) < 1e-9 * w[-1]
