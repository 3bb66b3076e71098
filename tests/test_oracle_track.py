"""Pins of the oracle's subspace tracking (a sequence of slowly varying
operators, each solved from the previous final iterate; Sec. 1) against
mathematics other than the oracle itself."""
import numpy as np

from oracle import gsi_oracle as O
from paper_2306_10379_gb300 import inputs as I


def _mats(seq):
    return [O.csr_operator(A.n, A.rowptr, A.colidx, A.val) for A in seq]


def test_drifting_sequence_is_what_it_says():
    """A_k - A_0 = eps k diag(v) with v the stated product of sin cos at the nodes."""
    dims, eps = (7, 5), 0.03
    seq = I.drifting_laplacians(dims, 3, eps)
    L = O.csr_operator(*(lambda A: (A.n, A.rowptr, A.colidx, A.val))(I.fd_laplacian(dims))).toarray()
    for k, A in enumerate(seq):
        D = O.csr_operator(A.n, A.rowptr, A.colidx, A.val).toarray() - L
        assert np.allclose(D, np.diag(np.diag(D)), atol=0)
        for i1 in range(dims[1]):
            for i0 in range(dims[0]):
                x0, x1 = (i0 + 1) / (dims[0] + 1), (i1 + 1) / (dims[1] + 1)
                want = eps * k * np.sin(np.pi * x0) * np.cos(np.pi * x0) * np.sin(np.pi * x1) * np.cos(np.pi * x1)
                assert abs(D[i0 + dims[0] * i1, i0 + dims[0] * i1] - want) < 1e-15


def test_identical_operator_needs_no_iteration():
    """Tracking A, A: the second solve starts from a basis that already meets the
    tolerance, so it stops after the explicit AX with 0 iterations and keeps the
    subspace."""
    dims, p = (20, 18), 6
    A = I.fd_laplacian(dims)
    S = O.csr_operator(A.n, A.rowptr, A.colidx, A.val)
    lam = I.laplacian_eigenvalues(dims)
    r = O.track([S, S], I.start_block(A.n, p, 11), O.Options(method="cg", tol=1e-8, anorm=lam[0]))
    assert r[0].converged and r[1].converged
    assert r[0].iters > 50 and r[1].iters == 0
    X1, X2 = r[0].X, r[1].X  # sine of the largest principal angle
    assert np.linalg.norm(X2 - X1 @ (X1.T @ X2), 2) < 1e-12


def test_tracked_subspaces_are_the_dominant_ones_and_cheaper():
    """Each tracked result spans the dominant subspace of its own operator
    (dense eigendecomposition, within the Davis-Kahan bound 2 ||R||_F / gap),
    and every solve after the first needs fewer iterations than from a fresh
    random start."""
    dims, p, K, eps = (20, 18), 6, 4, 0.05
    seq = I.drifting_laplacians(dims, K, eps)
    mats = _mats(seq)
    lam = I.laplacian_eigenvalues(dims)
    anorm = lam[0] + K * eps
    opts = O.Options(method="cg", tol=1e-8, anorm=anorm)
    res = O.track(mats, I.start_block(seq[0].n, p, 12), opts)
    for k, (S, r) in enumerate(zip(mats, res)):
        assert r.converged
        Ad = S.toarray()
        w, U = np.linalg.eigh(Ad)
        X = r.X
        th = np.linalg.eigvalsh(X.T @ Ad @ X)
        R = Ad @ X - X @ (X.T @ Ad @ X)
        gap = w[-p] - w[-p - 1]
        assert O.principal_angles(X, U[:, -p:]).max() <= 2 * np.linalg.norm(R) / gap + 1e-12
        assert np.max(np.abs(np.sort(th) - w[-p:])) < 1e-10 * anorm
        if k > 0:
            fresh = O.solve(S, I.start_block(seq[0].n, p, 100 + k), opts)
            assert r.iters < fresh.iters, (k, r.iters, fresh.iters)
