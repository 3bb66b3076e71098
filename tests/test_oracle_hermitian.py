"""Pins of the oracle's complex Hermitian solve (the footnote to Eq. (phi))
against facts that do not depend on it: the closed-form spectrum of a
twisted (magnetic) torus Laplacian, the reduction to the real algorithm for
a real symmetric A, equivariance under a diagonal unitary change of basis,
and the realification of Eq. (phi) used by the library (the real iteration
on [[Ar, -Ai], [Ai, Ar]] from the realified start block follows the complex
iterates)."""
import numpy as np
import scipy.sparse as sp

from oracle import gsi_oracle as O
from paper_2306_10379_gb300 import inputs as I


def _zop(A):
    return sp.csr_matrix((A.val, A.colidx, A.rowptr), shape=(A.n, A.n))


def _realify(S):
    Ar, Ai = sp.csr_matrix(S.real), sp.csr_matrix(S.imag)
    return sp.bmat([[Ar, -Ai], [Ai, Ar]], format="csr")


def test_twisted_torus_generator_and_closed_form():
    dims, th = (5, 4), (0.7, -1.1)
    A = I.twisted_torus_laplacian(dims, th)
    S = _zop(A).toarray()
    assert np.allclose(S, S.conj().T, atol=0)
    assert np.abs(S.imag).max() > 0.1  # genuinely complex
    w = np.linalg.eigvalsh(S)[::-1]
    assert np.max(np.abs(w - I.twisted_torus_eigenvalues(dims, th))) < 1e-12


def test_converges_to_the_closed_form_spectrum():
    """CG on a 16 x 14 twisted torus, p = 6: residual 1e-8, X^H X = I, Ritz
    values within the quadratic residual bound of the closed form."""
    dims, th, p = (16, 14), (0.9, 2.3), 6
    A = I.twisted_torus_laplacian(dims, th)
    lam = I.twisted_torus_eigenvalues(dims, th)
    S = _zop(A)
    r = O.solve_hermitian(S, I.complex_start_block(A.n, p, 3), O.Options(method="cg", tol=1e-8, anorm=lam[0]))
    assert r.converged
    X = r.X
    assert np.max(np.abs(X.conj().T @ X - np.eye(p))) < 1e-13
    th_r = np.sort(np.linalg.eigvalsh(X.conj().T @ (S @ X)))[::-1]
    gap = lam[p - 1] - lam[p]
    assert gap > 1e-3
    assert np.max(np.abs(th_r - lam[:p])) <= 2 * (1e-8 * lam[0]) ** 2 / gap + 1e-12 * lam[0]


def test_real_symmetric_input_reduces_to_the_real_algorithm():
    """A real symmetric A and a real start block: the complex iterates are
    the real ones (the imaginary parts stay zero)."""
    dims, p = (12, 11), 4
    A = I.fd_laplacian(dims)
    lam = I.laplacian_eigenvalues(dims)
    S = O.csr_operator(A.n, A.rowptr, A.colidx, A.val)
    X0 = I.start_block(A.n, p, 5)
    for m in ("sd", "cg"):
        o = O.Options(method=m, tol=1e-8, anorm=lam[0], max_iters=25)
        rr = O.solve(S, X0, o)
        rc = O.solve_hermitian(S.astype(np.complex128), X0.astype(np.complex128), o)
        assert rr.iters == rc.iters
        assert np.max(np.abs(rc.X.imag)) == 0.0
        assert np.max(np.abs(rc.X.real - rr.X)) < 1e-12


def test_equivariance_under_a_diagonal_unitary():
    """A' = Q A Q^H, X0' = Q X0 with Q = diag(exp(i phi)): the iterates are
    X' = Q X (every step commutes with the change of basis)."""
    dims, th, p = (9, 8), (0.4, 1.3), 5
    A = I.twisted_torus_laplacian(dims, th)
    lam = I.twisted_torus_eigenvalues(dims, th)
    S = _zop(A)
    phi = np.linspace(0.0, 5.0, A.n)
    Q = sp.diags(np.exp(1j * phi))
    X0 = I.complex_start_block(A.n, p, 7)
    o = O.Options(method="cg", tol=1e-8, anorm=lam[0], max_iters=15)
    r1 = O.solve_hermitian(S, X0, o)
    r2 = O.solve_hermitian(Q @ S @ Q.conj().T, Q @ X0, o)
    assert np.max(np.abs(r2.X - Q @ r1.X)) < 1e-11


def test_realification_follows_the_complex_iteration():
    """The library's route: the real method on the realified operator
    [[Ar, -Ai], [Ai, Ar]] (2n x 2n) from [[X0r, -X0i], [X0i, X0r]] (2p
    columns) keeps that structure, and its first p columns are the complex
    iterate [Xr; Xi] (Eq. (phi) for the realification is twice the complex
    objective; the gradient, the Polak-Ribiere beta, the exact step t and the
    polar factor all commute with it). Checked over 20 CG iterations and at
    convergence (p complex Ritz values = the realified ones, each twice)."""
    dims, th, p = (10, 9), (0.9, 2.3), 4
    A = I.twisted_torus_laplacian(dims, th)
    lam = I.twisted_torus_eigenvalues(dims, th)
    S = _zop(A)
    R = _realify(S)
    X0 = I.complex_start_block(A.n, p, 9)
    Xh0 = np.block([[X0.real, -X0.imag], [X0.imag, X0.real]])
    for k in (3, 20):
        oc = O.Options(method="cg", tol=1e-8, anorm=lam[0], max_iters=k)
        orl = O.Options(method="cg", tol=1e-8, anorm=np.sqrt(2.0) * lam[0], max_iters=k)
        rc = O.solve_hermitian(S, X0, oc)
        rr = O.solve(R, Xh0, orl)
        n = A.n
        Xc = rr.X[:n, :p] + 1j * rr.X[n:, :p]
        assert np.max(np.abs(Xc - rc.X)) < 1e-10, k
        assert np.max(np.abs(rr.X[:n, p:] + rr.X[n:, :p])) < 1e-10
    oc = O.Options(method="cg", tol=1e-8, anorm=lam[0])
    orl = O.Options(method="cg", tol=1e-8, anorm=np.sqrt(2.0) * lam[0])
    rc = O.solve_hermitian(S, X0, oc)
    rr = O.solve(R, Xh0, orl)
    assert rc.converged and rr.converged and abs(rc.iters - rr.iters) <= 2
    wr = np.sort(np.linalg.eigvalsh(rr.X.T @ (R @ rr.X)))[::-1]
    assert np.max(np.abs(wr[0::2] - wr[1::2])) < 1e-12
    assert np.max(np.abs(wr[0::2] - lam[:p])) < 1e-10
