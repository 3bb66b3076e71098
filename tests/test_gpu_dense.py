"""Dense operator (A = Q diag(lambda) Q^T with a prescribed gap) and the
mixed-precision mode: the dense tensor-core apply against A X, whole solves
against the oracle and the known spectrum."""
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


def _dense(n, p, gap=1e-2, seed=I.SEED_BASE + 2, reflectors=4):
    A, lam = I.dense_spectrum(n, p, gap, seed, reflectors=reflectors)
    return A, lam


@pytest.mark.parametrize("n,p,nd", [(1000, 16, 7), (777, 100, 7), (1000, 16, 3), (130, 1, 7),
                                    (2048, 128, 3), (2048, 128, 7), (2113, 128, 3)])
def test_dense_apply(gsi, n, p, nd):
    import torch
    A, lam = _dense(n, max(p, 2))
    A = gsi.from_df(gsi.to_df(A))
    A = 0.5 * (A + A.T)
    X = gsi.from_df(gsi.to_df(I.start_block(n, p, 3)))
    W = torch.empty((n, p, 2), dtype=torch.float32, device="cuda")
    gsi.oz_dense_apply(torch.from_numpy(gsi.to_df(A)).cuda(), torch.from_numpy(gsi.to_df(X)).cuda(), W, nd=nd)
    got = gsi.from_df(W.cpu().numpy())
    ref = A @ X
    # per exponent chunk of the kernel that runs (the apply is a Gram of
    # 64-column blocks of A: 3 digits on the maxima-warp kernel, 384-row
    # chunks; 7 digits on the whole-chunk kernel, 160-row chunks): products
    # cut at the chunk's column maxima
    ec = 384 if nd == 3 else 160
    bound = np.zeros_like(ref)
    for r0 in range(0, n, ec):
        ca = np.abs(A[r0:r0 + ec]).max(0)     # column maxima of A^T's chunk = rows of A
        cx = np.abs(X[r0:r0 + ec]).max(0)
        bound += np.outer(ca, cx) * min(ec, n - r0)
    scale = 2.0 ** -44 if nd == 7 else 2.0 ** -19
    assert np.all(np.abs(got - ref) <= scale * bound + 2.0 ** -46 * (np.abs(A) @ np.abs(X)))


@pytest.mark.parametrize("precision", ["df64", "f64"])
def test_dense_trajectory(gsi, precision):
    n, p = 600, 8
    A, lam = _dense(n, p)
    X0 = I.start_block(n, p, 5)
    ref = []
    O.solve(A, X0, O.Options(method="cg", tol=1e-8, anorm=lam[0], max_iters=8),
            callback=lambda k, X, Y, t: ref.append((X.copy(), t)))
    with gsi.Solver(gsi.Dense(A), p, X0, method="cg", tol=1e-8, anorm=lam[0], precision=precision) as s:
        for k in range(8):
            info = s.step(1)
            X, _ = s.basis(evals=False)
            assert abs(info["last_step"] - ref[k][1]) <= 1e-9 * ref[k][1], k
            assert np.max(np.abs(X - ref[k][0])) <= 1e-9, k


@pytest.mark.parametrize("precision", ["mixed", "df64", "f64"])
def test_dense_solve(gsi, precision):
    """Converges to relative residual 1e-8; the Ritz values match the prescribed
    spectrum; the mixed mode ends in its 7-digit correction phase."""
    n, p = 1024, 16
    A, lam = _dense(n, p)
    X0 = I.start_block(n, p, 6)
    with gsi.Solver(gsi.Dense(A), p, X0, method="cg", tol=1e-8, anorm=lam[0], precision=precision,
                    max_iters=2000) as s:
        info = s.solve()
        X, ev = s.basis()
    assert info["converged"] == 1
    R = A @ X - X * ev
    assert np.linalg.norm(R) / lam[0] <= 1.01e-8
    gap = lam[p - 1] - lam[p]
    # residual bound plus the df64 floor of the Ritz values (~1e-13)
    assert np.max(np.abs(ev - lam[:p])) <= 2 * (1e-8 * lam[0]) ** 2 / gap + 5e-13
    w, U = np.linalg.eigh(A)
    ang = O.principal_angles(X, U[:, ::-1][:, :p]).max()
    assert ang <= 2 * np.linalg.norm(R) / gap + 1e-12


def test_dense_mixed_solve_p128(gsi):
    """The mixed-precision form at the dense config's block size, p = 128: the
    3-digit direction apply runs on two 64-column output slices, then the
    7-digit correction phase. Converges to 1e-8; Ritz values and the subspace
    against the prescribed spectrum within the Davis-Kahan bounds; the Ritz
    values also against the float64 oracle's own solve from the same start."""
    n, p = 2048, 128
    A, lam = _dense(n, p, reflectors=4)
    X0 = I.start_block(n, p, 7)
    with gsi.Solver(gsi.Dense(A), p, X0, method="cg", tol=1e-8, anorm=lam[0], precision="mixed",
                    max_iters=3000) as s:
        info = s.solve()
        X, ev = s.basis()
    assert info["converged"] == 1
    R = A @ X - X * ev
    assert np.linalg.norm(R) / lam[0] <= 1.01e-8
    gap = lam[p - 1] - lam[p]
    assert np.max(np.abs(ev - lam[:p])) <= 2 * (1e-8 * lam[0]) ** 2 / gap + 5e-13
    w, U = np.linalg.eigh(A)
    assert O.principal_angles(X, U[:, ::-1][:, :p]).max() <= 2 * np.linalg.norm(R) / gap + 1e-12
    ores = O.solve(A, X0, O.Options(method="cg", tol=1e-8, anorm=lam[0], max_iters=3000))
    assert ores.converged
    th = np.sort(np.linalg.eigvalsh(ores.X.T @ A @ ores.X))[::-1]
    assert np.max(np.abs(ev - th)) <= 4 * (1e-8 * lam[0]) ** 2 / gap + 1e-12
