"""The staged SpMM for stencil-shaped operators (diagonal layout, shared-memory
window of 64-row tiles, far diagonals from global memory) against the CSR
kernel (bit for bit on sorted CSR rows: the same summation order, and absent
entries add exact zeros) and the oracle; and the solver, which takes it for
such operators, against its own CSR path."""
import os

import numpy as np
import pytest

from oracle import gsi_oracle as O
from paper_2306_10379_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import torch
    from paper_2306_10379_gb300 import build, gsi
    build.build()
    return torch, gsi


def _df(torch, gsi, x):
    return torch.from_numpy(gsi.to_df(x)).cuda()


def _exact(gsi, x):
    return gsi.from_df(gsi.to_df(x))


@pytest.mark.parametrize("name,A,p", [
    ("3d_20x22x24", lambda: I.fd_laplacian((20, 22, 24)), 64),   # 0, +-1, +-20 near; +-440 far
    ("3d_20x22x24_p8", lambda: I.fd_laplacian((20, 22, 24)), 8),
    ("3d_100x5x4", lambda: I.fd_laplacian((100, 5, 4)), 64),     # +-100 near (q = 2), +-500 far
    ("2d_33x31", lambda: I.fd_laplacian((33, 31)), 32),          # no far diagonal
    ("1d_1000", lambda: I.fd_laplacian((1000,)), 2),
    ("drift_3d", lambda: I.drifting_laplacians((17, 9, 11), 3, 0.3)[2], 64),
])
def test_dia_equals_csr_and_oracle(G, name, A, p):
    torch, gsi = G
    A = A()
    off, dia = gsi.csr_to_dia(A.n, A.rowptr, A.colidx, A.val)
    val = _exact(gsi, A.val * (1 + 1e-9 * np.arange(A.nnz) / A.nnz))  # non-integer values
    _, dia = gsi.csr_to_dia(A.n, A.rowptr, A.colidx, val)
    X = _exact(gsi, I.start_block(A.n, p, 4))
    Wd = torch.empty((A.n, p, 2), dtype=torch.float32, device="cuda")
    Wc = torch.empty_like(Wd)
    gsi.df_spmm_dia(off, _df(torch, gsi, dia), _df(torch, gsi, X), Wd)
    gsi.df_spmm_csr(torch.from_numpy(A.rowptr).cuda(), torch.from_numpy(A.colidx).cuda(),
                    _df(torch, gsi, val), _df(torch, gsi, X), Wc)
    assert torch.equal(Wd, Wc), name
    S = O.csr_operator(A.n, A.rowptr, A.colidx, val)
    got = gsi.from_df(Wd.cpu().numpy())
    assert np.all(np.abs(got - O.spmm(S, X)) <= 1e-13 * O.spmm(abs(S), np.abs(X)))


def test_dia_rejects_unsupported_shapes(G):
    torch, gsi = G
    A = I.fd_laplacian((10, 10))
    off, dia = gsi.csr_to_dia(A.n, A.rowptr, A.colidx, A.val)
    X = torch.zeros((A.n, 7, 2), dtype=torch.float32, device="cuda")
    W = torch.empty_like(X)
    with pytest.raises(gsi.GsiError):  # odd p
        gsi.df_spmm_dia(off, _df(torch, gsi, dia), X, W)


def test_solver_takes_the_staged_kernel(G):
    """A 3D Laplacian solve through the staged SpMM (GSI_SPMM_DIA=1 at
    creation) and through the CSR kernel (the default): identical
    trajectories (the two SpMMs are bit-identical), identical results."""
    torch, gsi = G
    dims, p = (24, 22, 20), 16
    A = I.fd_laplacian(dims)
    lam = I.laplacian_eigenvalues(dims)
    X0 = I.start_block(A.n, p, 2)
    out = []
    for env in ("1", "0"):
        os.environ["GSI_SPMM_DIA"] = env
        try:
            with gsi.Solver(A, p, X0, method="cg", tol=1e-8, anorm=lam[0]) as s:
                info = s.solve()
                X, ev = s.basis()
        finally:
            os.environ.pop("GSI_SPMM_DIA", None)
        out.append((info, X, ev))
    (i1, X1, e1), (i2, X2, e2) = out
    assert i1["iters"] == i2["iters"] and i1["rel_residual"] == i2["rel_residual"]
    assert np.array_equal(X1, X2) and np.array_equal(e1, e2)
    assert np.max(np.abs(e1 - lam[:p]) / lam[:p]) < 1e-10
