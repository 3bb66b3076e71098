"""The hot-path kernels at the full bench size: the 3D 7-point FD Laplacian
128^3 (n = 2,097,152, nnz = 14,581,760) with p = 64 df64 blocks, through the
same kernels and grid shapes the solve uses. Outputs are checked where the
oracle can compute them one by one: sampled rows of the SpMM and of a block
product, sampled entries of the Grams (exact sums of the float64 products).
The bounds are those of the smaller parity tests."""
import math

import numpy as np
import pytest

from oracle import gsi_oracle as O
from paper_2306_10379_gb300 import inputs as I

pytestmark = pytest.mark.gpu

DIMS, P = (128, 128, 128), 64


@pytest.fixture(scope="module")
def big(torch_cuda):
    torch = torch_cuda
    from paper_2306_10379_gb300 import gsi
    A = I.fd_laplacian(DIMS)
    rng = np.random.default_rng(2306)
    U = gsi.from_df(gsi.to_df(rng.standard_normal((A.n, P))))
    V = gsi.from_df(gsi.to_df(rng.standard_normal((A.n, P)) * np.exp(rng.uniform(-2, 2, (A.n, 1)))))
    Ud = torch.from_numpy(gsi.to_df(U)).cuda()
    Vd = torch.from_numpy(gsi.to_df(V)).cuda()
    rows = np.unique(np.concatenate([[0, 1, 127, 128 * 128, A.n - 2, A.n - 1], rng.integers(0, A.n, 58)]))
    return torch, gsi, A, U, V, Ud, Vd, rows, rng


def _rows(torch, T, rows):
    return T[torch.from_numpy(rows).cuda()].cpu().numpy()


def test_spmm_full_size_sampled_rows(big):
    torch, gsi, A, U, V, Ud, Vd, rows, rng = big
    assert A.n == 2097152 and A.nnz == 14581760
    W = torch.empty((A.n, P, 2), dtype=torch.float32, device="cuda")
    gsi.df_spmm_csr(torch.from_numpy(A.rowptr).cuda(), torch.from_numpy(A.colidx).cuda(),
                    torch.from_numpy(gsi.to_df(A.val)).cuda(), Ud, W)
    got = gsi.from_df(_rows(torch, W, rows))
    for i, r in enumerate(rows):
        ks = range(A.rowptr[r], A.rowptr[r + 1])
        ref = sum(A.val[k] * U[A.colidx[k]] for k in ks)
        mag = sum(abs(A.val[k]) * np.abs(U[A.colidx[k]]) for k in ks)
        assert np.all(np.abs(got[i] - ref) <= 1e-13 * mag), r


def _chunk_bound(u, v):
    """Digit-split Gram bound of the smaller tests: 2^-44 times the sum over
    1536-row windows (each holding whole 512- and 384-row exponent chunks of
    the tcgen05 Grams) of rows x column maxima, plus 2^-46 sum |u||v|."""
    b = 0.0
    for r0 in range(0, u.shape[0], 1536):
        b += float(np.abs(u[r0:r0 + 1536]).max() * np.abs(v[r0:r0 + 1536]).max()) * min(1536, u.shape[0] - r0)
    return 2.0 ** -44 * b + 2.0 ** -46 * float(np.abs(u) @ np.abs(v))


@pytest.mark.parametrize("sym", [False, True])
def test_gram_full_size_sampled_entries(big, sym):
    torch, gsi, A, U, V, Ud, Vd, rows, rng = big
    G = torch.full((P, P), float("nan"), dtype=torch.float64, device="cuda")
    gsi.oz_gram(Ud, Ud if sym else Vd, G, sym=sym)
    got = G.cpu().numpy()
    assert np.all(np.isfinite(got))
    Vr = U if sym else V
    for a, b in [(0, 0), (63, 63), (5, 40), (40, 5), (17, 17), (33, 2), (1, 62), (62, 1)]:
        ref = math.fsum(U[:, a] * Vr[:, b])
        assert abs(got[a, b] - ref) <= _chunk_bound(U[:, a], Vr[:, b]), (a, b)
    if sym:
        assert np.array_equal(got, got.T)


def test_block_product_full_size_sampled_rows(big):
    """out = V - U M (the shape of R = Y - X C), rows sampled."""
    torch, gsi, A, U, V, Ud, Vd, rows, rng = big
    M = rng.standard_normal((P, P)) * np.exp(rng.uniform(-1, 1, (1, P)))
    out = torch.empty_like(Ud)
    gsi.oz_gemm(Ud, torch.from_numpy(M).cuda(), out, s0=-1.0, E=[Vd], c=[1.0])
    got = gsi.from_df(_rows(torch, out, rows))
    ref = V[rows] - U[rows] @ M
    bound = (np.abs(U[rows]).max(1, keepdims=True) * np.abs(M).max(0, keepdims=True) * P * 2.0 ** -44
             + np.abs(V[rows]) * 2.0 ** -46)
    assert np.all(np.abs(got - ref) <= bound)
