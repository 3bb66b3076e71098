"""Parity of the df64 / Ozaki-split tensor-core kernels with the CPU oracle.

Inputs are float64 values rounded to df64 (hi + lo, 48-bit significand); the
oracle computes with those exact values in float64. Bounds follow the
construction: operands are cut at 2^-49 of a row/column/chunk maximum, so
errors are measured against products of those maxima.
"""
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


def _df_dev(torch, gsi, x):
    return torch.from_numpy(gsi.to_df(x)).cuda()


def _exact(gsi, x):
    return gsi.from_df(gsi.to_df(x))


@pytest.mark.parametrize("p", [1, 2, 7, 8, 16, 32, 64, 100, 128])
def test_df_spmm(G, p):
    torch, gsi = G
    A = I.er_laplacian(20011, 3)
    X = _exact(gsi, I.start_block(A.n, p, 1))
    val = _exact(gsi, A.val * (1 + 1e-9 * np.arange(A.nnz) / A.nnz))  # non-integer values
    S = O.csr_operator(A.n, A.rowptr, A.colidx, val)
    W = torch.empty((A.n, p, 2), dtype=torch.float32, device="cuda")
    gsi.df_spmm_csr(torch.from_numpy(A.rowptr).cuda(), torch.from_numpy(A.colidx).cuda(),
                    _df_dev(torch, gsi, val), _df_dev(torch, gsi, X), W)
    got = gsi.from_df(W.cpu().numpy())
    ref = O.spmm(S, X)
    assert np.all(np.abs(got - ref) <= 1e-13 * O.spmm(abs(S), np.abs(X)))


def test_df_spmm_empty_rows_and_unaligned_blocks(G):
    """Rows without nonzeros give zero rows; blocks that are not 16-byte
    aligned take the per-column-pair kernel, which sums in the same order as
    the row-group kernel: bit-identical results."""
    torch, gsi = G
    p = 64
    A = I.er_laplacian(5003, 11)
    rp = A.rowptr.copy()
    keep = np.ones(A.nnz, bool)
    empty = np.arange(0, A.n, 97)
    for r in empty:  # drop every nonzero of these rows
        keep[rp[r]:rp[r + 1]] = False
    cnt = np.diff(rp).copy()
    cnt[empty] = 0
    rowptr = np.concatenate([[0], np.cumsum(cnt)]).astype(np.int64)
    colidx, val = A.colidx[keep], A.val[keep]
    X = _exact(gsi, I.start_block(A.n, p, 2))
    S = O.csr_operator(A.n, rowptr, colidx, val)
    args = (torch.from_numpy(rowptr).cuda(), torch.from_numpy(colidx).cuda(), _df_dev(torch, gsi, val))
    W = torch.empty((A.n, p, 2), dtype=torch.float32, device="cuda")
    gsi.df_spmm_csr(*args, _df_dev(torch, gsi, X), W)
    got = gsi.from_df(W.cpu().numpy())
    assert np.all(got[empty] == 0.0)
    assert np.all(np.abs(got - O.spmm(S, X)) <= 1e-13 * O.spmm(abs(S), np.abs(X)))
    # the same product from blocks 8 bytes off a 16-byte boundary
    xb = torch.empty((A.n * p + 1, 2), dtype=torch.float32, device="cuda")
    wb = torch.empty((A.n * p + 1, 2), dtype=torch.float32, device="cuda")
    Xu, Wu = xb[1:].view(A.n, p, 2), wb[1:].view(A.n, p, 2)
    Xu.copy_(_df_dev(torch, gsi, X))
    gsi.df_spmm_csr(*args, Xu, Wu)
    assert torch.equal(Wu, W)


@pytest.mark.parametrize("n,p,nk,ne", [(1, 1, 1, 0), (33, 8, 1, 1), (1000, 17, 2, 2), (100003, 64, 1, 1),
                                       (50001, 64, 2, 0), (20000, 100, 1, 2), (20000, 128, 2, 1),
                                       (777, 5, 2, 2)])
def test_oz_gemm(G, n, p, nk, ne):
    torch, gsi = G
    rng = np.random.default_rng(n + p)
    U = [_exact(gsi, rng.standard_normal((n, p)) * np.exp(rng.uniform(-3, 3, (n, 1)))) for _ in range(nk)]
    M = [rng.standard_normal((p, p)) * np.exp(rng.uniform(-2, 2, (1, p))) for _ in range(nk)]
    s = [0.7, -1.3][:nk]
    E = [_exact(gsi, rng.standard_normal((n, p))) for _ in range(ne)]
    c = [0.3, -2.5][:ne]
    ref = sum(sk * Uk @ Mk for sk, Uk, Mk in zip(s, U, M)) + sum(cm * Em for cm, Em in zip(c, E))
    out = torch.zeros((n, p, 2), dtype=torch.float32, device="cuda")
    Ud = [_df_dev(torch, gsi, u) for u in U]
    Md = [torch.from_numpy(m).cuda() for m in M]
    gsi.oz_gemm(Ud[0], Md[0], out, s0=s[0], U1=Ud[1] if nk > 1 else None, M1=Md[1] if nk > 1 else None,
                s1=s[1] if nk > 1 else 0.0, E=[_df_dev(torch, gsi, e) for e in E], c=c)
    got = gsi.from_df(out.cpu().numpy())
    # bound: K terms, each cut at 2^-49 of its row max times its column max
    bound = sum(abs(sk) * np.abs(Uk).max(1, keepdims=True) * np.abs(Mk).max(0, keepdims=True)
                for sk, Uk, Mk in zip(s, U, M)) * (nk * p) * 2.0 ** -44
    bound = bound + sum(abs(cm) * np.abs(Em) for cm, Em in zip(c, E)) * 2.0 ** -46
    assert np.all(np.abs(got - ref) <= bound + 1e-300)
    assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(ref)


def test_oz_gemm_exact_on_grid(G):
    """Operands on the digit grid (small integers times a row power of two)
    are represented exactly, so the products are exact: bit-equal results."""
    torch, gsi = G
    rng = np.random.default_rng(7)
    n, p = 4099, 64
    U = rng.integers(-2 ** 20, 2 ** 20, (n, p)).astype(np.float64) * 2.0 ** rng.integers(-10, 10, (n, 1))
    M = rng.integers(-2 ** 20, 2 ** 20, (p, p)).astype(np.float64) * 2.0 ** -20
    out = torch.zeros((n, p, 2), dtype=torch.float32, device="cuda")
    gsi.oz_gemm(_df_dev(torch, gsi, U), torch.from_numpy(M).cuda(), out)
    ref = U @ M
    got = gsi.from_df(out.cpu().numpy())
    # exact integers up to 2^46 * scale: float64 reference is exact too
    assert np.array_equal(got, ref)


def test_oz_gemm_in_place(G):
    torch, gsi = G
    rng = np.random.default_rng(9)
    n, p = 3001, 32
    U = _exact(gsi, rng.standard_normal((n, p)))
    M = rng.standard_normal((p, p))
    E = _exact(gsi, rng.standard_normal((n, p)))
    Ud = _df_dev(torch, gsi, U)
    Ed = _df_dev(torch, gsi, E)
    gsi.oz_gemm(Ud, torch.from_numpy(M).cuda(), Ud, E=[Ed], c=[1.0])  # U <- U M + E
    assert np.linalg.norm(gsi.from_df(Ud.cpu().numpy()) - (U @ M + E)) <= 1e-13 * np.linalg.norm(U @ M)
    gsi.oz_gemm(_df_dev(torch, gsi, U), torch.from_numpy(M).cuda(), Ed, E=[Ed], c=[-1.0])  # E <- U M - E
    assert np.linalg.norm(gsi.from_df(Ed.cpu().numpy()) - (U @ M - E)) <= 1e-13 * np.linalg.norm(U @ M)


def _gram_bound(U, V, rows=1536):
    """Error bound of the digit-split Gram: per chunk of `rows` rows every
    product is cut at 2^-49 of the chunk's column maxima. Windows of 1536
    rows hold whole exponent chunks of every kernel that may run (64 rows
    for mma.sync; 512, 384 and 256 for the tcgen05 Grams), and a chunk's
    maxima are at most its window's; the unaligned-block kernel's 160-row
    chunks straddle them, for which the 2^-44 factor leaves room."""
    n, p = U.shape
    chunk_bound = np.zeros((p, V.shape[1]))
    for r0 in range(0, n, rows):
        cu = np.abs(U[r0:r0 + rows]).max(0)
        cv = np.abs(V[r0:r0 + rows]).max(0)
        chunk_bound += np.outer(cu, cv) * min(rows, n - r0)
    return 2.0 ** -44 * chunk_bound + 2.0 ** -46 * (np.abs(U).T @ np.abs(V))


@pytest.mark.parametrize("path", [0, 1])
@pytest.mark.parametrize("n,p,q,sym", [(1, 1, 1, False), (63, 8, 8, True), (65, 8, 3, False),
                                       (10007, 64, 64, True), (10007, 64, 64, False),
                                       (200001, 64, 64, True), (30000, 128, 128, True),
                                       (30000, 65, 128, False), (5000, 100, 17, False),
                                       (4099, 48, 64, False), (1000, 33, 33, True), (777, 33, 17, False)])
def test_oz_gram(G, n, p, q, sym, path):
    """Both tensor paths against the oracle's float64 Gram of the same df64
    values (tcgen05 on path 0 -- one 64 x 64 block, or one CTA per block
    when p or q > 64, upper blocks only and mirrored when symmetric;
    mma.sync on path 1)."""
    torch, gsi = G
    rng = np.random.default_rng(n * 3 + p)
    U = _exact(gsi, rng.standard_normal((n, p)) * np.exp(rng.uniform(-4, 4, (1, p))))
    V = U if sym else _exact(gsi, rng.standard_normal((n, q)) * np.exp(rng.uniform(-4, 4, (1, q))))
    Ud = _df_dev(torch, gsi, U)
    Vd = Ud if sym else _df_dev(torch, gsi, V)
    Gm = torch.full((p, q), np.nan, dtype=torch.float64, device="cuda")
    gsi.set_tensor_path(path)
    try:
        gsi.oz_gram(Ud, Vd, Gm, sym=sym)
    finally:
        gsi.set_tensor_path(0)
    got = Gm.cpu().numpy()
    ref = O.gram(U, V)
    assert np.all(np.abs(got - ref) <= _gram_bound(U, V))
    if sym:
        assert np.array_equal(got, got.T)


def _six_digit_block(rng, n, p):
    """Entries sum_{i<6} d_i 2^(-7(i+1)) with large positive digits
    (d_0 in [100, 127], d_1..d_5 in [40, 63]): below 1, 42 significant bits,
    so exact in df64 and cut into exactly these digits (column exponent 0),
    with stacked digit-pair sums near 2^23.3 over the 512-row chunks of the
    U == V kernel (its 2^24 limit allows 582 rows). Returned as
    integers (the value times 2^42) and as float64."""
    d = np.concatenate([rng.integers(100, 128, (n, p, 1)), rng.integers(40, 64, (n, p, 5))], axis=2)
    k = np.zeros((n, p), dtype=np.int64)
    for i in range(6):
        k = k * 128 + d[:, :, i]
    return k, k.astype(np.float64) * 2.0 ** -42


def _exact_gram(ku, kv):
    """U^T V exactly for integer blocks below 2^42 (21-bit halves, int64
    products), returned as Python integers (scaled by 2^84)."""
    hu, lu = ku >> 21, ku & ((1 << 21) - 1)
    hv, lv = kv >> 21, kv & ((1 << 21) - 1)
    hh, hl, lh, ll = hu.T @ hv, hu.T @ lv, lu.T @ hv, lu.T @ lv
    return [[(int(hh[i, j]) << 42) + ((int(hl[i, j]) + int(lh[i, j])) << 21) + int(ll[i, j])
             for j in range(ku.shape[1])] for i in range(ku.shape[1])]


@pytest.mark.parametrize("path", [0, 1])
@pytest.mark.parametrize("n,sym", [(1000, True), (1000, False), (256, True)])
def test_oz_gram_large_digit_sums_exact(G, n, sym, path):
    """Digit-pair sums close to 2^24 (all digits large and positive, up to 512
    rows per exponent chunk) must still be summed exactly by the tensor
    cores: the Gram of these 42-bit entries equals the exact integer Gram to
    df64 rounding (relative 2^-46; a single lost unit in any group sum would
    be 2^-22 or more)."""
    torch, gsi = G
    rng = np.random.default_rng(1234 + n + sym)
    p = 64
    ku, U = _six_digit_block(rng, n, p)
    kv, V = (ku, U) if sym else _six_digit_block(rng, n, p)
    assert np.array_equal(gsi.from_df(gsi.to_df(U)), U)  # exact in df64
    Ud = _df_dev(torch, gsi, U)
    Vd = Ud if sym else _df_dev(torch, gsi, V)
    Gm = torch.full((p, p), np.nan, dtype=torch.float64, device="cuda")
    gsi.set_tensor_path(path)
    try:
        gsi.oz_gram(Ud, Vd, Gm, sym=sym)
    finally:
        gsi.set_tensor_path(0)
    got = Gm.cpu().numpy()
    ex = _exact_gram(ku, kv)
    rel = max(abs(got[i, j] * 2.0 ** 84 - ex[i][j]) / ex[i][j] for i in range(p) for j in range(p))
    assert rel <= 2.0 ** -46, rel


@pytest.mark.parametrize("n,p", [(5000, 64), (3001, 17), (4000, 128)])
def test_oz_gemm_fused_left_sum(G, n, p):
    """Same right operand for both terms: (U0 + a U1) M is formed with the sum
    taken in df64 before the split (the retraction X <- (X + tD) M)."""
    torch, gsi = G
    rng = np.random.default_rng(p)
    U0 = _exact(gsi, rng.standard_normal((n, p)))
    U1 = _exact(gsi, rng.standard_normal((n, p)) * 1e-3)
    M = rng.standard_normal((p, p))
    t = 0.37
    Md = torch.from_numpy(M).cuda()
    out = torch.zeros((n, p, 2), dtype=torch.float32, device="cuda")
    gsi.oz_gemm(_df_dev(torch, gsi, U0), Md, out, s0=1.0, U1=_df_dev(torch, gsi, U1), M1=Md, s1=t)
    ref = (U0 + t * U1) @ M
    got = gsi.from_df(out.cpu().numpy())
    bound = (np.abs(U0) + t * np.abs(U1)).max(1, keepdims=True) * np.abs(M).max(0, keepdims=True) * p * 2.0 ** -44
    assert np.all(np.abs(got - ref) <= bound)


@pytest.mark.parametrize("n,p,fused,ne", [(4099, 64, True, 2), (1000, 16, False, 1), (257, 48, True, 0),
                                          (130, 8, False, 2), (70001, 64, True, 1)])
def test_oz_gemm_tcgen05_equals_mma(G, n, p, fused, ne):
    """The tcgen05 block product (tensor memory accumulators) and the mma.sync
    one sum the same exact integer digit products and combine them in the
    same order: bit-identical results, including the fused left sum
    (X + tD) M and the elementwise terms."""
    torch, gsi = G
    rng = np.random.default_rng(n + 3 * p)
    U0 = _df_dev(torch, gsi, _exact(gsi, rng.standard_normal((n, p)) * np.exp(rng.uniform(-3, 3, (n, 1)))))
    U1 = _df_dev(torch, gsi, _exact(gsi, rng.standard_normal((n, p)))) if fused else None
    M = torch.from_numpy(rng.standard_normal((p, p)) * np.exp(rng.uniform(-2, 2, (1, p)))).cuda()
    E = [_df_dev(torch, gsi, _exact(gsi, rng.standard_normal((n, p)))) for _ in range(ne)]
    outs = []
    for path in (2, 1):
        gsi.set_tensor_path(path)
        out = torch.zeros((n, p, 2), dtype=torch.float32, device="cuda")
        gsi.oz_gemm(U0, M, out, s0=0.7, U1=U1, M1=M if fused else None, s1=0.3 if fused else 0.0,
                    E=E, c=[0.3, -2.5][:ne])
        outs.append(out.cpu().numpy())
    gsi.set_tensor_path(0)
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("n,p,fused,ne", [(4099, 128, True, 2), (3001, 72, False, 1), (1000, 65, True, 0),
                                          (20011, 100, False, 2), (257, 128, False, 0)])
def test_oz_gemm_tcgen05_contraction_slices(G, n, p, fused, ne):
    """p > 64: the tcgen05 block product cuts the contraction into slices of
    at most 64 (each an exact digit product with its own exponents) and sums
    them in df64, so it is a different rounding of the same product than the
    mma.sync kernel's single pass: both within the digit-split bound of the
    float64 product of the exact df64 inputs, and within twice that of each
    other. Odd p puts every other row's start 8 bytes off a 16-byte boundary."""
    torch, gsi = G
    rng = np.random.default_rng(n + 5 * p)
    U0h = _exact(gsi, rng.standard_normal((n, p)) * np.exp(rng.uniform(-3, 3, (n, 1))))
    U1h = _exact(gsi, rng.standard_normal((n, p))) if fused else None
    Mh = rng.standard_normal((p, p)) * np.exp(rng.uniform(-2, 2, (1, p)))
    Eh = [_exact(gsi, rng.standard_normal((n, p))) for _ in range(ne)]
    c = [0.3, -2.5][:ne]
    s0, s1 = 0.7, 0.3
    U0, M = _df_dev(torch, gsi, U0h), torch.from_numpy(Mh).cuda()
    U1 = _df_dev(torch, gsi, U1h) if fused else None
    E = [_df_dev(torch, gsi, e) for e in Eh]
    outs = []
    for path in (2, 1):
        gsi.set_tensor_path(path)
        out = torch.zeros((n, p, 2), dtype=torch.float32, device="cuda")
        gsi.oz_gemm(U0, M, out, s0=s0, U1=U1, M1=M if fused else None, s1=s1 if fused else 0.0, E=E, c=c)
        outs.append(gsi.from_df(out.cpu().numpy()))
    gsi.set_tensor_path(0)
    # the fused left operand s0 (U0 + (s1/s0) U1) is formed in df64 first
    L = s0 * U0h + (s1 * U1h if fused else 0.0)
    ref = L @ Mh + sum(cm * Em for cm, Em in zip(c, Eh))
    bound = (s0 * np.abs(U0h) + (s1 * np.abs(U1h) if fused else 0.0)).max(1, keepdims=True) \
        * np.abs(Mh).max(0, keepdims=True) * p * 2.0 ** -44
    bound = bound + sum(abs(cm) * np.abs(Em) for cm, Em in zip(c, Eh)) * 2.0 ** -46 + np.abs(ref) * 2.0 ** -46
    for o in outs:
        assert np.all(np.abs(o - ref) <= bound)
    assert np.all(np.abs(outs[0] - outs[1]) <= 2 * bound)
    assert np.linalg.norm(outs[0] - ref) <= 1e-13 * np.linalg.norm(ref)


@pytest.mark.parametrize("n,p,q,sym", [(100003, 64, 64, True), (100003, 64, 64, False), (4097, 17, 40, False),
                                       (70, 8, 8, True), (200000, 48, 5, False)])
def test_oz_gram_tcgen05_and_mma_agree(G, n, p, q, sym):
    """The tcgen05 Gram (512/384-row exponent chunks, tensor-memory group
    sums) and the mma.sync one (64-row chunks) are different roundings of the
    same exact Gram: each within the digit-split bound of the oracle, and
    within the sum of the two bounds of each other, on rows whose magnitudes
    vary by e^+-3 (so the chunk exponents differ)."""
    torch, gsi = G
    rng = np.random.default_rng(n + p + q)
    Uh = _exact(gsi, rng.standard_normal((n, p)) * np.exp(rng.uniform(-3, 3, (n, 1))))
    Vh = Uh if sym else _exact(gsi, rng.standard_normal((n, q)))
    U = _df_dev(torch, gsi, Uh)
    V = U if sym else _df_dev(torch, gsi, Vh)
    outs = []
    for path in (2, 1):
        gsi.set_tensor_path(path)
        Gm = torch.zeros((p, q), dtype=torch.float64, device="cuda")
        gsi.oz_gram(U, V, Gm, sym=sym)
        outs.append(Gm.cpu().numpy())
    gsi.set_tensor_path(0)
    bound = _gram_bound(Uh, Vh)
    ref = O.gram(Uh, Vh)
    for o in outs:
        assert np.all(np.abs(o - ref) <= bound)
    assert np.all(np.abs(outs[0] - outs[1]) <= 2 * bound)


def _place(torch, gsi, x, off):
    """df64 copy of x on the device starting `off` float2 entries into a fresh
    buffer (off = 1: 8 bytes past a 16-byte boundary)."""
    d = gsi.to_df(x)
    buf = torch.zeros(d.size + 2 * off, dtype=torch.float32, device="cuda")
    view = buf[2 * off:].view(d.shape)
    view.copy_(torch.from_numpy(d))
    assert (view.data_ptr() % 16 == 0) == (off == 0)
    return view


@pytest.mark.parametrize("sym", [True, False])
def test_oz_gram_unaligned_blocks(G, sym):
    """Blocks that start 8 bytes past a 16-byte boundary take the tcgen05
    Gram that stages whole chunks with 8-byte copies; aligned blocks take the
    one with the maxima warp (bulk copies, other exponent chunks). Both are
    within the digit-split bound of the oracle's Gram of the same values, and
    within twice that of each other; the unaligned result is symmetric when
    U == V."""
    torch, gsi = G
    n, p = 3001, 64
    rng = np.random.default_rng(77 + sym)
    U = _exact(gsi, rng.standard_normal((n, p)) * np.exp(rng.uniform(-3, 3, (n, 1))))
    V = U if sym else _exact(gsi, rng.standard_normal((n, p)))
    outs = []
    for off in (0, 1):
        Ud = _place(torch, gsi, U, off)
        Vd = Ud if sym else _place(torch, gsi, V, off)
        Gm = torch.zeros((p, p), dtype=torch.float64, device="cuda")
        gsi.oz_gram(Ud, Vd, Gm, sym=sym)
        outs.append(Gm.cpu().numpy())
    bound = _gram_bound(U, V)
    ref = O.gram(U, V)
    for o in outs:
        assert np.all(np.abs(o - ref) <= bound)
        if sym:
            assert np.array_equal(o, o.T)
    assert np.all(np.abs(outs[0] - outs[1]) <= 2 * bound)


@pytest.mark.parametrize("fused,ne", [(True, 0), (False, 2)])
def test_oz_gemm_unaligned_blocks(G, fused, ne):
    """Operands and output 8 bytes past a 16-byte boundary: the tcgen05 block
    product reads with 8-byte loads and finishes in its element-wise
    epilogue, with the same result bit for bit."""
    torch, gsi = G
    n, p = 2001, 64
    rng = np.random.default_rng(5 + ne)
    U0 = _exact(gsi, rng.standard_normal((n, p)))
    U1 = _exact(gsi, rng.standard_normal((n, p))) if fused else None
    E = [_exact(gsi, rng.standard_normal((n, p))) for _ in range(ne)]
    M = torch.from_numpy(rng.standard_normal((p, p))).cuda()
    outs = []
    for off in (0, 1):
        out = _place(torch, gsi, np.zeros((n, p)), off)
        gsi.oz_gemm(_place(torch, gsi, U0, off), M, out, s0=0.9,
                    U1=_place(torch, gsi, U1, off) if fused else None, M1=M if fused else None,
                    s1=0.2 if fused else 0.0, E=[_place(torch, gsi, e, off) for e in E], c=[0.5, -1.5][:ne])
        outs.append(out.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])


def test_fma_peaks_are_measured(G):
    """The float64 / float32 FMA throughput probe returns finite rates, the
    float32 pipe well ahead of the float64 one (the premise of the df64
    design)."""
    torch, gsi = G
    pk = gsi.measure_fma_peaks()
    assert np.isfinite(pk["fp64_fma_tflops"]) and pk["fp64_fma_tflops"] > 0
    assert pk["fp32_fma_tflops"] > 4 * pk["fp64_fma_tflops"]
