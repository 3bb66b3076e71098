"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Per-kernel results: normwise relative error <= 1e-12 against the oracle's
float64 result, and bit-exact where both sides are exact (integer layout
work; integer-valued A times dyadic X). Whole-method runs: the first
iterations follow the oracle's trajectory, and the converged subspace meets
the stopping tolerance and the closed-form spectrum.
"""
import math

import numpy as np
import pytest

from oracle import gsi_oracle as O
from paper_2306_10379_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-12




def _dev(torch, a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


# ------------------------------------------------------------------ SpMM

@pytest.mark.parametrize("dims,p", [((11, 7, 5), 1), ((11, 7, 5), 7), ((20, 17, 13), 8),
                                    ((20, 17, 13), 64), ((9, 9, 9), 128), ((33, 31), 6)])
def test_spmm_csr_exact_on_dyadic_inputs(torch_cuda, dims, p):
    """Integer A times dyadic X is exact in float64 on both sides: bit-exact."""
    torch = torch_cuda
    from paper_2306_10379_gb300 import gsi
    A = I.fd_laplacian(dims)
    rng = np.random.default_rng(p)
    X = rng.integers(-1024, 1024, size=(A.n, p)) / 64.0
    ref = O.spmm(O.csr_operator(A.n, A.rowptr, A.colidx, A.val), X)
    W = torch.empty((A.n, p), dtype=torch.float64, device="cuda")
    gsi.spmm_csr(_dev(torch, A.rowptr), _dev(torch, A.colidx), _dev(torch, A.val), _dev(torch, X), W)
    assert np.array_equal(W.cpu().numpy(), ref)


@pytest.mark.parametrize("p", [1, 5, 16, 64])
def test_spmm_csr_random(torch_cuda, p):
    torch = torch_cuda
    from paper_2306_10379_gb300 import gsi
    A = I.er_laplacian(5000, 17)
    X = I.start_block(A.n, p, 3)
    S = O.csr_operator(A.n, A.rowptr, A.colidx, A.val)
    ref = O.spmm(S, X)
    W = torch.empty((A.n, p), dtype=torch.float64, device="cuda")
    gsi.spmm_csr(_dev(torch, A.rowptr), _dev(torch, A.colidx), _dev(torch, A.val), _dev(torch, X), W)
    got = W.cpu().numpy()
    bound = O.spmm(abs(S), np.abs(X))
    assert np.all(np.abs(got - ref) <= TOL * bound)
    assert _rel(got, ref) <= TOL


@pytest.mark.parametrize("n,C,sigma", [(777, 32, 32), (4096, 32, 128), (1, 32, 32)])
def test_sell_layout_bit_exact(torch_cuda, n, C, sigma):
    """The library's host SELL-C-sigma builder equals the oracle's, bit for bit."""
    from paper_2306_10379_gb300 import gsi
    A = I.er_laplacian(max(n, 2), 5) if n > 1 else I.fd_laplacian((1,))
    lib = gsi.csr_to_sell(A.n, A.rowptr, A.colidx, A.val, C, sigma)
    ora = O.sell_c_sigma(A.n, A.rowptr, A.colidx, A.val, C, sigma)
    for a, b in zip(lib, ora):
        assert np.array_equal(np.asarray(a), np.asarray(b))


@pytest.mark.parametrize("p", [3, 32, 64])
def test_spmm_sell(torch_cuda, p):
    torch = torch_cuda
    from paper_2306_10379_gb300 import gsi
    A = I.er_laplacian(3001, 9)
    perm, cptr, clen, scol, sval = gsi.csr_to_sell(A.n, A.rowptr, A.colidx, A.val, 32, 32)
    X = I.start_block(A.n, p, 4)
    ref = O.spmm(O.csr_operator(A.n, A.rowptr, A.colidx, A.val), X)
    W = torch.full((A.n, p), float("nan"), dtype=torch.float64, device="cuda")
    gsi.spmm_sell(A.n, 32, *(_dev(torch, a) for a in (perm, cptr, clen, scol, sval)), _dev(torch, X), W)
    assert _rel(W.cpu().numpy(), ref) <= TOL


# ------------------------------------------------------------------ Gram

@pytest.mark.parametrize("n,p,q", [(10007, 8, 8), (10007, 17, 5), (70001, 64, 64), (3, 1, 1),
                                   (5000, 128, 128), (257, 64, 32)])
def test_gram(torch_cuda, n, p, q):
    torch = torch_cuda
    from paper_2306_10379_gb300 import gsi
    U = I.start_block(n, p, 1)
    V = I.start_block(n, q, 2)
    G = torch.empty((p, q), dtype=torch.float64, device="cuda")
    gsi.gram(_dev(torch, U), _dev(torch, V), G)
    ref = O.gram(U, V)
    bound = np.abs(U).T @ np.abs(V)
    assert np.all(np.abs(G.cpu().numpy() - ref) <= 1e-13 * bound * math.log2(n + 2))


def test_gram_exact_on_dyadic_inputs(torch_cuda):
    torch = torch_cuda
    from paper_2306_10379_gb300 import gsi
    rng = np.random.default_rng(0)
    U = rng.integers(-64, 64, size=(20000, 24)) / 8.0
    V = rng.integers(-64, 64, size=(20000, 24)) / 8.0
    G = torch.empty((24, 24), dtype=torch.float64, device="cuda")
    gsi.gram(_dev(torch, U), _dev(torch, V), G)
    assert np.array_equal(G.cpu().numpy(), O.gram(U, V))


# ---------------------------------------------------- residual, line search, retraction

def _state(dims=(16, 15), p=6, seed=3, cg=False, steps=3):
    """A mid-iteration state taken from the oracle: X, Y, C, R, D, W."""
    A = I.fd_laplacian(dims)
    S = O.csr_operator(A.n, A.rowptr, A.colidx, A.val)
    lam = I.laplacian_eigenvalues(dims)
    snap = {}
    def cb(k, X, Y, t):
        snap["X"], snap["Y"] = X.copy(), Y.copy()
    O.solve(S, I.start_block(A.n, p, seed), O.Options(method="cg" if cg else "sd", tol=0,
            anorm=lam[0], max_iters=steps), callback=cb)
    X, Y = snap["X"], snap["Y"]
    C = O.gram(X, Y); C = 0.5 * (C + C.T)
    R = O.residual(X, Y, C)
    if cg:
        rng = np.random.default_rng(seed)
        E = rng.standard_normal(X.shape)
        D = R + 0.2 * (E - X @ (X.T @ E)) * np.linalg.norm(R) / np.linalg.norm(E)
    else:
        D = R
    W = O.spmm(S, D)
    return S, X, Y, C, R, D, W


@pytest.mark.parametrize("p", [1, 6, 64])
def test_residual(torch_cuda, p):
    torch = torch_cuda
    from paper_2306_10379_gb300 import gsi
    S, X, Y, C, R, D, W = _state(dims=(40, 30), p=p)
    out = torch.empty(X.shape, dtype=torch.float64, device="cuda")
    gsi.residual(_dev(torch, X), _dev(torch, Y), _dev(torch, C), out)
    bound = np.abs(Y) + np.abs(X) @ np.abs(C)
    assert np.all(np.abs(out.cpu().numpy() - R) <= TOL * bound)


@pytest.mark.parametrize("precision", ["df64", "f64"])
@pytest.mark.parametrize("cg,p", [(False, 1), (False, 6), (True, 6), (True, 7), (False, 32), (True, 64),
                                  (True, 100), (False, 128)])
def test_linesearch(torch_cuda, cg, p, precision):
    """Alg. 3 + polar factor: t within 1e-12 (relative), phi(t) within 1e-13,
    M within 1e-12 of the oracle's (Z^T Z)^{-1/2}."""
    torch = torch_cuda
    from paper_2306_10379_gb300 import gsi
    dims = (24, 20) if p <= 32 else (30, 30) if p <= 64 else (40, 40)
    S, X, Y, C, R, D, W = _state(dims=dims, p=p, cg=cg)
    B, Gam, Z = O.gram(D, D), O.gram(D, W), (O.gram(D, R) if cg else O.gram(D, D))
    XX, XD = O.gram(X, X), O.gram(X, D)
    a, b, g, z, V = O.ls_coefficients(C, B, 0.5 * (Gam + Gam.T), Z)
    t_ref, ev, lo, hi = O.get_mu(a, b, g, z)
    Zt = X + t_ref * D
    M_ref = O.inverse_sqrt(O.gram(Zt, Zt))
    M = torch.empty((p, p), dtype=torch.float64, device="cuda")
    out = torch.zeros(16, dtype=torch.float64, device="cuda")
    gsi.linesearch(*(_dev(torch, m) for m in (C, B, Gam, Z, XX, XD)), M, out, precision=precision)
    o = out.cpu().numpy()
    assert o[3] == 0.0
    t = o[0]
    # t is a root of phi'; df64 coefficients move it by ~1e-12 relative, which
    # changes phi(t) only at second order (checked at 1e-13 below)
    assert abs(t - t_ref) <= (1e-12 if precision == "f64" else 1e-10) * t_ref
    phi_ref = O.phi_model(t_ref, a, b, g, z)
    assert abs(O.phi_model(t, a, b, g, z) - phi_ref) <= 1e-13 * abs(phi_ref)
    assert abs(o[1] - phi_ref) <= (1e-13 if precision == "f64" else 1e-12) * abs(phi_ref)
    assert _rel(M.cpu().numpy(), M_ref) <= TOL
    assert abs(o[4] - b.max()) <= (1e-12 if precision == "f64" else 1e-10) * b.max()


def test_retract(torch_cuda):
    torch = torch_cuda
    from paper_2306_10379_gb300 import gsi
    S, X, Y, C, R, D, W = _state(dims=(40, 30), p=16)
    t = 0.37
    Zt = X + t * D
    M = O.inverse_sqrt(O.gram(Zt, Zt))
    Xd, Yd = _dev(torch, X), _dev(torch, Y)
    gsi.retract(t, _dev(torch, M), Xd, _dev(torch, D), Yd, _dev(torch, W))
    assert _rel(Xd.cpu().numpy(), Zt @ M) <= TOL
    assert _rel(Yd.cpu().numpy(), (Y + t * W) @ M) <= TOL


# ------------------------------------------------------------------ whole method

def _trajectory_oracle(S, X0, opts, k):
    traj = []
    O.solve(S, X0, O.Options(**{**opts.__dict__, "max_iters": k}),
            callback=lambda i, X, Y, t: traj.append((X.copy(), t)))
    return traj


@pytest.mark.parametrize("precision", ["df64", "f64"])
@pytest.mark.parametrize("method", ["sd", "cg"])
def test_trajectory_matches_oracle(torch_cuda, method, precision):
    """First 10 iterations of the 2D 32 x 32 problem, p = 8: X_k and t_k agree."""
    from paper_2306_10379_gb300 import gsi
    dims, p = (32, 32), 8
    A = I.fd_laplacian(dims)
    S = O.csr_operator(A.n, A.rowptr, A.colidx, A.val)
    lam = I.laplacian_eigenvalues(dims)
    X0 = I.start_block(A.n, p, I.SEED_BASE)
    opts = O.Options(method=method, tol=1e-8, anorm=lam[0])
    ref = _trajectory_oracle(S, X0, opts, 10)
    with gsi.Solver(A, p, X0, method=method, tol=1e-8, anorm=lam[0], precision=precision) as s:
        for k in range(10):
            info = s.step(1)
            X, _ = s.basis(evals=False)
            Xr, tr = ref[k]
            assert abs(info["last_step"] - tr) <= 1e-10 * tr, k
            assert np.max(np.abs(X - Xr)) <= 1e-10, k


@pytest.mark.parametrize("method,fmt,precision", [("sd", "csr", "df64"), ("cg", "csr", "df64"),
                                                  ("cg", "sell", "df64"), ("sd", "csr", "f64"),
                                                  ("cg", "sell", "f64")])
def test_converges_2d_closed_form(torch_cuda, method, fmt, precision):
    """2D 5-point Laplacian 32 x 32, p = 8: relative residual 1e-8 and Ritz values
    4 sin^2(i pi/66) + 4 sin^2(j pi/66); the subspace is within the Davis-Kahan
    bound of the exact one; X^T X = I."""
    from paper_2306_10379_gb300 import gsi
    dims, p = (32, 32), 8
    A = I.fd_laplacian(dims)
    S = O.csr_operator(A.n, A.rowptr, A.colidx, A.val).toarray()
    lam = I.laplacian_eigenvalues(dims)
    with gsi.Solver(A, p, I.start_block(A.n, p, I.SEED_BASE), method=method, tol=1e-8,
                    anorm=lam[0], fmt=fmt, precision=precision) as s:
        info = s.solve()
        X, ev = s.basis()
    assert info["converged"] == 1 and info["rel_residual"] <= 1e-8
    assert np.max(np.abs(ev - lam[:p]) / lam[:p]) < 1e-10
    R = S @ X - X * ev
    assert np.linalg.norm(R) / lam[0] <= 1.01e-8
    # df64 block products round at ~2^-45
    assert np.max(np.abs(X.T @ X - np.eye(p))) < (1e-13 if precision == "f64" else 5e-13)
    w, U = np.linalg.eigh(S)
    Uex = U[:, ::-1][:, :p]
    ang = O.principal_angles(X, Uex).max()
    assert ang <= 2 * np.linalg.norm(R) / (lam[p - 1] - lam[p]) + 1e-12
    # iteration counts against the oracle's (same start, same rules)
    ores = O.solve(O.csr_operator(A.n, A.rowptr, A.colidx, A.val), I.start_block(A.n, p, I.SEED_BASE),
                   O.Options(method=method, tol=1e-8, anorm=lam[0]))
    assert abs(info["iters"] - ores.iters) <= max(2, 0.02 * ores.iters)


@pytest.mark.parametrize("precision", ["df64", "f64"])
def test_min_problem(torch_cuda, precision):
    """which = -1 runs on -A and returns the smallest eigenvalues (Sec. 2.1)."""
    from paper_2306_10379_gb300 import gsi
    dims, p = (14, 13), 4
    A = I.fd_laplacian(dims)
    lam = I.laplacian_eigenvalues(dims)
    with gsi.Solver(A, p, I.start_block(A.n, p, 2), method="cg", which=-1, tol=1e-9,
                    anorm=lam[0], precision=precision) as s:
        info = s.solve()
        X, ev = s.basis()
    assert info["converged"] == 1
    assert np.max(np.abs(ev - lam[::-1][:p])) < 1e-9


def test_breakdown_on_rank_deficient_start(torch_cuda):
    from paper_2306_10379_gb300 import gsi
    A = I.fd_laplacian((10, 10))
    X0 = I.start_block(A.n, 4, 1)
    X0[:, 3] = X0[:, 2]
    with pytest.raises(gsi.GsiError) as e:
        gsi.Solver(A, 4, X0)
    assert e.value.status == gsi.GSI_ERR_BREAKDOWN


def test_nonconvergence_status(torch_cuda):
    from paper_2306_10379_gb300 import gsi
    A = I.fd_laplacian((20, 20))
    with gsi.Solver(A, 4, I.start_block(A.n, 4, 1), max_iters=5) as s:
        info = s.solve()
        assert info["converged"] == 0 and info["iters"] == 5
        with pytest.raises(gsi.GsiError) as e:
            s.solve(raise_on_noconv=True)
        assert e.value.status == gsi.GSI_ERR_NOCONV


@pytest.mark.parametrize("p", [1, 6, 100])
def test_df64_solver_odd_sizes(torch_cuda, p):
    """Whole method in df64 with p outside the 16-multiple tile grid and p > 64
    (two output column slices): converges to the closed-form spectrum."""
    from paper_2306_10379_gb300 import gsi
    dims = (20, 19, 3) if p <= 6 else (30, 29)
    A = I.fd_laplacian(dims)
    lam = I.laplacian_eigenvalues(dims)
    gap = lam[p - 1] - lam[p]
    assert gap > 1e-6
    with gsi.Solver(A, p, I.start_block(A.n, p, 4), method="cg", tol=1e-9, anorm=lam[0],
                    max_iters=5000) as s:
        info = s.solve()
        X, ev = s.basis()
    assert info["converged"] == 1
    assert np.max(np.abs(ev - lam[:p])) <= 1e-12 * lam[0] + 2 * (1e-9 * lam[0]) ** 2 / gap * 10
    assert np.max(np.abs(X.T @ X - np.eye(p))) < 1e-12


def test_reset_and_profile(torch_cuda):
    from paper_2306_10379_gb300 import gsi
    dims, p = (24, 24), 8
    A = I.fd_laplacian(dims)
    lam = I.laplacian_eigenvalues(dims)
    X0 = I.start_block(A.n, p, 1)
    with gsi.Solver(A, p, X0, method="cg", tol=1e-8, anorm=lam[0]) as s:
        i1 = s.solve()
        s.profile(True)
        s.reset(X0)
        n0 = gsi.launch_count()
        i2 = s.solve()
        prof = s.profile_read()
        assert gsi.launch_count() > n0
    assert i1["iters"] == i2["iters"] and i1["rel_residual"] == i2["rel_residual"]
    assert prof["spmm"]["launches"] == i2["matvecs"]  # includes the start-block matvec of reset
    assert all(prof[k]["ms"] > 0 for k in ("spmm", "gram", "blockmul", "small"))


def test_fused_row_norm_matches_separate_pass(torch_cuda):
    """max_r sum_j |R[r, j]| formed in the tcgen05 block product's row-wise
    epilogue (tensor path 0, p even <= 64) against the separate reduction
    kernel (mma.sync path 1, where the product does not form it). The two
    paths' Grams round differently (512/256- against 64-row exponent
    chunks), so the runs agree to rounding: same iteration count, residuals
    within 1e-4 relative, infinity-norm residuals within 1e-3 (a lost row or a
    wrong reduction would be off by far more)."""
    from paper_2306_10379_gb300 import gsi
    dims, p = (30, 28), 8
    A = I.fd_laplacian(dims)
    lam = I.laplacian_eigenvalues(dims)
    out = []
    for path in (0, 1):
        gsi.set_tensor_path(path)
        try:
            with gsi.Solver(A, p, I.start_block(A.n, p, 5), method="cg", tol=1e-8, anorm=lam[0]) as s:
                out.append(s.solve())
        finally:
            gsi.set_tensor_path(0)
    a, b = out
    assert a["iters"] == b["iters"]
    assert abs(a["rel_residual"] - b["rel_residual"]) <= 1e-4 * b["rel_residual"]
    assert np.isfinite(a["rel_residual_inf"]) and a["rel_residual_inf"] > 0
    assert abs(a["rel_residual_inf"] - b["rel_residual_inf"]) <= 1e-3 * b["rel_residual_inf"]


@pytest.mark.parametrize("dims,p,precision", [((32, 32), 8, "df64"), ((32, 32), 7, "df64"),
                                              ((32, 32), 8, "f64"), ((16, 16, 16), 64, "df64")])
def test_residual_inf_matches_oracle(torch_cuda, dims, p, precision):
    """The paper's table criterion ||R_k||_inf / ||R_0||_inf (largest row sum of
    |R|, Table "Comparison of LOBCG and Riemannian CG") over the first 10 CG
    iterations, against the oracle's record from the same start. df64: the row
    sums are float32 sums of the high words -- formed in the tcgen05 block
    product's epilogue for even p <= 64 (a 6-level tree per row), in a separate
    reduction otherwise (p - 1 sequential adds) -- so each norm is within
    (p + 1) 2^-24 relative of the exact one and the ratio within twice that.
    float64: a float64 reduction, 1e-12. Both plus the trajectory's own drift
    (iterates within 1e-10 of the oracle's), 1e-9 absolute."""
    from paper_2306_10379_gb300 import gsi
    A = I.fd_laplacian(dims)
    S = O.csr_operator(A.n, A.rowptr, A.colidx, A.val)
    lam = I.laplacian_eigenvalues(dims)
    X0 = I.start_block(A.n, p, I.SEED_BASE)
    hist = O.solve(S, X0, O.Options(method="cg", tol=1e-8, anorm=lam[0], max_iters=10), record=True).history
    assert len(hist) == 10
    rel = 2.0 * (p + 1) * 2.0 ** -24 if precision == "df64" else 1e-12
    worst = 0.0
    with gsi.Solver(A, p, X0, method="cg", tol=1e-8, anorm=lam[0], precision=precision) as s:
        for k in range(10):
            got = s.step(1)["rel_residual_inf"]
            want = hist[k].res_inf
            assert abs(got - want) <= rel * want + 1e-9, (k, got, want)
            worst = max(worst, abs(got - want) / want)
    assert hist[-1].res_inf < hist[0].res_inf  # the criterion moved over the 10 steps


@pytest.mark.parametrize("precision", ["df64", "f64"])
def test_iteration_count_3d_matches_oracle(torch_cuda, precision):
    """The bench's form (3D 7-point Laplacian, p = 64, CG, CSR) at a size the
    oracle solves in seconds: 18 x 20 x 22 (n = 7920, gap lambda_64 -
    lambda_65 = 1.0e-2). Whole-solve iteration counts within 2% of the
    oracle's from the same start block, Ritz values within 1e-10 of the
    closed form."""
    from paper_2306_10379_gb300 import gsi
    dims, p = (18, 20, 22), 64
    A = I.fd_laplacian(dims)
    lam = I.laplacian_eigenvalues(dims)
    X0 = I.start_block(A.n, p, I.SEED_BASE + 1)
    with gsi.Solver(A, p, X0, method="cg", tol=1e-8, anorm=lam[0], precision=precision) as s:
        info = s.solve()
        _, ev = s.basis()
    ores = O.solve(O.csr_operator(A.n, A.rowptr, A.colidx, A.val), X0,
                   O.Options(method="cg", tol=1e-8, anorm=lam[0]))
    assert info["converged"] == 1 and ores.converged
    assert abs(info["iters"] - ores.iters) <= max(2, 0.02 * ores.iters), (info["iters"], ores.iters)
    assert np.max(np.abs(ev - lam[:p]) / lam[:p]) < 1e-10
