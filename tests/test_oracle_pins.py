"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these tests compares the oracle with itself: each checks it against
a closed form, a brute-force computation of a different kind, an invariant
proved in the paper, or a value printed in the paper.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import gsi_oracle as O
from paper_2306_10379_gb300 import inputs as I
from tests.jacobi_ref import jacobi_eigh

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_spd(n, seed, lo=0.5, hi=3.0):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.sort(rng.uniform(lo, hi, n))[::-1]
    return (Q * lam) @ Q.T, lam, Q


def _orth(n, p, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, p)))
    return Q


def _dense_lap(dims):
    A = I.fd_laplacian(dims)
    return O.csr_operator(A.n, A.rowptr, A.colidx, A.val).toarray()


# ---------------------------------------------------------------- inputs

def test_fd_laplacian_is_kronecker_sum():
    """The stencil CSR equals sum_a I x .. x T_a x .. x I with T = tridiag(-1, 2, -1)."""
    dims = (4, 3, 5)
    def T(d):
        return 2 * np.eye(d) - np.eye(d, k=1) - np.eye(d, k=-1)
    n = int(np.prod(dims))
    K = np.zeros((n, n))
    # index = i0 + d0*(i1 + d1*i2): axis 0 is fastest -> rightmost Kronecker factor
    for a in range(3):
        mats = [np.eye(d) for d in dims]
        mats[a] = T(dims[a])
        M = mats[2]
        M = np.kron(M, mats[1])
        M = np.kron(M, mats[0])
        K += M
    assert np.array_equal(_dense_lap(dims), K)


def test_jacobi_reference_matches_closed_form():
    """The hand-written Jacobi solver reproduces the closed-form FD spectrum."""
    for dims in [(17,), (6, 5), (3, 4, 2)]:
        w, V = jacobi_eigh(_dense_lap(dims))
        ref = I.laplacian_eigenvalues(dims)
        assert np.max(np.abs(w - ref)) < 1e-12
        assert np.max(np.abs(V.T @ V - np.eye(len(w)))) < 1e-12


def test_fd3d_condition_numbers_match_paper():
    """Sec. 6.3, FD3D table: kappa = (l1 - ln)/(lp - lp+1) is 3.53e4 for the
    min problem with p = 64 and 5.54e3 for the max problem with p = 32."""
    with open(os.path.join(GOLDEN, "fd3d_kappa.json")) as f:
        g = json.load(f)
    lam = I.laplacian_eigenvalues(tuple(g["grid"]))
    L = lam[0] - lam[-1]
    for row in g["rows"]:
        p = row["p"]
        lv = lam if row["type"] == "max" else -lam[::-1]
        kappa = L / (lv[p - 1] - lv[p])
        assert f"{kappa:.2e}" == row["kappa"]


def test_philox_known_answers():
    """Philox-4x32-10 known-answer vectors (Random123 distribution kat file)."""
    with open(os.path.join(GOLDEN, "philox_kat.json")) as f:
        kat = json.load(f)
    for case in kat["cases"]:
        ctr = np.array([[int(x, 16) for x in case["ctr"]]], dtype=np.uint64)
        key = tuple(int(x, 16) for x in case["key"])
        out = I.philox4x32_10(ctr, key)[0]
        assert [f"{int(x):08x}" for x in out] == case["out"]


def test_gaussian_moments():
    z = I.gaussian(200000, 7)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1) < 0.01


def test_er_laplacian_structure():
    A = I.er_laplacian(3000, 11)
    D = O.csr_operator(A.n, A.rowptr, A.colidx, A.val)
    off = D - __import__("scipy.sparse", fromlist=["diags"]).diags(D.diagonal())
    assert (abs(D - D.T)).max() == 0
    assert off.nnz == 2 * 4 * 3000                  # M = 4n distinct undirected edges
    rows = np.asarray(abs(off).sum(axis=1)).ravel()
    shift = D.diagonal() - rows
    assert np.all((shift >= 0) & (shift <= 1))
    # every entry (degree + shift on the diagonal) is exactly a float32
    assert np.all(A.val.astype(np.float32).astype(np.float64) == A.val)


# ---------------------------------------------------------- line search

def _ls_problem(n=60, p=5, seed=0, cg=False):
    A, lam, _ = _rand_spd(n, seed)
    X = _orth(n, p, seed + 1)
    Y = A @ X
    C = X.T @ Y
    R = Y - X @ C
    if cg:
        rng = np.random.default_rng(seed + 2)
        E = rng.standard_normal((n, p))
        D = R + 0.3 * (E - X @ (X.T @ E)) * np.linalg.norm(R) / np.linalg.norm(E)
    else:
        D = R
    W = A @ D
    B, Gam, Z = D.T @ D, D.T @ W, D.T @ Y
    a, b, g, z, V = O.ls_coefficients(C, B, 0.5 * (Gam + Gam.T), Z)
    return A, lam, X, D, R, (a, b, g, z, V)


@pytest.mark.parametrize("cg", [False, True])
def test_phi_model_equals_explicit_trace(cg):
    """Eq. (phinew)/(phi_P): the rational model equals -1/2 tr(Q^T A Q) for an
    orthonormal basis Q of span(X + tD) obtained by Householder QR."""
    A, lam, X, D, R, (a, b, g, z, V) = _ls_problem(cg=cg)
    for t in [0.0, 0.05, 0.3, 1.0, 4.0, 40.0]:
        Q, _ = np.linalg.qr(X + t * D)
        explicit = -0.5 * np.trace(Q.T @ A @ Q)
        assert abs(O.phi_model(t, a, b, g, z) - explicit) <= 1e-13 * abs(explicit)


@pytest.mark.parametrize("cg", [False, True])
def test_dphi_matches_finite_difference(cg):
    A, lam, X, D, R, c = _ls_problem(seed=3, cg=cg)
    for t in [0.01, 0.2, 0.7, 2.0]:
        h = 1e-5 * max(t, 1e-3)
        fd = (O.phi_model(t + h, *c[:4]) - O.phi_model(t - h, *c[:4])) / (2 * h)
        assert abs(O.dphi_model(t, *c[:4]) - fd) <= 1e-6 * max(1.0, abs(fd))


def test_dphi_at_zero_is_minus_gradient_norm():
    """Footnote to Eq. (dqnew): phi'(0) = -sum beta_i = -||G||_F^2 (SD)."""
    A, lam, X, D, R, (a, b, g, z, V) = _ls_problem(seed=4)
    assert abs(O.dphi_model(0.0, a, b, g, z) + np.sum(R * R)) <= 1e-13 * np.sum(R * R)


def test_gamma_over_beta_in_spectrum():
    """Eq. (gamRel): gamma_i / beta_i is a Rayleigh quotient of A."""
    A, lam, X, D, R, (a, b, g, z, V) = _ls_problem(seed=5)
    q = g / b
    assert np.all(q <= lam[0] + 1e-12) and np.all(q >= lam[-1] - 1e-12)


def test_grad_norm_bound():
    """||G||_2 <= L/2 with L = lambda_max - lambda_min (Lemma upper_bound_grad)."""
    for s in range(5):
        A, lam, X, D, R, _ = _ls_problem(seed=10 + s)
        assert np.linalg.norm(R, 2) <= 0.5 * (lam[0] - lam[-1]) + 1e-12


def test_branch_roots_are_roots():
    """Each bracket end xi_i zeroes its branch numerator (Eq. (xii)); the
    stable forms (derv1)/(derv2) agree with the plain quadratic formula."""
    A, lam, X, D, R, (a, b, g, z, V) = _ls_problem(seed=6)
    xs = O.branch_roots(a, b, g, z)
    assert xs.size == len(b) and np.all(xs > 0)
    for x, ai, bi, gi in zip(xs, a, b, g):
        d = gi - ai * bi
        plain = (d + math.sqrt(d * d + 4 * bi ** 3)) / (2 * bi * bi)
        assert abs(x - plain) <= 1e-9 * plain
        num = bi + d * x - bi * bi * x * x
        assert abs(num) <= 1e-10 * (bi + abs(d) * x + bi * bi * x * x)


@pytest.mark.parametrize("seed", range(6))
def test_get_mu_is_global_minimum(seed):
    """The Brent step minimises the model on [0, 2 xi_max] (dense scan)."""
    A, lam, X, D, R, (a, b, g, z, V) = _ls_problem(seed=20 + seed, cg=bool(seed % 2))
    t, ev, lo, hi = O.get_mu(a, b, g, z)
    grid = np.linspace(0.0, 2.0 * max(hi, t), 20001)
    vals = np.array([O.phi_model(s, a, b, g, z) for s in grid])
    f = O.phi_model(t, a, b, g, z)
    assert f <= vals.min() + 1e-13 * abs(f)
    assert abs(O.dphi_model(t, a, b, g, z)) <= 1e-10 * np.sum(b)
    assert ev <= 30


def test_get_mu_single_column_closed_form():
    """p = 1: phi' has one branch, so the exact step is its positive root xi_1."""
    A, lam, X, D, R, (a, b, g, z, V) = _ls_problem(p=1, seed=8)
    t, ev, lo, hi = O.get_mu(a, b, g, z)
    d = g[0] - a[0] * b[0]
    xi = (d + math.sqrt(d * d + 4 * b[0] ** 3)) / (2 * b[0] ** 2)
    assert abs(t - xi) <= 1e-14 * xi


@pytest.mark.parametrize("f,a,b,root", [
    (lambda x: math.cos(x) - x, 0.0, 1.0, 0.7390851332151607),
    (lambda x: x ** 3 - 2.0, 0.0, 3.0, 2.0 ** (1.0 / 3.0)),
    (lambda x: math.exp(x) - 10.0, 0.0, 5.0, math.log(10.0)),
    (lambda x: (x - 1e-3) * (1 + x * x), -2.0, 7.0, 1e-3),
])
def test_brent_closed_form_roots(f, a, b, root):
    r, ev = O.brent_zero(f, a, b, f(a), f(b))
    assert abs(r - root) <= 4 * O.EPS * abs(root) + 1e-300
    assert ev < 60


def test_polar_factor_matches_svd():
    """Eq. (Ynew): (X + tD) V D_t^{-1} V^T is the polar factor U W^T of X + tD."""
    A, lam, X, D, R, (a, b, g, z, V) = _ls_problem(seed=9)
    t = 0.7
    Xn = (X + t * D) @ O.polar_factor_matrix(V, b, t)
    U, s, Wt = np.linalg.svd(X + t * D, full_matrices=False)
    assert np.max(np.abs(Xn - U @ Wt)) < 1e-14
    assert np.max(np.abs(Xn.T @ Xn - np.eye(X.shape[1]))) < 1e-14


# ------------------------------------------------------------- whole method

def _lap_problem(dims, p, seed=1):
    A = I.fd_laplacian(dims)
    S = O.csr_operator(A.n, A.rowptr, A.colidx, A.val)
    X0 = I.start_block(A.n, p, seed)
    lam = I.laplacian_eigenvalues(dims)
    return S, X0, lam


def test_sufficient_decrease_and_monotone_sd():
    """Lemma conv2: phi_k - phi_{k+1} >= (2/5) ||G_k||_F^2 / L for SD with exact
    line search; hence phi is non-increasing."""
    S, X0, lam = _lap_problem((12, 10), 4)
    L = lam[0] - lam[-1]
    phis, grads = [], []
    def cb(k, X, Y, t):
        phis.append(-0.5 * np.trace(X.T @ (S @ X)))
    o = O.Options(method="sd", tol=1e-9, anorm=lam[0], max_iters=60)
    res = O.solve(S, X0, o, record=True, callback=cb)
    phi0 = -0.5 * np.trace(O.orthonormalize(X0).T @ (S @ O.orthonormalize(X0)))
    seq = [phi0] + phis
    for k, rec in enumerate(res.history):
        assert seq[k] - seq[k + 1] >= 0.4 * rec.res_f ** 2 / L - 1e-12 * abs(seq[k])


def test_cg_phi_non_increasing():
    S, X0, lam = _lap_problem((12, 10), 4, seed=2)
    phis = []
    o = O.Options(method="cg", tol=1e-10, anorm=lam[0], max_iters=200)
    O.solve(S, X0, o, callback=lambda k, X, Y, t: phis.append(-0.5 * np.trace(X.T @ (S @ X))))
    assert all(b <= a + 1e-12 * abs(a) for a, b in zip(phis, phis[1:]))


@pytest.mark.parametrize("method", ["sd", "cg"])
def test_converges_to_closed_form_2d(method):
    """2D 5-point Laplacian on a 32 x 32 grid, p = 8: the Ritz values at
    relative residual 1e-8 match 4 sin^2(i pi/66) + 4 sin^2(j pi/66)."""
    S, X0, lam = _lap_problem((32, 32), 8, seed=I.SEED_BASE + 0)
    o = O.Options(method=method, tol=1e-8, anorm=lam[0], max_iters=20000)
    res = O.solve(S, X0, o)
    assert res.converged
    theta, Xr, _ = O.rayleigh_ritz(res.X, S @ res.X)
    assert np.max(np.abs(theta - lam[:8]) / lam[:8]) < 1e-10
    # the explicit residual confirms the recursive one
    R = S @ Xr - Xr * theta
    assert np.linalg.norm(R) / lam[0] <= 1e-8
    assert np.max(np.abs(res.X.T @ res.X - np.eye(8))) < 1e-13


def test_iteration_counts_follow_rates():
    """Sec. 6.2: iteration counts are predicted by gamma_SD = ((k-1)/(k+1))^2 and
    gamma_CG = ((sqrt k - 1)/(sqrt k + 1))^2 with kappa = (l1 - ln)/(lp - lp+1)."""
    S, X0, lam = _lap_problem((32, 32), 8, seed=3)
    kappa = (lam[0] - lam[-1]) / (lam[7] - lam[8])
    g_sd = ((kappa - 1) / (kappa + 1)) ** 2
    g_cg = ((math.sqrt(kappa) - 1) / (math.sqrt(kappa) + 1)) ** 2
    its = {}
    for m in ["sd", "cg"]:
        its[m] = O.solve(S, X0, O.Options(method=m, tol=1e-8, anorm=lam[0], max_iters=20000)).iters
    # residual^2 ~ error in phi: a 1e-8 residual is ~1e-16 in phi
    pred_sd = math.log(1e-16) / math.log(g_sd)
    pred_cg = math.log(1e-16) / math.log(g_cg)
    assert 0.3 * pred_sd < its["sd"] < 2.0 * pred_sd
    assert 0.3 * pred_cg < its["cg"] < 2.0 * pred_cg
    assert its["cg"] < its["sd"] / 4


def test_min_problem_via_negation():
    """Sec. 2.1: the smallest eigenvalues are found by applying the method to -A."""
    S, X0, lam = _lap_problem((10, 9), 3)
    res = O.solve(-S, X0, O.Options(method="cg", tol=1e-9, anorm=lam[0]))
    theta, _, _ = O.rayleigh_ritz(res.X, -(S @ res.X))
    assert np.max(np.abs(-theta - lam[::-1][:3])) < 1e-12 * lam[0] * 1e3


def test_subspace_matches_jacobi_on_tiny_problem():
    """Brute force: the converged subspace equals the top-p eigenvectors from the
    hand-written Jacobi solver (principal angle within the Davis-Kahan bound)."""
    import scipy.sparse as sp
    A, lam, Q = _rand_spd(40, 31, lo=-1.0, hi=2.0)
    w, V = jacobi_eigh(A)
    p = 4
    res = O.solve(sp.csr_matrix(A), I.start_block(40, p, 5),
                  O.Options(method="cg", tol=1e-12, anorm=abs(w).max()))
    assert res.converged
    ang = O.principal_angles(res.X, V[:, :p]).max()
    R = A @ res.X - res.X @ (res.X.T @ A @ res.X)
    assert ang <= 2 * np.linalg.norm(R) / (w[p - 1] - w[p]) + 1e-13


def test_shift_invariance_of_iterates():
    """Sec. 6.3: the iterates for A and A + cI coincide (R and the line-search
    data are shift invariant)."""
    S, X0, lam = _lap_problem((9, 8), 3)
    import scipy.sparse as sp
    Xs = {}
    for c in [0.0, 5.0]:
        T = S + c * sp.eye(S.shape[0])
        traj = []
        O.solve(T, X0, O.Options(method="cg", tol=0.0, anorm=1.0, max_iters=12, recompute_every=0),
                callback=lambda k, X, Y, t: traj.append(X.copy()))
        Xs[c] = traj
    for a, b in zip(Xs[0.0], Xs[5.0]):
        assert np.max(np.abs(a - b)) < 1e-10


def test_representative_equivariance():
    """With the polar retraction, starting from X0 W (W orthogonal) gives X_k W."""
    S, X0, lam = _lap_problem((9, 8), 3)
    W = _orth(3, 3, 4)
    X0o = O.orthonormalize(X0)
    runs = []
    for start in [X0o, X0o @ W]:
        traj = []
        O.solve(S, start, O.Options(method="cg", tol=0.0, anorm=1.0, max_iters=10, recompute_every=0),
                callback=lambda k, X, Y, t: traj.append(X.copy()))
        runs.append(traj)
    for a, b in zip(*runs):
        assert np.max(np.abs(a @ W - b)) < 1e-10


# ------------------------------------------------------------- Chebyshev SI

def test_chebyshev_filter_equals_polynomial():
    """Eq. (optimal_poly): the three-term recurrence applies
    C_d((A - cI)/h) / C_d((l1 - c)/h) (Chebyshev closed form cos/cosh(d acos/acosh))."""
    A, lam, Q = _rand_spd(30, 41, lo=0.0, hi=4.0)
    p, d = 3, 7
    c = 0.5 * (lam[p] + lam[-1]); h = 0.5 * (lam[p] - lam[-1])
    def cheb(d, x):
        x = np.asarray(x, dtype=np.float64)
        out = np.empty_like(x)
        inside = np.abs(x) <= 1
        out[inside] = np.cos(d * np.arccos(x[inside]))
        out[~inside] = np.sign(x[~inside]) ** d * np.cosh(d * np.arccosh(np.abs(x[~inside])))
        return out
    X = _orth(30, p, 2)
    ref = (Q * (cheb(d, (lam - c) / h) / cheb(d, np.array([(lam[0] - c) / h]))[0])) @ Q.T @ X
    got = O.chebyshev_filter(A, X, d, c, h, lam[0])
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))


def test_chebyshev_si_converges_to_closed_form():
    S, X0, lam = _lap_problem((16, 16), 6, seed=9)
    X, theta, outer, mv, rel = O.chebyshev_si(S, X0, 8, lam[6], lam[-1], lam[0], tol=1e-9, anorm=lam[0])
    assert rel <= 1e-9
    assert np.max(np.abs(theta - lam[:6])) < 1e-12 * 1e3


# ------------------------------------------------------------- SELL-C-sigma

def test_sell_layout_invariants():
    A = I.er_laplacian(777, 3)
    perm, cptr, clen, scol, sval = O.sell_c_sigma(A.n, A.rowptr, A.colidx, A.val, C=32, sigma=32)
    real = perm[perm >= 0]
    assert np.array_equal(np.sort(real), np.arange(A.n))
    lens = np.diff(A.rowptr)
    X = np.random.default_rng(0).standard_normal((A.n, 5))
    W = np.zeros((A.n, 5))
    for ch in range(len(clen)):
        rows = perm[ch * 32:(ch + 1) * 32]
        assert clen[ch] == max(lens[r] for r in rows if r >= 0)
        for lane, r in enumerate(rows):
            for j in range(clen[ch]):
                slot = cptr[ch] + j * 32 + lane
                if r >= 0 and j < lens[r]:
                    assert scol[slot] == A.colidx[A.rowptr[r] + j]
                else:
                    assert sval[slot] == 0.0
                if r >= 0:
                    W[r] += sval[slot] * X[scol[slot]]
    ref = O.csr_operator(A.n, A.rowptr, A.colidx, A.val) @ X
    assert np.max(np.abs(W - ref)) < 1e-12 * np.max(np.abs(ref))
    # windows of sigma rows are sorted by length, descending
    for w0 in range(0, A.n, 32):
        seg = [lens[r] for r in perm[w0:w0 + 32] if r >= 0]
        assert seg == sorted(seg, reverse=True)
