"""Batched solver on the GPU against the oracle: per-problem trajectories of
Alg. 2 / Alg. 4 over the first passes, whole solves (iteration counts, Ritz
values, residuals, subspaces), the graph and host-loop drivers, the tuner,
the min problem, ragged tiles and the smallest sizes."""
import numpy as np
import pytest

from oracle import gsi_oracle as O
from paper_2306_10379_gb300 import inputs as I

pytestmark = pytest.mark.gpu

# sizes spanning several tiles with ragged tails, every block width
SIZES = (np.array([509, 260, 181, 190, 293, 645, 97], np.int32),
         np.array([4, 32, 2, 8, 32, 16, 8], np.int32))


def _batch(seed=7, sizes=SIZES):
    return I.er_batch(len(sizes[0]), I.SEED_BASE + seed, sizes=sizes)


def _scipy(B):
    return [O.csr_operator(m.n, m.rowptr, m.colidx, m.val) for m in B.mats]


def _anorms(mats):
    return np.array([O.anorm_inf(A) for A in mats])


@pytest.mark.parametrize("method", ["sd", "cg"])
def test_batched_trajectory(torch_cuda, method):
    """X_k and t_k of every problem after each of the first 6 passes agree
    with the oracle's iterates (tile rows 64: several ragged tiles)."""
    from paper_2306_10379_gb300 import gsi
    B = _batch()
    mats = _scipy(B)
    an = _anorms(mats)
    K = 6
    ref = [[] for _ in mats]
    O.batched_solve(mats, B.X0s, O.Options(method=method, tol=1e-8, max_iters=K), anorms=an,
                    callback=lambda i, k, X, Y, t: ref[i].append((X.copy(), t)))
    with gsi.Batch(B, method=method, tol=1e-8, anorm=an) as b:
        b.set_tiles(64, 2, 1)
        for k in range(K):
            b.step(1)
            for i in range(B.nprob):
                X, _ = b.basis(i, evals=False)
                Xr, tr = ref[i][k]
                info = b.info(i)
                assert info["iters"] == k + 1
                assert abs(info["last_step"] - tr) <= 1e-10 * abs(tr), (i, k)
                assert np.max(np.abs(X - Xr)) <= 1e-10, (i, k)


def _check_solution(b, B, mats, an, which=1):
    for i, A in enumerate(mats):
        X, th = b.basis(i)
        info = b.info(i)
        assert info["converged"] == 1 and info["status"] == 0, (i, info)
        p = int(B.p[i])
        Ad = A.toarray()
        lam = np.linalg.eigvalsh(Ad)
        lam = lam[::-1][:p] if which == 1 else lam[:p]
        # orthonormal Ritz vectors with the Ritz values, residual at tolerance
        assert np.max(np.abs(X.T @ X - np.eye(p))) <= 1e-12
        R = Ad @ X - X * th
        assert np.linalg.norm(R) / an[i] <= 1.05e-8, i
        assert np.max(np.abs(th - lam)) <= 1e-8 * an[i] * np.sqrt(p) + 1e-12, i


def test_batched_solve_matches_oracle(torch_cuda):
    """CG on the Erdos-Renyi batch to 1e-8: iteration and restart counts as
    the oracle's, the oracle's subspace, Ritz pairs of the exact spectrum."""
    from paper_2306_10379_gb300 import gsi
    B = _batch()
    mats = _scipy(B)
    an = _anorms(mats)
    ref = O.batched_solve(mats, B.X0s, O.Options(method="cg", tol=1e-8, max_iters=5000), anorms=an)
    with gsi.Batch(B, method="cg", tol=1e-8, anorm=an, max_iters=5000) as b:
        b.set_tiles(128, 4, 2)
        passes = b.solve(use_graph=True)
        assert passes >= max(r.iters for r in ref)
        for i, r in enumerate(ref):
            info = b.info(i)
            assert r.converged
            assert abs(info["iters"] - r.iters) <= 2, (i, info["iters"], r.iters)
            assert info["restarts"] == r.restarts
            # same subspace as the oracle's converged basis
            X, _ = b.basis(i, evals=False)
            s = np.linalg.svd(X.T @ r.X, compute_uv=False)
            assert np.sqrt(max(0.0, 1.0 - s.min() ** 2)) <= 1e-5, i
        _check_solution(b, B, mats, an)


def test_batched_sd_closed_form(torch_cuda):
    """SD on 2D Laplacians of several grids and block widths: iteration
    counts as the oracle's, Ritz values 4 sin^2(i pi/(2(nx+1))) +
    4 sin^2(j pi/(2(ny+1))) (largest p)."""
    from paper_2306_10379_gb300 import gsi
    dims = [(7, 9), (12, 17), (5, 11), (9, 14), (16, 21)]
    ps = [2, 8, 4, 2, 16]
    mats = [I.fd_laplacian(dm) for dm in dims]
    X0s = [I.start_block(m.n, p, I.SEED_BASE + 70 + k) for k, (m, p) in enumerate(zip(mats, ps))]
    B = I.ERBatch([m.n for m in mats], ps, mats, X0s)
    lams = [I.laplacian_eigenvalues(dm) for dm in dims]
    an = np.array([lam[0] for lam in lams])
    sm = _scipy(B)
    ref = O.batched_solve(sm, X0s, O.Options(method="sd", tol=1e-8, max_iters=20000), anorms=an)
    with gsi.Batch(B, method="sd", tol=1e-8, anorm=an, max_iters=20000) as b:
        b.solve()
        for i, (lam, p) in enumerate(zip(lams, ps)):
            info = b.info(i)
            assert ref[i].converged and info["converged"] == 1
            assert abs(info["iters"] - ref[i].iters) <= 2, (i, info["iters"], ref[i].iters)
            _, th = b.basis(i)
            gap = lam[p - 1] - lam[p]
            # quadratic Ritz bound plus the df64 Rayleigh-Ritz rounding level
            assert np.max(np.abs(th - lam[:p])) <= 2 * (1e-8 * an[i]) ** 2 / gap + 1e-12 * an[i], i


def test_graph_and_host_loop_agree(torch_cuda):
    """The while-graph and the host loop run the same passes: identical
    pass counts, iteration counts and bases (the kernels sum in a fixed
    order)."""
    from paper_2306_10379_gb300 import gsi
    B = _batch(seed=11)
    an = _anorms(_scipy(B))
    out = []
    for use_graph in (True, False):
        with gsi.Batch(B, method="cg", tol=1e-8, anorm=an) as b:
            passes = b.solve(use_graph=use_graph)
            out.append((passes, [b.info(i)["iters"] for i in range(B.nprob)],
                        [b.basis(i, evals=False)[0] for i in range(B.nprob)]))
    assert out[0][0] == out[1][0]
    assert out[0][1] == out[1][1]
    for Xa, Xb in zip(out[0][2], out[1][2]):
        assert np.array_equal(Xa, Xb)


def test_tuner_picks_a_candidate_and_solves(torch_cuda):
    from paper_2306_10379_gb300 import gsi
    B = _batch(seed=13)
    mats = _scipy(B)
    an = _anorms(mats)
    with gsi.Batch(B, method="cg", tol=1e-8, anorm=an) as b:
        best = b.tune(npasses=2)
        assert best["tile_max"] in (256, 512, 1024, 2048, 4096)
        assert best["ctas_per_sm"] in (2, 4, 8)
        assert best["tiles_per_cta"] in (1, 2)
        assert b.tiles()["tile_max"] == best["tile_max"]
        b.solve()
        _check_solution(b, B, mats, an)


def test_batched_min_problem(torch_cuda):
    """which = -1: the lowest p eigenpairs (the method on -A, Sec. 2.1)."""
    from paper_2306_10379_gb300 import gsi
    B = _batch(seed=17, sizes=(np.array([300, 150], np.int32), np.array([8, 4], np.int32)))
    mats = _scipy(B)
    an = _anorms(mats)
    with gsi.Batch(B, method="cg", which=-1, tol=1e-8, anorm=an, max_iters=20000) as b:
        b.solve()
        _check_solution(b, B, mats, an, which=-1)


def test_smallest_sizes(torch_cuda):
    """n = 2p problems and p = 2 blocks next to larger ones: 1D Laplacians
    with the closed-form spectrum 2 - 2 cos(k pi/(n+1))."""
    from paper_2306_10379_gb300 import gsi
    ns, ps = [4, 8, 64, 40], [2, 4, 32, 2]
    mats = [I.fd_laplacian((n,)) for n in ns]
    X0s = [I.start_block(n, p, I.SEED_BASE + 50 + k) for k, (n, p) in enumerate(zip(ns, ps))]
    B = I.ERBatch(ns, ps, mats, X0s)
    sm = _scipy(B)
    an = _anorms(sm)
    with gsi.Batch(B, method="cg", tol=1e-8, anorm=an) as b:
        b.solve()
        for i, (n, p) in enumerate(zip(ns, ps)):
            _, th = b.basis(i)
            exact = 2 - 2 * np.cos(np.arange(n, n - p, -1) * np.pi / (n + 1))
            assert np.max(np.abs(th - exact)) <= 1e-8 * an[i] * np.sqrt(p) + 1e-12, i


def test_noconv_status(torch_cuda):
    """max_iters reached: GSI_ERR_NOCONV from solve, status per problem."""
    from paper_2306_10379_gb300 import gsi
    B = _batch(seed=19)
    an = _anorms(_scipy(B))
    with gsi.Batch(B, method="sd", tol=1e-8, anorm=an, max_iters=3) as b:
        with pytest.raises(gsi.GsiError):
            b.solve()
        for i in range(B.nprob):
            info = b.info(i)
            assert info["status"] == gsi.GSI_ERR_NOCONV and info["iters"] == 3


def test_device_plan_matches_oracle(torch_cuda):
    """The tile table the device builds at the start of a pass is the
    oracle's plan over the problems still active (bit-exact integers), both
    with every problem active and near the end of the solve."""
    from paper_2306_10379_gb300 import gsi
    B = _batch(seed=23)
    an = _anorms(_scipy(B))
    with gsi.Batch(B, method="cg", tol=1e-8, anorm=an) as b:
        b.set_tiles(128, 2, 1)
        grid = b.tiles()["grid"]
        checked_partial = False
        for _ in range(400):
            b.step(1)
            st = [b.info(i)["status"] for i in range(B.nprob)]
            plan = b.last_plan()
            active = [int(i in {t[0] for t in plan}) for i in range(B.nprob)]
            assert plan == O.batched_plan(B.n, B.p, 128, grid, active)[1]
            if 0 < sum(active) < B.nprob:
                checked_partial = True
            if all(s != -1 for s in st):
                break
        assert checked_partial
