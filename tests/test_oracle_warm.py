"""Pins of the warm-start oracle against facts that do not depend on it:
interpolation exactness, the bfloat16 format, finite differences, principal
angles from an SVD, and Adam's first step."""
import numpy as np
import scipy.linalg as sla

from oracle import gsi_oracle as O


def test_prolongation_1d_reproduces_linear_functions():
    """Hat interpolation is exact on functions linear between two coarse
    nodes, and linear on [0, x_c(0)] from the zero boundary value."""
    nc, nf = 8, 37
    P1 = O.prolongation_1d(nc, nf)
    xc = (np.arange(nc) + 1.0) / (nc + 1)
    xf = (np.arange(nf) + 1.0) / (nf + 1)
    g = 0.3 + 2.0 * xc
    f = P1 @ g
    inner = (xf >= xc[0]) & (xf <= xc[-1])
    assert np.allclose(f[inner], 0.3 + 2.0 * xf[inner], atol=1e-14)
    left = xf < xc[0]
    assert np.allclose(f[left], g[0] * xf[left] / xc[0], atol=1e-14)
    assert np.allclose(P1[inner].sum(1), 1.0, atol=1e-14)
    # coincident nodes (nf + 1 a multiple of nc + 1) copy the coarse value
    P = O.prolongation_1d(4, 9)
    assert np.allclose(P[1::2], np.eye(4), atol=1e-15)


def test_prolongation_2d_is_separable_in_operator_order():
    """P (f(x) g(y)) on the coarse grid equals the product of the 1D
    interpolants, row i + nf j <-> (x_i, y_j)."""
    nc, nf = 5, 11
    P = O.prolongation(nc, nf)
    P1 = O.prolongation_1d(nc, nf)
    fx = np.arange(nc) ** 2 + 1.0
    gy = np.cos(np.arange(nc))
    coarse = (gy[:, None] * fx[None, :]).ravel()  # index a + nc b
    fine = (P @ coarse).reshape(nf, nf)           # [j, i]
    assert np.allclose(fine, np.outer(P1 @ gy, P1 @ fx), atol=1e-13)


def test_bf16_round():
    """bfloat16 keeps 8 significant bits; ties go to the even neighbour."""
    x = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, 1 + 2 ** -7, 1 + 1.5 * 2 ** -8, -2.5e-3, 3.0e38])
    r = O.bf16_round(x)
    assert r[0] == 1.0
    assert r[1] == 1.0                    # tie -> even (1.0)
    assert r[2] == 1 + 2 ** -6            # tie -> even (mantissa ...10)
    assert r[3] == 1 + 2 ** -7            # representable
    assert r[4] == 1 + 2 ** -7            # above the tie -> up
    assert abs(r[5] / -2.5e-3 - 1) < 2 ** -8
    assert np.isfinite(r[6])


def _tiny_mlp(seed=3):
    prm = O.mlp_init(5, 12, 7, seed)
    prm["b1"] = (np.arange(12) * 0.01 - 0.05).astype(np.float32)
    prm["b2"] = (np.arange(12) * -0.02 + 0.1).astype(np.float32)
    prm["b3"] = (np.arange(7) * 0.03).astype(np.float32)
    return prm


def test_mlp_backward_matches_finite_differences():
    prm = {k: v.astype(np.float64) for k, v in _tiny_mlp().items()}
    rng = np.random.default_rng(0)
    x = rng.standard_normal((4, 5))
    dout = rng.standard_normal((4, 7))
    out, cache = O.mlp_forward(prm, x, bf16=False)
    g = O.mlp_backward(prm, cache, dout, bf16=False)

    def f(p):
        return float(np.sum(O.mlp_forward(p, x, bf16=False)[0] * dout))

    h = 1e-6
    for name in ("W1", "b1", "W2", "b2", "W3", "b3"):
        flat = prm[name].ravel()
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            pp = {k: v.copy() for k, v in prm.items()}
            pm = {k: v.copy() for k, v in prm.items()}
            pp[name].ravel()[idx] += h
            pm[name].ravel()[idx] -= h
            fd = (f(pp) - f(pm)) / (2 * h)
            assert abs(fd - g[name].ravel()[idx]) <= 1e-6 * max(1.0, abs(fd)), (name, idx)


def _warm_case(m=40, p=3, n_fine=None, seed=1):
    nc = int(round(np.sqrt(m)))
    P = O.prolongation(nc, 2 * nc + 1).toarray()
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((P.shape[0], p)))
    C = rng.standard_normal((P.shape[1], p))
    return P, U, C


def test_warm_loss_is_sum_of_sin2_principal_angles():
    P, U, C = _warm_case(m=36, p=4)
    L, _ = O.warm_loss_grad(C, P.T @ P, P.T @ U)
    th = sla.subspace_angles(P @ C, U)
    assert abs(L - np.sum(np.sin(th) ** 2)) <= 1e-12
    assert 0.0 <= L <= 4.0


def test_warm_loss_zero_on_target_and_basis_invariant():
    P, _, C = _warm_case(m=25, p=3, seed=4)
    U, _ = np.linalg.qr(P @ C)
    S, Bt = P.T @ P, P.T @ U
    L, dC = O.warm_loss_grad(C, S, Bt)
    assert abs(L) <= 1e-12 and np.max(np.abs(dC)) <= 1e-10
    rng = np.random.default_rng(7)
    U2, _ = np.linalg.qr(rng.standard_normal((P.shape[0], 3)))
    G = rng.standard_normal((3, 3)) + 3 * np.eye(3)
    L1, g1 = O.warm_loss_grad(C, S, P.T @ U2)
    L2, g2 = O.warm_loss_grad(C @ G, S, P.T @ U2)
    assert abs(L1 - L2) <= 1e-12
    # chain rule of L(C G): dL/dC = (dL/d(CG)) G^T
    assert np.allclose(g2 @ G.T, g1, atol=1e-10)


def test_warm_loss_gradient_matches_finite_differences():
    P, U, C = _warm_case(m=49, p=4, seed=2)
    S, Bt = P.T @ P, P.T @ U
    L, dC = O.warm_loss_grad(C, S, Bt)
    rng = np.random.default_rng(5)
    h = 1e-6
    for _ in range(12):
        i, j = rng.integers(C.shape[0]), rng.integers(C.shape[1])
        Cp, Cm = C.copy(), C.copy()
        Cp[i, j] += h
        Cm[i, j] -= h
        fd = (O.warm_loss_grad(Cp, S, Bt)[0] - O.warm_loss_grad(Cm, S, Bt)[0]) / (2 * h)
        assert abs(fd - dC[i, j]) <= 1e-7 * max(1.0, abs(fd)), (i, j)


def test_adam_first_step_is_signed_lr():
    """At t = 1 the bias corrections make the step lr g / (|g| + eps)."""
    w = np.array([1.0, -2.0, 0.5])
    g = np.array([3.0, -0.25, 1e-3])
    w1, m, v = O.adam_step(w, g, np.zeros(3), np.zeros(3), 1, 0.01)
    assert np.allclose(w1, w - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)
