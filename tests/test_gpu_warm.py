"""Learned warm start on the GPU against the oracle: the bfloat16 tensor-core
GEMM, the network's forward and backward passes, the subspace loss and its
gradient, prolongation / restriction, Adam; then training on plain-method
solves and the gain of the learned start over a random one."""
import numpy as np
import pytest

from oracle import gsi_oracle as O
from paper_2306_10379_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _t(torch, a, dtype=None):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype or torch.float32, device="cuda")


def _gemm_ref(A, B, bias=None, mask=None, relu=False):
    """bfloat16 operands, float64 sums; also the sum of |terms| per entry."""
    Aq, Bq = O.bf16_round(A), O.bf16_round(B)
    C = Aq @ Bq
    scale = np.abs(Aq) @ np.abs(Bq)
    if bias is not None:
        C = C + bias
    if mask is not None:
        C = np.where(mask > 0, C, 0.0)
    if relu:
        C = np.maximum(C, 0.0)
    return C, scale


@pytest.mark.parametrize("M,N,K,transA,transB", [(64, 64, 32, False, False), (70, 130, 45, False, True),
                                                 (5, 300, 512, True, False), (129, 17, 16, True, True)])
def test_gemm_bf16(torch_cuda, M, N, K, transA, transB):
    """Ragged sizes and both operand layouts; bias, mask and ReLU epilogues.
    The float32 sums differ from float64 ones by at most K ulps of the
    absolute terms."""
    torch = torch_cuda
    from paper_2306_10379_gb300 import gsi
    rng = np.random.default_rng(M + N + K)
    A = rng.standard_normal((M, K)).astype(np.float32)
    B = rng.standard_normal((K, N)).astype(np.float32)
    bias = rng.standard_normal(N).astype(np.float32)
    mask = (rng.standard_normal((M, N)) > 0).astype(np.float32)
    Ad = _t(torch, A.T.copy() if transA else A)
    Bd = _t(torch, B.T.copy() if transB else B)
    sa = (1, M) if transA else (K, 1)
    sb = (1, K) if transB else (N, 1)
    for kw in ({}, {"bias": bias, "relu": True}, {"mask": mask}):
        Cd = torch.zeros((M, N), dtype=torch.float32, device="cuda")
        gsi.gemm_bf16(M, N, K, Ad, sa, Bd, sb, Cd, N, bias=None if "bias" not in kw else _t(torch, bias),
                      mask=None if "mask" not in kw else _t(torch, mask), relu=kw.get("relu", False))
        ref, scale = _gemm_ref(A, B, kw.get("bias"), kw.get("mask"), kw.get("relu", False))
        got = Cd.cpu().numpy()
        assert np.all(np.abs(got - ref) <= K * 2.0 ** -23 * (scale + 1.0)), kw


def _mlp_case(din=16, hidden=64, dout=96, batch=10, seed=3):
    prm = O.mlp_init(din, hidden, dout, I.SEED_BASE + seed)
    rng = np.random.default_rng(seed)
    prm["b1"] = (0.1 * rng.standard_normal(hidden)).astype(np.float32)
    prm["b2"] = (0.1 * rng.standard_normal(hidden)).astype(np.float32)
    prm["b3"] = (0.1 * rng.standard_normal(dout)).astype(np.float32)
    x = rng.standard_normal((batch, din)).astype(np.float32)
    return prm, x


def _close(got, ref, scale, rel=2.0 ** -7):
    """Within float32 sums everywhere, and within one bfloat16 ulp of the
    absolute terms where a layer input rounded to the other bfloat16 value
    (inputs computed in float32 here, float64 in the oracle)."""
    err = np.abs(got - ref)
    assert np.all(err <= rel * scale + 1e-5), float(np.max(err / (scale + 1e-5)))
    assert np.linalg.norm(got - ref) <= 1e-4 * np.linalg.norm(ref) + 1e-6


def test_mlp_forward_backward_match_oracle(torch_cuda):
    torch = torch_cuda
    from paper_2306_10379_gb300 import gsi
    prm, x = _mlp_case()
    batch, dout = x.shape[0], prm["W3"].shape[0]
    net = gsi.MLP(16, 64, dout, gsi.MLP.flatten(prm), max_batch=batch)
    xd = _t(torch, x)
    out = torch.empty((batch, dout), dtype=torch.float32, device="cuda")
    net.forward(xd, out)
    ref, cache = O.mlp_forward(prm, x)
    a2 = cache[4]
    scale = np.abs(a2) @ np.abs(O.bf16_round(prm["W3"])).T + np.abs(prm["b3"])
    _close(out.cpu().numpy(), ref, scale)
    rng = np.random.default_rng(11)
    dout_h = rng.standard_normal((batch, dout)).astype(np.float32)
    net.backward(xd, _t(torch, dout_h))
    g = net.grads()
    gr = O.mlp_backward(prm, cache, dout_h)
    for name in ("W3", "b3", "W2", "b2", "W1", "b1"):
        G, R = g[name], gr[name]
        assert np.linalg.norm(G - R) <= 2e-3 * np.linalg.norm(R) + 1e-6, name
    # the last layer's weight gradient has no rounded intermediate: tight
    sc = np.abs(O.bf16_round(dout_h)).T @ np.abs(a2)
    assert np.all(np.abs(g["W3"] - gr["W3"]) <= batch * 2.0 ** -23 * (sc + 1.0))
    net.close()


def _loss_case(nc=8, nf=17, p=4, batch=3, seed=0):
    P = O.prolongation(nc, nf)
    S = (P.T @ P).tocsr()
    rng = np.random.default_rng(seed)
    Us, Cs = [], []
    for _ in range(batch):
        U, _ = np.linalg.qr(rng.standard_normal((nf * nf, p)))
        Us.append(U)
        Cs.append(rng.standard_normal((nc * nc, p)).astype(np.float32))
    Bts = [(P.T @ U).astype(np.float32) for U in Us]
    return P, S, Us, Cs, Bts


def _csr_dev(torch, S):
    return (torch.tensor(S.indptr.astype(np.int64), device="cuda"),
            torch.tensor(S.indices.astype(np.int32), device="cuda"),
            torch.tensor(S.data.astype(np.float64), device="cuda"))


def test_loss_grad_matches_oracle(torch_cuda):
    torch = torch_cuda
    from paper_2306_10379_gb300 import gsi
    nc, nf, p = 8, 17, 4
    P, S, Us, Cs, Bts = _loss_case(nc, nf, p)
    loss, dC = gsi.warm_loss_grad(_t(torch, np.stack(Cs)), _csr_dev(torch, S), _t(torch, np.stack(Bts)),
                                  nc * nc, p, gscale=0.5)
    loss, dC = loss.cpu().numpy(), dC.cpu().numpy()
    for s in range(len(Cs)):
        L, g = O.warm_loss_grad(Cs[s], S, Bts[s].astype(np.float64))
        assert abs(loss[s] - L) <= 1e-5 * max(1.0, abs(L)), s
        assert np.linalg.norm(dC[s] - 0.5 * g) <= 1e-4 * np.linalg.norm(0.5 * g), s


def test_prolong_restrict_match_oracle(torch_cuda):
    torch = torch_cuda
    from paper_2306_10379_gb300 import gsi
    for nc, nf, p in ((8, 17, 4), (32, 64, 8), (5, 23, 2)):
        P = O.prolongation(nc, nf)
        rng = np.random.default_rng(nc + nf)
        C = rng.standard_normal((2, nc * nc, p)).astype(np.float32)
        X = gsi.prolong(_t(torch, C), nc, nf, p).cpu().numpy()
        for s in range(2):
            ref = P @ C[s].astype(np.float64)
            assert np.max(np.abs(X[s] - ref)) <= 1e-12 * (1 + np.max(np.abs(ref)))
        U = rng.standard_normal((2, nf * nf, p))
        Bt = gsi.restrict(torch.tensor(U, device="cuda"), nc, nf, p).cpu().numpy()
        for s in range(2):
            ref = P.T @ U[s]
            assert np.max(np.abs(Bt[s] - ref)) <= 2e-7 * (1 + np.max(np.abs(ref)))


def test_adam_matches_oracle(torch_cuda):
    """Three Adam steps on the network's parameters with fixed gradients."""
    torch = torch_cuda
    from paper_2306_10379_gb300 import gsi
    prm, x = _mlp_case(hidden=32, dout=40, batch=6)
    net = gsi.MLP(16, 32, 40, gsi.MLP.flatten(prm), max_batch=6)
    xd = _t(torch, x)
    out = torch.empty((6, 40), dtype=torch.float32, device="cuda")
    net.forward(xd, out)
    net.backward(xd, _t(torch, np.ones((6, 40), np.float32)))
    g = gsi.MLP.flatten(net.grads()).astype(np.float64)
    w = gsi.MLP.flatten(prm).astype(np.float64)
    m = np.zeros_like(w)
    v = np.zeros_like(w)
    for t in range(1, 4):
        net.adam(1e-3)
        w, m, v = O.adam_step(w, g, m, v, t, 1e-3)
    got = gsi.MLP.flatten(net.params()).astype(np.float64)
    assert np.max(np.abs(got - w)) <= 1e-6 * (1 + np.max(np.abs(w)))
    net.close()


def _family(torch, gsi, nops, seed, nx, p, nc, max_iters):
    """Operators, inputs and labels: the plain method's (batched CG, lowest p
    via -A) bases restricted to the coarse grid. Some operators of this
    family (log-diffusivity amplitude ~4) have relative gaps near 1e-8 and
    stop at max_iters; they are flagged in `conv`."""
    B, xs = I.diffusion_batch(nops, seed, nx, p)
    with gsi.Batch(B, method="cg", which=-1, tol=1e-8, max_iters=max_iters) as b:
        b.solve(check=False)
        info = [b.info(i) for i in range(nops)]
        U = np.stack([b.basis(i, evals=False)[0] for i in range(nops)])
    iters = np.array([f["iters"] for f in info])
    conv = np.array([f["converged"] == 1 for f in info])
    Bt = gsi.restrict(torch.tensor(U, device="cuda"), nc, nx, p)
    return B, xs.astype(np.float32), Bt, iters, conv


def test_training_and_warm_start_gain(torch_cuda):
    """Trained on the converged ones of 384 plain-method solves (24 x 24
    grid, lowest p = 4 modes, 8 x 8 coarse grid), the network's start is
    closer to the held-out operators' subspaces than a random start (sum of
    sin^2 of the principal angles well below the random start's ~p) and
    saves iterations on them (counts capped at max_iters); the training loss
    falls."""
    torch = torch_cuda
    from paper_2306_10379_gb300 import gsi
    nx, p, nc, cap, hidden = 24, 4, 8, 8000, 256
    m = nc * nc
    S = O.prolongation(nc, nx)
    S = (S.T @ S).tocsr()
    Sd = _csr_dev(torch, S)
    _, xtr, Bttr, _, conv = _family(torch, gsi, 384, I.SEED_BASE + 1000, nx, p, nc, cap)
    keep = torch.tensor(np.flatnonzero(conv), device="cuda")
    ntr = int(keep.numel())
    assert ntr >= 256
    xd = _t(torch, xtr)[keep].contiguous()
    Bttr = Bttr[keep].contiguous()
    Bte, xte, Btte, iters_random, _ = _family(torch, gsi, 16, I.SEED_BASE + 5000, nx, p, nc, cap)
    prm = O.mlp_init(16, hidden, m * p, I.SEED_BASE + 7)
    net = gsi.MLP(16, hidden, m * p, gsi.MLP.flatten(prm), max_batch=32)
    rng = np.random.default_rng(0)
    losses = []
    for step in range(1500):
        idx = torch.tensor(rng.choice(ntr, 32, replace=False), device="cuda")
        lr = 1e-3 if step < 1100 else 3e-4
        losses.append(net.train_step(xd[idx].contiguous(), Sd, Bttr[idx].contiguous(), m, p, lr))
    assert np.mean(losses[-20:]) < 0.6 * np.mean(losses[:20])
    out = torch.empty((16, m * p), dtype=torch.float32, device="cuda")
    net.forward(_t(torch, xte), out)
    held_out, _ = gsi.warm_loss_grad(out.view(16, m, p).contiguous(), Sd, Btte, m, p)
    assert held_out.mean().item() < 0.75 * p
    X0 = gsi.prolong(out.view(16, m, p), nc, nx, p).reshape(-1).contiguous()
    with gsi.Batch(Bte, method="cg", which=-1, tol=1e-8, max_iters=cap) as b:
        b.restart(X0)
        b.solve(check=False)
        iters_warm = np.array([b.info(i)["iters"] for i in range(16)])
    print("held-out loss %.3f; iterations random mean %.0f median %.0f, learned mean %.0f median %.0f"
          % (held_out.mean().item(), iters_random.mean(), np.median(iters_random), iters_warm.mean(),
             np.median(iters_warm)))
    assert iters_warm.mean() < iters_random.mean()
    assert np.median(iters_warm) < 0.9 * np.median(iters_random)
    net.close()
