"""Seeded synthetic inputs shared by the CUDA path and the CPU oracle.

This module holds no arithmetic of the eigen-solver itself: it only builds
the operator A (as CSR arrays, or dense) and the random start block X0 from a
seed, so that both sides of every parity test see bit-identical inputs.

Random numbers come from Philox-4x32-10 (Salmon, Moraes, Dror & Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11), written here from its
published round function, followed by 53-bit uniform doubles and the
Box-Muller transform evaluated with numpy's libm.

Operators (the paper's workloads, Sec. 6, and their synthetic stand-ins):
  * fd_laplacian   -- 1D/2D/3D finite-difference Dirichlet Laplacian, unscaled
                      (2*d on the diagonal, -1 for each grid neighbour), the
                      FD matrices of Sec. 6.2 and Sec. 6.3 ("FD3D").
  * er_laplacian   -- Erdos-Renyi G(n, 4n) graph Laplacian + diagonal shift,
                      a synthetic stand-in for the power-grid graph matrix of
                      Sec. 6.3, which is not available here.
  * diffusion_fd   -- 5-point -div(kappa grad u) with a smooth random kappa.
  * dense_spectrum -- dense Q diag(lambda) Q^T with a prescribed gap.
"""
from __future__ import annotations

import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)

# Seed convention for the workloads: base + workload index + problem index.
SEED_BASE = 2306103790


def philox4x32_10(ctr: np.ndarray, key: tuple[int, int]) -> np.ndarray:
    """Philox-4x32 with 10 rounds.

    ctr: uint32 array of shape (m, 4); key: two 32-bit words.
    Returns a uint32 array of shape (m, 4).
    """
    c = np.asarray(ctr, dtype=np.uint64) & _MASK
    c0, c1, c2, c3 = c[:, 0].copy(), c[:, 1].copy(), c[:, 2].copy(), c[:, 3].copy()
    k0 = np.uint64(key[0] & 0xFFFFFFFF)
    k1 = np.uint64(key[1] & 0xFFFFFFFF)
    for r in range(10):
        if r:
            k0 = (k0 + _W0) & _MASK
            k1 = (k1 + _W1) & _MASK
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0), lo1, (hi0 ^ c3 ^ k1), lo0
    return np.stack([c0, c1, c2, c3], axis=1).astype(np.uint32)


def _key(seed: int) -> tuple[int, int]:
    return (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)


def uniform_words(count: int, seed: int, stream: int = 0) -> np.ndarray:
    """`count` uint32 words (rounded up to a multiple of 4) from one Philox stream."""
    m = (count + 3) // 4
    ctr = np.zeros((m, 4), dtype=np.uint64)
    ctr[:, 0] = np.arange(m, dtype=np.uint64) & _MASK
    ctr[:, 1] = np.arange(m, dtype=np.uint64) >> np.uint64(32)
    ctr[:, 2] = np.uint64(stream & 0xFFFFFFFF)
    return philox4x32_10(ctr, _key(seed)).reshape(-1)[:count]


def uniform53(count: int, seed: int, stream: int = 0) -> np.ndarray:
    """Doubles in [0, 1) with 53 random bits, two Philox words each."""
    w = uniform_words(2 * count, seed, stream).astype(np.uint64)
    a = w[0::2] >> np.uint64(5)   # 27 bits
    b = w[1::2] >> np.uint64(6)   # 26 bits
    return (a.astype(np.float64) * 67108864.0 + b.astype(np.float64)) / 9007199254740992.0


def gaussian(count: int, seed: int, stream: int = 0) -> np.ndarray:
    """N(0,1) samples by Box-Muller on pairs of 53-bit uniforms."""
    m = (count + 1) // 2
    u = uniform53(2 * m, seed, stream)
    u1 = 1.0 - u[0::2]            # (0, 1], safe for log
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m)
    z[0::2] = r * np.cos(2.0 * np.pi * u2)
    z[1::2] = r * np.sin(2.0 * np.pi * u2)
    return z[:count]


def start_block(n: int, p: int, seed: int) -> np.ndarray:
    """n x p i.i.d. N(0,1) start block, row-major float64 (not orthonormal)."""
    return gaussian(n * p, seed, stream=1).reshape(n, p)


class CSR:
    """Plain CSR container: rowptr int64 (n+1), colidx int32 (nnz), val float64."""

    def __init__(self, n: int, rowptr: np.ndarray, colidx: np.ndarray, val: np.ndarray):
        self.n = int(n)
        self.rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
        self.colidx = np.ascontiguousarray(colidx, dtype=np.int32)
        self.val = np.ascontiguousarray(val, dtype=np.float64)

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def negated(self) -> "CSR":
        return CSR(self.n, self.rowptr, self.colidx, -self.val)


def fd_laplacian(dims) -> CSR:
    """Unscaled FD Dirichlet Laplacian on a grid of shape `dims` (1 to 3 axes).

    Grid point (i0, i1, i2) has index i0 + d0*(i1 + d1*i2). Each row holds the
    diagonal 2*len(dims) and -1 for every in-grid neighbour; column indices
    are ascending within a row.
    """
    dims = tuple(int(d) for d in dims)
    nd = len(dims)
    n = int(np.prod(dims))
    strides = [1]
    for d in dims[:-1]:
        strides.append(strides[-1] * d)
    coords = np.indices(dims[::-1]).reshape(nd, -1)[::-1]  # coords[a] = index along axis a
    idx = np.arange(n, dtype=np.int64)
    # candidate neighbours in ascending column order: -s_{nd-1} .. -s_0, 0, +s_0 .. +s_{nd-1}
    offs, axes = [], []
    for a in reversed(range(nd)):
        offs.append(-strides[a]); axes.append((a, -1))
    offs.append(0); axes.append(None)
    for a in range(nd):
        offs.append(strides[a]); axes.append((a, +1))
    cols, vals, valid = [], [], []
    for off, ax in zip(offs, axes):
        if ax is None:
            ok = np.ones(n, dtype=bool)
            v = np.full(n, 2.0 * nd)
        else:
            a, s = ax
            ok = (coords[a] > 0) if s < 0 else (coords[a] < dims[a] - 1)
            v = np.full(n, -1.0)
        cols.append(idx + off); vals.append(v); valid.append(ok)
    cols = np.stack(cols, axis=1)
    vals = np.stack(vals, axis=1)
    valid = np.stack(valid, axis=1)
    counts = valid.sum(axis=1)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return CSR(n, rowptr, cols[valid].astype(np.int32), vals[valid])


class ZCSR:
    """CSR container of a complex matrix: rowptr int64 (n+1), colidx int32,
    val complex128."""

    def __init__(self, n: int, rowptr: np.ndarray, colidx: np.ndarray, val: np.ndarray):
        self.n = int(n)
        self.rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
        self.colidx = np.ascontiguousarray(colidx, dtype=np.int32)
        self.val = np.ascontiguousarray(val, dtype=np.complex128)

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])


def twisted_torus_laplacian(dims, thetas) -> ZCSR:
    """Complex Hermitian test operator: the periodic FD Laplacian on a grid of
    shape dims (each d >= 3) whose wrap-around edge along axis a carries the
    phase exp(i theta_a) (a discrete magnetic Laplacian with flux theta_a
    through each cycle). Node (i0, i1, ...) is row i0 + d0 (i1 + d1 ...).
    Row r holds 2 len(dims) on the diagonal and -1 for each neighbour, the
    neighbour across the wrap edge -exp(+i theta) forwards and -exp(-i theta)
    backwards; column indices ascending."""
    dims = tuple(int(d) for d in dims)
    n = int(np.prod(dims))
    strides = [1]
    for d in dims[:-1]:
        strides.append(strides[-1] * d)
    rows = [dict() for _ in range(n)]
    for r in range(n):
        rows[r][r] = complex(2 * len(dims))
        rem = r
        for a, d in enumerate(dims):
            ia = (rem // strides[a]) % d
            fwd = r + strides[a] if ia + 1 < d else r - (d - 1) * strides[a]
            bwd = r - strides[a] if ia > 0 else r + (d - 1) * strides[a]
            ph_f = np.exp(1j * thetas[a]) if ia + 1 == d else 1.0
            ph_b = np.exp(-1j * thetas[a]) if ia == 0 else 1.0
            rows[r][fwd] = rows[r].get(fwd, 0.0) - ph_f
            rows[r][bwd] = rows[r].get(bwd, 0.0) - ph_b
    rowptr = np.zeros(n + 1, np.int64)
    cols, vals = [], []
    for r in range(n):
        ks = sorted(rows[r])
        cols += ks
        vals += [rows[r][k] for k in ks]
        rowptr[r + 1] = len(cols)
    return ZCSR(n, rowptr, np.array(cols), np.array(vals))


def twisted_torus_eigenvalues(dims, thetas) -> np.ndarray:
    """Closed-form spectrum of twisted_torus_laplacian, descending: sums over
    the axes of 2 - 2 cos((2 pi k + theta_a) / d_a), k = 0..d_a - 1."""
    total = np.zeros(1)
    for d, th in zip(dims, thetas):
        k = np.arange(d)
        s = 2.0 - 2.0 * np.cos((2.0 * np.pi * k + th) / d)
        total = (total[:, None] + s[None, :]).ravel()
    return np.sort(total)[::-1]


def complex_start_block(n: int, p: int, seed: int) -> np.ndarray:
    """n x p complex start block: real and imaginary parts i.i.d. N(0,1)
    (start_block for the real part, stream 7 for the imaginary part)."""
    return start_block(n, p, seed) + 1j * gaussian(n * p, seed, stream=7).reshape(n, p)


def drifting_laplacians(dims, count: int, eps: float) -> list:
    """A slowly varying sequence for subspace tracking: A_k = L + eps k diag(v),
    k = 0..count-1, L = fd_laplacian(dims) and v the smooth potential
    v(x) = prod over axes of sin(pi x_a) cos(pi x_a) at the nodes
    x_a = (i_a + 1)/(d_a + 1). Same sparsity for every k (L's diagonal)."""
    L = fd_laplacian(dims)
    # node index i0 + d0 i1 (+ d0 d1 i2): the first axis varies fastest
    v = np.ones(1)
    for d in dims:
        x = (np.arange(d) + 1.0) / (d + 1.0)
        v = np.kron(np.sin(np.pi * x) * np.cos(np.pi * x), v)
    rows = np.repeat(np.arange(L.n), np.diff(L.rowptr))
    diag = np.flatnonzero(L.colidx == rows)
    out = []
    for k in range(count):
        val = L.val.copy()
        val[diag] += eps * k * v[rows[diag]]
        out.append(CSR(L.n, L.rowptr.copy(), L.colidx.copy(), val))
    return out


def er_laplacian(n: int, seed: int, mean_degree: int = 8) -> CSR:
    """Graph Laplacian D - W of an Erdos-Renyi G(n, M) graph, M = n*mean_degree/2
    distinct undirected unit-weight edges drawn in Philox order (self-loops and
    repeats rejected), plus a diagonal shift U(0,1); each diagonal entry
    degree + shift is rounded to float32, so that every entry is exactly
    representable in float32."""
    m_target = n * mean_degree // 2
    keys = np.empty(0, dtype=np.int64)
    chunk = int(m_target * 1.25) + 64
    stream = 2
    while keys.size < m_target:
        w = uniform_words(2 * chunk, seed, stream).astype(np.int64)
        u = w[0::2] % n
        v = w[1::2] % n
        ok = u != v
        lo = np.minimum(u, v)[ok]
        hi = np.maximum(u, v)[ok]
        keys = np.concatenate([keys, lo * n + hi])
        _, first = np.unique(keys, return_index=True)
        keys = keys[np.sort(first)]
        stream += 1
    keys = keys[:m_target]
    lo, hi = keys // n, keys % n
    shift = uniform53(n, seed, stream=1)
    rows = np.concatenate([lo, hi, np.arange(n)])
    cols = np.concatenate([hi, lo, np.arange(n)])
    deg = np.bincount(lo, minlength=n) + np.bincount(hi, minlength=n)
    diag = (deg + shift).astype(np.float32).astype(np.float64)
    vals = np.concatenate([-np.ones(2 * m_target), diag])
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=rowptr[1:])
    return CSR(n, rowptr, cols.astype(np.int32), vals)


def diffusion_coefficients(seed: int) -> np.ndarray:
    """16 N(0,1) coefficients xi_ab (a, b = 0..3) of the log-diffusivity field."""
    return gaussian(16, seed, stream=3).reshape(4, 4)


def diffusion_fd(nx: int, xi: np.ndarray, corr_len: float = 0.1, f32: bool = False) -> CSR:
    """5-point FD of -div(kappa grad u) on the unit square, nx*nx interior points,
    Dirichlet boundary, h = 1/(nx+1), unscaled by h^2. With f32, the face
    coefficients are rounded to float32 first, so that every entry (the
    diagonal summed in float32) is exactly a float32 and A stays symmetric.

    log kappa(x, y) = sum_ab xi_ab w_ab cos(pi a x) cos(pi b y),
    w_ab = exp(-pi^2 l^2 (a^2 + b^2) / 4). Face coefficients are harmonic means
    of the two adjacent nodal values (boundary nodes included)."""
    h = 1.0 / (nx + 1)
    g = np.arange(nx + 2) * h
    a = np.arange(4)
    w = np.exp(-np.pi ** 2 * corr_len ** 2 * (a[:, None] ** 2 + a[None, :] ** 2) / 4.0)
    cx = np.cos(np.pi * a[:, None] * g[None, :])      # (4, nx+2)
    logk = np.einsum("ab,ai,bj->ij", xi * w, cx, cx)  # node (i, j) -> x index i, y index j
    k = np.exp(logk)
    kx = 2.0 * k[:-1, :] * k[1:, :] / (k[:-1, :] + k[1:, :])  # faces between i and i+1
    ky = 2.0 * k[:, :-1] * k[:, 1:] / (k[:, :-1] + k[:, 1:])
    n = nx * nx
    I, J = np.meshgrid(np.arange(1, nx + 1), np.arange(1, nx + 1), indexing="ij")
    I, J = I.T.ravel(), J.T.ravel()                   # row r = (i-1) + nx*(j-1)
    if f32:
        kx = kx.astype(np.float32).astype(np.float64)
        ky = ky.astype(np.float32).astype(np.float64)
    west, east = kx[I - 1, J], kx[I, J]
    south, north = ky[I, J - 1], ky[I, J]
    diag = west + east + south + north
    if f32:
        diag = (((west.astype(np.float32) + east.astype(np.float32)) + south.astype(np.float32))
                + north.astype(np.float32)).astype(np.float64)
    r = np.arange(n)
    entries = [(r - nx, -south, J > 1), (r - 1, -west, I > 1), (r, diag, np.ones(n, bool)),
               (r + 1, -east, I < nx), (r + nx, -north, J < nx)]
    cols = np.stack([e[0] for e in entries], 1)
    vals = np.stack([e[1] for e in entries], 1)
    ok = np.stack([e[2] for e in entries], 1)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(ok.sum(1), out=rowptr[1:])
    return CSR(n, rowptr, cols[ok].astype(np.int32), vals[ok])


def dense_spectrum(n: int, p: int, gap: float, seed: int, reflectors: int = 8):
    """Dense symmetric A = Q diag(lam) Q^T, Q a product of Householder reflectors
    built from N(0,1) vectors. lam_i = 1 - i/n for i > p; the top p values sit
    `gap` above lam_{p+1}: lam_i = lam_{p+1} + gap + (p - i)/n (1-based i).
    Returns (A, lam) with lam sorted descending."""
    i = np.arange(1, n + 1, dtype=np.float64)
    lam = 1.0 - i / n
    lam_p1 = 1.0 - (p + 1) / n
    lam[:p] = lam_p1 + gap + (p - i[:p]) / n
    A = np.diag(lam)
    V = gaussian(reflectors * n, seed, stream=4).reshape(reflectors, n)
    for v in V:
        v = v / np.linalg.norm(v)
        # A <- H A H with H = I - 2 v v^T
        Av = A @ v
        A = A - 2.0 * np.outer(v, Av) - 2.0 * np.outer(Av, v) + 4.0 * (v @ Av) * np.outer(v, v)
    A = 0.5 * (A + A.T)
    return A, lam


def laplacian_eigenvalues(dims) -> np.ndarray:
    """Closed-form spectrum of fd_laplacian(dims), descending:
    sum over axes of 4 sin^2(k pi / (2 (d + 1))), k = 1..d."""
    total = np.zeros(1)
    for d in dims:
        k = np.arange(1, d + 1)
        s = 4.0 * np.sin(k * np.pi / (2.0 * (d + 1))) ** 2
        total = (total[:, None] + s[None, :]).ravel()
    return np.sort(total)[::-1]


class ERBatch:
    """A batch of Erdos-Renyi graph Laplacians with their start blocks.

    mats[i] is problem i's CSR (float64 values, each exactly a float32);
    rowptr/colidx/val is the concatenated CSR of the batched solver (rowptr
    global, column indices local to the problem, values float32); X0 the
    concatenated row-major start blocks."""

    def __init__(self, n, p, mats, X0s):
        self.n = np.asarray(n, dtype=np.int32)
        self.p = np.asarray(p, dtype=np.int32)
        self.mats = mats
        self.X0s = X0s
        nnz = np.array([m.rowptr[-1] for m in mats], dtype=np.int64)
        base = np.concatenate([[0], np.cumsum(nnz)[:-1]])
        self.rowptr = np.concatenate([[0]] + [m.rowptr[1:] + b for m, b in zip(mats, base)]).astype(np.int64)
        self.colidx = np.concatenate([m.colidx for m in mats]).astype(np.int32)
        self.val = np.concatenate([m.val for m in mats]).astype(np.float32)
        self.X0 = np.concatenate([x.ravel() for x in X0s]).astype(np.float64)

    @property
    def nprob(self) -> int:
        return int(self.n.size)


def batched_sizes(nprob: int, seed: int, n_lo: int = 2048, n_hi: int = 65536,
                  p_choices=(4, 8, 16, 32)):
    """n_i uniform on the integers [n_lo, n_hi] and p_i uniform over p_choices
    (Philox stream 4 of `seed`)."""
    u = uniform53(2 * nprob, seed, stream=4)
    n = n_lo + np.floor(u[0::2] * (n_hi - n_lo + 1)).astype(np.int64)
    p = np.asarray(p_choices, dtype=np.int64)[np.floor(u[1::2] * len(p_choices)).astype(np.int64)]
    return n.astype(np.int32), p.astype(np.int32)


def er_batch(nprob: int, seed: int, n_lo: int = 2048, n_hi: int = 65536,
             p_choices=(4, 8, 16, 32), sizes=None) -> ERBatch:
    """Problem i: er_laplacian(n_i, seed + 1 + i) (mean degree 8, diagonal
    shift U(0,1) rounded to float32) and start block
    start_block(n_i, p_i, seed + 1_000_003 + i). `sizes` = (n, p) overrides
    the drawn sizes."""
    n, p = sizes if sizes is not None else batched_sizes(nprob, seed, n_lo, n_hi, p_choices)
    mats = [er_laplacian(int(n[i]), seed + 1 + i) for i in range(len(n))]
    X0s = [start_block(int(n[i]), int(p[i]), seed + 1_000_003 + i) for i in range(len(n))]
    return ERBatch(n, p, mats, X0s)


def diffusion_batch(nops: int, seed: int, nx: int, p: int) -> tuple:
    """Operators i = 0..nops-1 of the diffusion family on an nx x nx grid:
    coefficients diffusion_coefficients(seed + i) (the 16 network inputs),
    float32-exact 5-point operators, start blocks
    start_block(nx^2, p, seed + 2_000_003 + i). Returns (ERBatch, params
    (nops x 16))."""
    xis = [diffusion_coefficients(seed + i) for i in range(nops)]
    mats = [diffusion_fd(nx, xi, f32=True) for xi in xis]
    X0s = [start_block(nx * nx, p, seed + 2_000_003 + i) for i in range(nops)]
    return ERBatch([nx * nx] * nops, [p] * nops, mats, X0s), np.stack([x.ravel() for x in xis])


def mlp_init(din: int, hidden: int, dout: int, seed: int) -> dict:
    """Seeded initial weights of the warm-start network: W ~ N(0, 2/fan_in)
    for the two hidden layers, N(0, 1/fan_in) for the output layer (Philox
    normals, streams 20..22), zero biases; float32 arrays W1 (hidden x din),
    b1, W2 (hidden x hidden), b2, W3 (dout x hidden), b3."""
    sizes = [("W1", hidden, din, 2.0), ("W2", hidden, hidden, 2.0), ("W3", dout, hidden, 1.0)]
    prm = {}
    for k, (name, r, c, g) in enumerate(sizes):
        prm[name] = (gaussian(r * c, seed, stream=20 + k).reshape(r, c) * np.sqrt(g / c)).astype(np.float32)
    prm["b1"] = np.zeros(hidden, np.float32)
    prm["b2"] = np.zeros(hidden, np.float32)
    prm["b3"] = np.zeros(dout, np.float32)
    return prm
