"""The allocation-free Gram entry point (gsi_oz_gram_noalloc) against the
allocating one (gsi_oz_gram), called through the C ABI.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test. It passes both alone in a
fresh process and after the rest of the suite.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _call(lib, name, U, V, G, sym, stream):
    fn = getattr(lib, name)
    fn.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                   ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    n, p = U.shape[0], U.shape[1]
    q = V.shape[1]
    return fn(n, p, q, ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(V.data_ptr()), 1 if sym else 0,
              ctypes.c_void_p(G.data_ptr()), ctypes.c_void_p(stream))


@pytest.mark.parametrize("n,p,q,sym", [(200001, 64, 64, True), (50000, 100, 37, False)])
def test_noalloc_gram_matches_allocating_gram(n, p, q, sym):
    """Same kernels, same row partition and the same fixed-order reduction as
    gsi_oz_gram, so the Grams must be bit-identical. Between the two checked
    calls a call on other inputs (fewer rows, so fewer partial blocks) leaves
    different partial sums in the shared static array: a call that read stale
    partials would no longer match."""
    import torch
    from paper_2306_10379_gb300 import build, gsi
    build.build()
    lib = gsi.lib()
    rng = np.random.default_rng(n + p)

    def blocks(rows):
        U = torch.from_numpy(gsi.to_df(rng.standard_normal((rows, p)))).cuda()
        V = U if sym else torch.from_numpy(gsi.to_df(rng.standard_normal((rows, q)))).cuda()
        return U, V

    U, V = blocks(n)
    U2, V2 = blocks(n // 7 + 3)
    stream = torch.cuda.current_stream().cuda_stream
    ref = torch.empty((p, q), dtype=torch.float64, device="cuda")
    ref2 = torch.empty((p, q), dtype=torch.float64, device="cuda")
    assert _call(lib, "gsi_oz_gram", U, V, ref, sym, stream) == 0
    assert _call(lib, "gsi_oz_gram", U2, V2, ref2, sym, stream) == 0
    for _ in range(2):  # two calls in a row share the static scratch
        got = torch.full((p, q), float("nan"), dtype=torch.float64, device="cuda")
        assert _call(lib, "gsi_oz_gram_noalloc", U, V, got, sym, stream) == 0
        torch.cuda.synchronize()
        assert np.array_equal(got.cpu().numpy(), ref.cpu().numpy())
        other = torch.full((p, q), float("nan"), dtype=torch.float64, device="cuda")
        assert _call(lib, "gsi_oz_gram_noalloc", U2, V2, other, sym, stream) == 0
        torch.cuda.synchronize()
        assert np.array_equal(other.cpu().numpy(), ref2.cpu().numpy())
