"""The C-ABI library builds, loads and exports every entry point that
include/gsi.h declares (no compute call: runs without a GPU)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    hdrs = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
            if f.endswith(".h")]
    names = set()
    for h in hdrs:
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names |= set(re.findall(r"\b(gsi_[a-z0-9_]+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_2306_10379_gb300 import build
    return build.build()


def test_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(gsi_[a-z0-9_]+)", out))
    missing = _declared() - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"


def test_loads_with_ctypes(libpath):
    from paper_2306_10379_gb300 import gsi
    L = gsi.lib()
    for name in _declared():
        assert hasattr(L, name)
    assert L.gsi_status_str(0) == b"ok"
    assert set(gsi.EXPORTED) <= _declared()


def test_host_only_calls():
    """Argument checks and the host SELL builder need no GPU."""
    import ctypes
    import numpy as np
    from paper_2306_10379_gb300 import gsi
    o = gsi.Opts()
    assert gsi.lib().gsi_default_opts(ctypes.byref(o)) == 0
    assert o.tol == 1e-8 and o.max_iters == 10000 and o.which == 1
    assert gsi.lib().gsi_create(None, 4, None, 0, None, None, None) == gsi.GSI_ERR_ARG
    rp = np.array([0, 2, 3, 3], np.int64)
    ci = np.array([0, 1, 1], np.int32)
    va = np.array([1.0, 2.0, 3.0])
    perm, cptr, clen, scol, sval = gsi.csr_to_sell(3, rp, ci, va, C=2, sigma=2)
    assert perm.tolist() == [0, 1, 2, -1]
    assert clen.tolist() == [2, 0]


def test_csr_to_dia_host_layout():
    """The host diagonal layout: offsets of a 3D stencil, values by row and
    diagonal with zeros where the CSR has no entry, and None beyond max_diags."""
    import numpy as np
    from paper_2306_10379_gb300 import gsi, inputs as I
    A = I.fd_laplacian((5, 4, 3))
    off, dia = gsi.csr_to_dia(A.n, A.rowptr, A.colidx, A.val)
    assert off.tolist() == [-20, -5, -1, 0, 1, 5, 20]
    dense = np.zeros((A.n, A.n))
    for r in range(A.n):
        for k in range(A.rowptr[r], A.rowptr[r + 1]):
            dense[r, A.colidx[k]] = A.val[k]
    for r in range(A.n):
        for d, o in enumerate(off):
            c = r + o
            assert dia[r, d] == (dense[r, c] if 0 <= c < A.n else 0.0)
    assert gsi.csr_to_dia(A.n, A.rowptr, A.colidx, A.val, max_diags=5) is None
