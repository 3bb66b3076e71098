"""Bounded device waits: a wait on the tensor core that runs out returns
GSI_ERR_TIMEOUT through the solver, and the context stays usable.

The first waits of the tcgen05 kernels are given a limit of 0 polls, so they
give up at once; the kernel then drains the tensor core with the full bound
(every product already issued completes before the tensor memory is
released), leaves non-finite outputs and counts the event, which the solver
maps to GSI_ERR_TIMEOUT. Nothing faults or hangs: no wait is left without a
bound and no product is in flight when a kernel returns.
"""
import numpy as np
import pytest

from paper_2306_10379_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_wait_limit_gives_timeout_status_then_normal_solve(torch_cuda):
    from paper_2306_10379_gb300 import gsi
    dims, p = (32, 32), 8
    A = I.fd_laplacian(dims)
    lam = I.laplacian_eigenvalues(dims)
    X0 = I.start_block(A.n, p, I.SEED_BASE)
    gsi.set_tensor_path(0)
    with gsi.Solver(A, p, X0, method="cg", tol=1e-8, anorm=lam[0]) as s:
        before = gsi.device_timeouts()
        gsi.set_wait_limit(0)
        try:
            with pytest.raises(gsi.GsiError) as e:
                s.step(1)
        finally:
            gsi.set_wait_limit(-1)
        assert e.value.status == gsi.GSI_ERR_TIMEOUT
        assert gsi.device_timeouts() > before
        # same context: a restart from X0 and a normal solve
        s.reset(X0)
        info = s.solve()
        X, ev = s.basis()
    assert info["converged"] == 1
    assert np.max(np.abs(ev - lam[:p]) / lam[:p]) < 1e-10
    # and a fresh context
    with gsi.Solver(A, p, X0, method="cg", tol=1e-8, anorm=lam[0]) as s:
        assert s.solve()["converged"] == 1
