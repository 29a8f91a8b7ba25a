"""Failure detection on the GPU without a fault: every wait of the persistent
kernel's barriers is bounded.  A barrier at which one CTA never arrives makes
the others' waits run out; they record ACS_ERR_DEVICE_TIMEOUT, the kernel
returns normally, and the same handle then solves a problem as usual."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2103_00736_gb300 import capi, instances as I  # noqa: E402
from oracle import kkt  # noqa: E402


def test_barrier_wait_runs_out_and_the_context_stays_usable():
    inst = I.small_lp()
    with capi.Solver(inst, projection=capi.PROJ_CG) as s:
        ns = capi.acs_debug_barrier_ns(s.h, 100)            # the healthy barrier first
        assert 0 < ns < 1e6
        st, waited = capi.acs_debug_barrier_timeout(s.h)
        assert st == capi.ERR_DEVICE_TIMEOUT, capi.acs_status_string(st)
        assert 1500.0 <= waited <= 20000.0                    # the bound is 2 s
        assert s.solve(tol=1e-6, max_iter=5000) == capi.SOLVED
        rc, x, y, z, iters, res = s.get()
    assert kkt.max_residual(kkt.residuals(inst.to_scipy(), inst.b, inst.c, x, y, z, inst.n, [])) <= 1e-6
    assert torch.cuda.is_available() and torch.zeros(4, device="cuda").sum().item() == 0.0
