"""Bounded waits.  Every wait of a kernel on something another party provides (the staged smoother's bulk copies on
an mbarrier, the persistent tail's grid barrier) gives up after a bounded time, sets an error word and returns; the
host reports MG_ERR_TIMEOUT.  mg_selftest_waits makes such a wait run out on purpose (nothing ever arrives): the
status comes back within about a second and the forest keeps working."""
import time

import pytest
import torch

import synthetic as syn

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
MG_ERR_INVALID_ARG, MG_ERR_TIMEOUT = 1, 7


@pytest.mark.parametrize("which,what", [(0, "staged smoother"), (1, "grid barrier")])
def test_a_wait_that_never_completes_times_out(which, what):
    from paper_2403_08063_gb300 import Forest, _lib
    R, n, keys = syn.workload_forest("uniform_2x8")
    f = syn.gaussian_bump_with_noise(R, n, keys, seed=7).to(DEV)
    F = Forest(R, n, keys, precision=1, inner_cycles=2)
    F.set_rhs(f)
    t0 = time.perf_counter()
    st = F.lib.mg_selftest_waits(F.h, which)
    dt = time.perf_counter() - t0
    assert st == MG_ERR_TIMEOUT
    assert what in _lib.load().mg_last_error().decode()
    assert dt < 10.0
    # the error word was cleared and the context is intact: a solve afterwards converges normally
    u = torch.zeros_like(f)
    cycles, rel = F.solve(u, rtol=1e-8)
    assert rel <= 1e-8 and cycles <= 20
    assert F.lib.mg_selftest_waits(F.h, 2) == MG_ERR_INVALID_ARG
