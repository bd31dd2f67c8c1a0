"""Failure detection on the GPU without a GPU fault.

The tensor-core kernels never wait unboundedly: every wait gives up after about a
second and the next synchronising call returns OFA_ERR_TIMEOUT.  The self-test runs
such a wait on a barrier that nothing signals (nothing faults or hangs) and checks
the status and that the context stays usable.  Allocation failures are injected on
the host (OFA_FAULT_ALLOC) and must surface as OFA_ERR_OOM with nothing leaked.
"""
import os
import time

import numpy as np
import pytest

from paper_2206_12661_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev(ofa):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def small_plan(ofa, prec="f16x3"):
    w = I.named("pupil256_grid100_uniform")
    return w, ofa.Plan.from_workload(w, precision=prec)


def test_bounded_wait_gives_up_and_context_survives(ofa, dev):
    t0 = time.perf_counter()
    st = ofa.ofa_selftest_bounded_wait()
    dt = time.perf_counter() - t0
    assert st == ofa.OFA_ERR_TIMEOUT, ofa.ofa_status_string(st)
    assert "gave up" in ofa.ofa_last_error(None)
    assert 0.5 < dt < 30.0, dt
    # the context is still usable: a plan runs and its loop converges as usual
    w, p = small_plan(ofa)
    it, xi = p.iterate(20, want_stats=True)
    p.close()
    assert it == 20 and xi > 0.9


@pytest.mark.parametrize("n", [1, 3, 8, 14, 16])
@pytest.mark.parametrize("prec", ["f16x3", "fp32"])
def test_allocation_failure_is_reported_and_cleaned_up(ofa, dev, n, prec):
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    os.environ["OFA_FAULT_ALLOC"] = str(n)
    try:
        with pytest.raises(ofa.OfaError) as e:
            small_plan(ofa, prec)
    finally:
        del os.environ["OFA_FAULT_ALLOC"]
    assert e.value.status == ofa.OFA_ERR_OOM, e.value
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert abs(free1 - free0) < (8 << 20), (free0, free1)
    # and the next creation, without injection, succeeds
    w, p = small_plan(ofa, prec)
    phase = p.phase()
    p.close()
    assert np.isfinite(phase).all()


def test_destroyed_plan_memory_is_kept_for_reuse_and_trim_releases_it(ofa, dev):
    """ofa_destroy keeps the plan's arena for the next plan; ofa_trim frees it."""
    w = I.named("pupil1024_poisson1000")
    ofa.ofa_trim()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    p = ofa.Plan.from_workload(w, precision="f16x3")
    p.iterate(2)
    phase_a = p.phase()
    p.close()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free0 - free1 > (32 << 20), (free0, free1)    # the arena (~75 MB) is kept
    # a second plan of the same shape reuses it: no further device memory, same result
    q = ofa.Plan.from_workload(w, precision="f16x3")
    torch.cuda.synchronize()
    free2, _ = torch.cuda.mem_get_info()
    q.iterate(2)
    phase_b = q.phase()
    q.close()
    assert abs(free2 - free1) < (8 << 20), (free1, free2)
    assert np.array_equal(phase_a, phase_b)
    ofa.ofa_trim()
    torch.cuda.synchronize()
    free3, _ = torch.cuda.mem_get_info()
    assert abs(free3 - free0) < (8 << 20), (free0, free3)
