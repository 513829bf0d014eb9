"""Failure detection of the grid barrier, without faulting the GPU: every
wait of the cooperative iteration loop has a time limit after which the
kernel records APO_ERR_TIMEOUT and returns, so the host sees an error code and
the context stays usable.  The test makes a wait run out by launching fewer
CTAs than the barrier expects (nothing else is broken)."""
import time

import numpy as np
import pytest

from paper_2510_14982_gb300 import inputs

pytestmark = pytest.mark.gpu

APO_OK, APO_ERR_TIMEOUT = 0, 4


@pytest.fixture(scope="module")
def apo():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_14982_gb300 import apo as m
    return m


def test_grid_barrier_completes_with_all_ctas(apo):
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert apo.apo_barrier_selftest(8, 8, rounds=2000) == APO_OK
    assert apo.apo_barrier_selftest(sms, sms, rounds=200) == APO_OK


def test_grid_barrier_wait_runs_out_and_the_context_stays_usable(apo):
    t0 = time.perf_counter()
    rc = apo.apo_barrier_selftest(1, 2, rounds=1)        # the second CTA never arrives
    dt = time.perf_counter() - t0
    assert rc == APO_ERR_TIMEOUT
    assert 3.0 < dt < 60.0                               # the 4 s limit, not a hang
    assert "limit" in apo.apo_last_error()
    # the status was cleared and the context is usable: barriers and runs work again
    assert apo.apo_barrier_selftest(4, 4, rounds=100) == APO_OK
    prob = apo.problem_from_spec(inputs.single_rastrigin(0))
    x, f, c = apo.apo_run(prob, apo.apo_params_make(256, 1, 0.1, 20, 3))   # a grid-mode run
    assert np.isfinite(f) and np.all(np.diff(c) <= 0)
