"""Failure path of the bounded waits (Sec. 2 step 2's single-pass scans), made on
purpose without any GPU fault: the test hook pa_set_wait_test makes the first scan
block of every run withhold its prefix, so the other blocks' bounded waits run out.
The step must end with PA_ERR_TIMEOUT within seconds, the context must keep
answering (the same status, then destroy), and a new context on the same device
must run normally afterwards."""
import time

import numpy as np
import pytest

from tests.conftest import gpu_available

pytestmark = pytest.mark.gpu

if not gpu_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2401_07965_gb300 import pa  # noqa: E402


@pytest.mark.parametrize("rule", ["systematic", "multinomial"])
def test_scan_wait_runs_out_and_reports_timeout(rule):
    betas = np.linspace(0.0, 1.0, 11)
    thetas = np.full(10, 2, np.uint32)
    pop = pa.Population(2, 16, 3000, betas, thetas, rule, 5)   # 6 scan blocks
    pop.step(2)
    assert pop.observables()["R_i"] == 3000
    pa.pa_set_wait_test(pop.ctx, 1)
    t0 = time.time()
    with pytest.raises(pa.PAError) as ei:
        pop.step(1)
        pop.observables()
    assert ei.value.status == pa.PA_ERR_TIMEOUT
    assert time.time() - t0 < 60
    # the context still answers: the failure is sticky, nothing else runs
    with pytest.raises(pa.PAError):
        pop.step(1)
    pop.close()
    # the device is fine: a fresh run of the same shape steps normally
    ok = pa.Population(2, 16, 3000, betas, thetas, rule, 5)
    ok.step(3)
    assert ok.observables()["R_i"] == 3000
    ok.close()


def test_wait_test_hook_off_changes_nothing():
    betas = np.linspace(0.0, 1.0, 7)
    thetas = np.full(6, 2, np.uint32)
    a = pa.Population(2, 16, 1500, betas, thetas, "systematic", 9)
    b = pa.Population(2, 16, 1500, betas, thetas, "systematic", 9)
    pa.pa_set_wait_test(b.ctx, 0)
    a.step(6)
    b.step(6)
    assert np.array_equal(a.counts(), b.counts())
    assert a.observables()["lnQ"] == b.observables()["lnQ"]
    a.close()
    b.close()
