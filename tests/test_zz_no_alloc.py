"""pa_weights_static: the reweighting of one temperature step for callers that
cannot allocate device memory (framework-owned memory pools, services that
forbid allocation after start-up, one-off queries without a context).

The entry point is called through the C ABI on buffers the test owns; its ln Q
must equal the ln Q that pa_step computed for the same population, and its
fixed-point weights must reproduce the sampling variance that pa_step reported
together with its copy counts.  Two calls in a row, the second on a smaller
lattice, show that no stale scratch from the first call leaks into the second.
This file is collected last on purpose.
"""
import math

import numpy as np
import pytest

from tests.conftest import gpu_available

pytestmark = pytest.mark.gpu

if not gpu_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import torch  # noqa: E402

from oracle import oracle as O  # noqa: E402
from paper_2401_07965_gb300 import pa  # noqa: E402


def _one_call(dim, L, R, rule, couplings, parity, seed, steps_before):
    betas = np.linspace(0.0, 1.2, 13)
    thetas = np.full(12, 3, np.uint32)
    pop = pa.Population(dim, L, R, betas, thetas, rule, seed, couplings=couplings)
    pop.step(steps_before)
    E_host = pop.energies().copy()
    pop.step(1)
    obs = pop.observables()
    counts = pop.counts().astype(np.float64)
    i = steps_before + 1
    dbeta = float(betas[i] - betas[i - 1])
    dev = torch.device("cuda", torch.cuda.current_device())
    E_dev = torch.from_numpy(E_host.astype(np.int32)).to(dev)
    lnQ_dev = torch.full((1,), float("inf"), dtype=torch.float64, device=dev)
    f_dev = torch.zeros(len(E_host), dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream(dev)
    pa.pa_weights_static(E_dev.data_ptr(), len(E_host), R, dim, L, parity, dbeta,
                         lnQ_dev.data_ptr(), f_dev.data_ptr(), stream.cuda_stream)
    torch.cuda.synchronize(dev)
    lnQ = float(lnQ_dev.cpu()[0])
    f = f_dev.cpu().numpy().view(np.uint64)
    assert math.isclose(lnQ, obs["lnQ"], rel_tol=1e-12, abs_tol=1e-15)
    sv = float(((counts - f.astype(np.float64) / 2.0 ** 40) ** 2).sum() / len(E_host))
    assert math.isclose(sv, obs["sv"], rel_tol=1e-9, abs_tol=1e-15)
    pop.close()


def test_weights_without_allocation_match_pa_step_twice():
    # call 1: 2D Ising L=16 (257 energy levels), nearest-integer rule
    _one_call(2, 16, 1000, "nearest", ("ferro",), 0, 3, 4)
    # call 2: 3D +-J spin glass L=4 (97 levels) right after: stale histogram
    # entries of call 1 would change its weights
    J = O.disorder(3, 4, 3, 2)
    parity = int((J == -1).sum()) & 1
    _one_call(3, 4, 700, "systematic", ("ea", 3, 2), parity, 5, 6)


def test_weights_static_rejects_oversized_lattices():
    dev = torch.device("cuda", torch.cuda.current_device())
    buf = torch.zeros(4, dtype=torch.int64, device=dev)
    with pytest.raises(pa.PAError) as ei:
        pa.pa_weights_static(buf.data_ptr(), 4, 4, 2, 256, 0, 0.01, buf.data_ptr(),
                             buf.data_ptr(), 0)
    assert ei.value.status == pa.PA_ERR_LIMIT
