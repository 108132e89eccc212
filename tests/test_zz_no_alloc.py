"""pa_weights_static: the reweighting of one temperature step for callers that
cannot allocate device memory (framework-owned memory pools, services that
forbid allocation after start-up, one-off queries without a context).

The entry point is called through the C ABI on buffers the test owns.  Its
fixed-point expected copy numbers must equal the CPU oracle's element by
element and its ln Q the oracle's to 1e-12, on energies taken from a GPU
population; the copy numbers pa_step drew from the same population must be
consistent with them.  Two calls in a row (the second on a smaller lattice)
show that no stale scratch from the first call leaks into the second, and the
device's free memory is the same before and after the calls.  This file is
collected last on purpose.
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

FRAC = 2.0 ** 40


def _case(dim, L, R, rule, couplings, seed, steps_before):
    """A population advanced to steps_before, its energies there, and what pa_step
    then computed from them (ln Q, copy numbers)."""
    betas = np.linspace(0.0, 1.2, 13)
    thetas = np.full(12, 3, np.uint32)
    pop = pa.Population(dim, L, R, betas, thetas, rule, seed, couplings=couplings)
    pop.step(steps_before)
    E_host = pop.energies().copy()
    pop.step(1)
    i = steps_before + 1
    case = {"dim": dim, "L": L, "R": R, "rule": rule, "seed": seed, "i": i,
            "dbeta": float(betas[i] - betas[i - 1]), "E": E_host,
            "lnQ_step": pop.observables()["lnQ"], "counts": pop.counts().copy()}
    pop.close()
    return case


def _call(case, parity, E_dev, lnQ_dev, f_dev, stream):
    pa.pa_weights_static(E_dev.data_ptr(), len(case["E"]), case["R"], case["dim"], case["L"],
                         parity, case["dbeta"], lnQ_dev.data_ptr(), f_dev.data_ptr(),
                         stream.cuda_stream)


def _check(case, lnQ_dev, f_dev):
    lnQ = float(lnQ_dev.cpu()[0])
    f = f_dev.cpu().numpy().view(np.uint64)
    ref = O.resample(case["E"], case["R"], case["dbeta"], O.RESAMPLERS[case["rule"]],
                     case["seed"], case["i"])
    assert ref["status"] == 0
    assert np.array_equal(f, ref["f"])                      # bit-exact fixed point
    assert math.isclose(lnQ, ref["lnQ"], rel_tol=1e-12, abs_tol=1e-15)
    assert math.isclose(lnQ, case["lnQ_step"], rel_tol=1e-12, abs_tol=1e-15)
    # the copy numbers pa_step drew are the oracle's draws on these weights
    assert np.array_equal(case["counts"], ref["counts"])
    if case["rule"] == "nearest":
        lo = (f >> np.uint64(40)).astype(np.int64)
        c = case["counts"].astype(np.int64)
        assert np.all((c >= lo) & (c <= lo + 1))
    tau = f.astype(np.float64) / FRAC
    assert abs(tau.sum() - case["R"]) < 1e-6 * case["R"]     # sum of tau-hat is R


def test_weights_without_allocation_match_oracle_twice():
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream(dev)
    # call 1: 2D Ising L=16 (257 energy levels), nearest-integer rule
    c1 = _case(2, 16, 1000, "nearest", ("ferro",), 3, 4)
    # call 2: 3D +-J spin glass L=4 (97 levels): stale histogram entries of call 1
    # would change its weights
    J = O.disorder(3, 4, 3, 2)
    par2 = int((J == -1).sum()) & 1
    c2 = _case(3, 4, 700, "systematic", ("ea", 3, 2), 5, 6)
    bufs = []
    for c in (c1, c2):
        bufs.append((torch.from_numpy(c["E"].astype(np.int32)).to(dev),
                     torch.full((1,), float("inf"), dtype=torch.float64, device=dev),
                     torch.zeros(len(c["E"]), dtype=torch.int64, device=dev)))
    # a first call loads the library's device code on this device
    _call(c2, par2, *bufs[1], stream)
    torch.cuda.synchronize(dev)
    free0, _ = torch.cuda.mem_get_info(dev)
    bufs[1][1].fill_(float("inf"))
    bufs[1][2].zero_()
    torch.cuda.synchronize(dev)
    _call(c1, 0, *bufs[0], stream)
    _call(c2, par2, *bufs[1], stream)
    torch.cuda.synchronize(dev)
    free1, _ = torch.cuda.mem_get_info(dev)
    assert free1 == free0  # the calls allocated no device memory
    _check(c1, bufs[0][1], bufs[0][2])
    _check(c2, bufs[1][1], bufs[1][2])


def test_weights_static_rejects_wrong_parity_energies():
    """An energy whose unsatisfied-bond count has the wrong parity for the given
    coupling parity is not a valid energy of the lattice: ln Q is NaN and the
    copy-number buffer is left untouched."""
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream(dev)
    L, N = 8, 64
    E = np.full(50, -2 * N + 8, np.int32)        # U = 4: parity 0
    E_dev = torch.from_numpy(E).to(dev)
    lnQ = torch.zeros(1, dtype=torch.float64, device=dev)
    f = torch.full((50,), 7, dtype=torch.int64, device=dev)
    pa.pa_weights_static(E_dev.data_ptr(), 50, 50, 2, L, 0, 0.1, lnQ.data_ptr(), f.data_ptr(),
                         stream.cuda_stream)
    torch.cuda.synchronize(dev)
    assert math.isfinite(float(lnQ.cpu()[0]))
    f.fill_(7)
    pa.pa_weights_static(E_dev.data_ptr(), 50, 50, 2, L, 1, 0.1, lnQ.data_ptr(), f.data_ptr(),
                         stream.cuda_stream)   # the same energies claimed for parity 1
    torch.cuda.synchronize(dev)
    assert math.isnan(float(lnQ.cpu()[0]))
    assert np.all(f.cpu().numpy() == 7)
    E[17] += 2                                   # U = 5 among parity-0 energies
    E_dev = torch.from_numpy(E).to(dev)
    lnQ.zero_()
    pa.pa_weights_static(E_dev.data_ptr(), 50, 50, 2, L, 0, 0.1, lnQ.data_ptr(), f.data_ptr(),
                         stream.cuda_stream)
    torch.cuda.synchronize(dev)
    assert math.isnan(float(lnQ.cpu()[0]))
    assert np.all(f.cpu().numpy() == 7)


def test_weights_static_rejects_oversized_lattices():
    dev = torch.device("cuda", torch.cuda.current_device())
    buf = torch.zeros(4, dtype=torch.int64, device=dev)
    with pytest.raises(pa.PAError) as ei:
        pa.pa_weights_static(buf.data_ptr(), 4, 4, 2, 256, 0, 0.01, buf.data_ptr(),
                             buf.data_ptr(), 0)
    assert ei.value.status == pa.PA_ERR_LIMIT
