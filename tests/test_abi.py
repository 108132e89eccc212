"""Host-side checks of the C ABI: the library loads, exports every entry point
that include/pa.h declares, and validates arguments before touching a GPU."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"\b(pa_[a-z0-9_]+)\s*\(", txt)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2401_07965_gb300 import build
    build.build()
    return C.CDLL(build.LIB)


def test_header_declares_the_boundary():
    names = _declared()
    for required in ["pa_init", "pa_step", "pa_observables", "pa_free_energy", "pa_get_array",
                     "pa_destroy", "pa_strerror"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_the_header():
    from paper_2401_07965_gb300 import build
    build.build()
    from paper_2401_07965_gb300 import pa
    for name in _declared():
        if name in ("pa_workspace_bytes", "pa_init", "pa_step", "pa_sync", "pa_observables",
                    "pa_trace", "pa_free_energy", "pa_get_array", "pa_set_state",
                    "pa_enable_timing", "pa_sweep_timing", "pa_launch_count", "pa_destroy",
                    "pa_strerror"):
            assert callable(getattr(pa, name))


def test_strerror_and_workspace_sizes(lib):
    from paper_2401_07965_gb300 import pa
    assert pa.pa_strerror(0) == "ok"
    assert "capacity" in pa.pa_strerror(4)
    n1 = pa.pa_workspace_bytes(2, 64, 100000, 0, 200, pa.PA_SYSTEMATIC)
    # two spin buffers of R x 128 words dominate: ~102 MB
    assert 100000 * 128 * 4 * 2 <= n1 < 100000 * 128 * 4 * 2 * 1.1
    assert pa.pa_workspace_bytes(2, 63, 10, 0, 5, pa.PA_SYSTEMATIC) == 0   # odd L
    assert pa.pa_workspace_bytes(4, 8, 10, 0, 5, pa.PA_SYSTEMATIC) == 0    # dim 4
    assert pa.pa_workspace_bytes(2, 8, 0, 0, 5, pa.PA_SYSTEMATIC) == 0     # R = 0
    assert pa.pa_workspace_bytes(2, 8, 10, 5, 5, pa.PA_SYSTEMATIC) == 0    # R_cap < R
    assert pa.pa_workspace_bytes(2, 256, 10, 0, 5, pa.PA_SYSTEMATIC) == 0  # N > 32768
    big = pa.pa_workspace_bytes(2, 8, 1000, 0, 5, pa.PA_NEAREST)
    small = pa.pa_workspace_bytes(2, 8, 1000, 0, 5, pa.PA_SYSTEMATIC)
    assert big > small  # variable-size rules reserve R + 10 sqrt(R) + 64 slots


def test_init_rejects_bad_schedules_without_a_gpu(lib):
    import numpy as np
    from paper_2401_07965_gb300 import pa
    th = np.ones(3, np.uint32)
    for betas in ([0.1, 0.2, 0.3, 0.4], [0.0, 0.2, 0.2, 0.4], [0.0, 0.3, 0.2, 0.4]):
        with pytest.raises(pa.PAError) as ei:
            pa.pa_init(2, 8, ("ferro",), 10, 0, np.array(betas), th, pa.PA_SYSTEMATIC, 1)
        assert ei.value.status == pa.PA_ERR_ARG
    with pytest.raises(pa.PAError):
        pa.pa_init(2, 8, ("explicit", np.zeros(128, np.int8)), 10, 0,
                   np.array([0.0, 0.1, 0.2, 0.3]), th, pa.PA_SYSTEMATIC, 1)
    with pytest.raises(pa.PAError):
        pa.pa_init(2, 8, ("ferro",), 10, 0, np.array([0.0, 0.1, 0.2, 0.3]),
                   np.array([1, 1 << 24, 1], np.uint32), pa.PA_SYSTEMATIC, 1)


def test_population_bound_is_refused_without_a_gpu(lib):
    """R and R_cap must stay below 2^24: the expected copy numbers are 2^-40
    fixed-point integers whose total R 2^40 has to fit in 64 bits."""
    import numpy as np
    from paper_2401_07965_gb300 import pa
    betas, th = np.array([0.0, 0.1, 0.2]), np.ones(2, np.uint32)
    top = (1 << 24) - 1
    assert pa.pa_workspace_bytes(2, 4, top, 0, 2, pa.PA_SYSTEMATIC) > 0
    assert pa.pa_workspace_bytes(2, 4, top + 1, 0, 2, pa.PA_SYSTEMATIC) == 0
    assert pa.pa_workspace_bytes(2, 4, 1000, top + 1, 2, pa.PA_NEAREST) == 0
    for R, cap in ((top + 1, 0), (1000, top + 1), (1 << 30, 0)):
        with pytest.raises(pa.PAError) as ei:
            pa.pa_init(2, 4, ("ferro",), R, cap, betas, th, pa.PA_SYSTEMATIC, 1)
        assert ei.value.status == pa.PA_ERR_LIMIT
        with pytest.raises(pa.PAError) as ei:
            pa.pa_batch_init([{"dim": 2, "L": 4, "R": 10}, {"dim": 2, "L": 4, "R": R,
                                                            "R_cap": cap}],
                             betas, th, pa.PA_SYSTEMATIC, 1)
        assert ei.value.status == pa.PA_ERR_LIMIT
    # the allocation-free weights entry point checks its sizes before any CUDA call
    with pytest.raises(pa.PAError) as ei:
        pa.pa_weights_static(8, 4, top + 1, 2, 8, 0, 0.01, 8, 8, 0)
    assert ei.value.status == pa.PA_ERR_LIMIT
    with pytest.raises(pa.PAError) as ei:
        pa.pa_weights_static(8, 4, 4, 3, 1 << 20, 0, 0.01, 8, 8, 0)
    assert ei.value.status == pa.PA_ERR_LIMIT
    with pytest.raises(pa.PAError) as ei:
        pa.pa_weights_static(8, 4, 4, 2, 8, 2, 0.01, 8, 8, 0)  # parity not 0 or 1
    assert ei.value.status == pa.PA_ERR_ARG


def test_sweep_queue_hook_validates_arguments(lib):
    from paper_2401_07965_gb300 import pa
    assert pa._lib.pa_set_sweep_queue(None, 0) == pa.PA_ERR_ARG


def test_wait_test_hook_validates_arguments(lib):
    from paper_2401_07965_gb300 import pa
    assert pa._lib.pa_set_wait_test(None, 0) == pa.PA_ERR_ARG
    assert pa._lib.pa_set_wait_test(None, 1) == pa.PA_ERR_ARG


def test_sweep_groups_hook_validates_arguments(lib):
    from paper_2401_07965_gb300 import pa
    assert pa._lib.pa_set_sweep_groups(None, 1) == pa.PA_ERR_ARG
    assert pa._lib.pa_get_sweep_groups(None) == 0
