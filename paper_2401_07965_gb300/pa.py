"""Thin Python binding of the C ABI in include/pa.h (argument marshalling only).

Every function below has the name of the C entry point it calls; the work of a
population-annealing step runs in the CUDA kernels of libpa.so.  PyTorch is
used, when wanted, only to own the device workspace and to supply the stream.

If libpa.so cannot be loaded this module raises at import time: there is no
fallback path.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

from . import build as _build

PA_OK, PA_ERR_ARG, PA_ERR_CUDA, PA_ERR_NOMEM, PA_ERR_CAPACITY = 0, 1, 2, 3, 4
PA_ERR_POISSON_KMAX, PA_ERR_TIMEOUT, PA_ERR_STATE, PA_ERR_DONE, PA_ERR_LIMIT = 5, 6, 7, 8, 9

PA_MULTINOMIAL, PA_SYSTEMATIC, PA_RESIDUAL, PA_POISSON, PA_NEAREST = 0, 1, 2, 3, 4
RESAMPLERS = {"multinomial": 0, "systematic": 1, "residual": 2, "poisson": 3, "nearest": 4}

PA_COUPLING_FERRO, PA_COUPLING_EA_PM, PA_COUPLING_EXPLICIT = 0, 1, 2
PA_ARRAY_SPINS, PA_ARRAY_ENERGY, PA_ARRAY_FAMILY = 0, 1, 2
PA_ARRAY_COUNTS, PA_ARRAY_ANCESTOR, PA_ARRAY_MAGNET, PA_ARRAY_WEIGHT = 3, 4, 5, 6

EXPORTS = ["pa_workspace_bytes", "pa_init", "pa_step", "pa_sync", "pa_observables", "pa_trace",
           "pa_free_energy", "pa_get_array", "pa_set_state", "pa_enable_timing",
           "pa_sweep_timing", "pa_launch_count", "pa_destroy", "pa_strerror",
           "pa_weights_static", "pa_set_sweep_threads", "pa_get_sweep_threads",
           "pa_batch_workspace_bytes", "pa_batch_init", "pa_batch_size", "pa_run_observables",
           "pa_run_trace", "pa_run_free_energy", "pa_run_get_array", "pa_weighted",
           "pa_set_graph", "pa_set_controller", "pa_schedule_taken", "pa_mlp_scratch_bytes",
           "pa_mlp_forward", "pa_mlp_gradients", "pa_mlp_adam", "pa_overlap",
           "pa_set_partial_resampling", "pa_weighted_rows", "pa_set_sweep_queue",
           "pa_run_schedule_taken", "pa_set_wait_test", "pa_set_sweep_groups",
           "pa_get_sweep_groups"]


class pa_lattice(C.Structure):
    _fields_ = [("dim", C.c_int32), ("L", C.c_int32)]


class pa_couplings(C.Structure):
    _fields_ = [("kind", C.c_int32), ("realization", C.c_uint32), ("disorder_seed", C.c_uint64),
                ("J", C.POINTER(C.c_int8))]


class pa_schedule(C.Structure):
    _fields_ = [("n_steps", C.c_int32), ("beta", C.POINTER(C.c_double)),
                ("theta", C.POINTER(C.c_uint32))]


class pa_obs(C.Structure):
    _fields_ = [("step", C.c_int32), ("R_i", C.c_uint32), ("R_prev", C.c_uint32),
                ("pad0", C.c_uint32), ("beta", C.c_double), ("lnQ", C.c_double),
                ("sum_lnQ", C.c_double), ("sumE", C.c_int64), ("sumE2", C.c_int64),
                ("sumAbsM", C.c_int64), ("sumM2", C.c_int64), ("sumC2", C.c_int64),
                ("accepts", C.c_uint64), ("entropy", C.c_double), ("sv", C.c_double),
                ("e", C.c_double), ("e2", C.c_double), ("absm", C.c_double), ("m2", C.c_double),
                ("c", C.c_double), ("chi", C.c_double), ("rho_t", C.c_double),
                ("accept_rate", C.c_double), ("features", C.c_float * 8),
                ("u_next", C.c_int32), ("theta_next", C.c_uint32), ("ess", C.c_double),
                ("resampled", C.c_int32), ("pad1", C.c_int32)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_
             if k not in ("pad0", "pad1", "features")}
        d["features"] = list(self.features)
        return d


class pa_run_spec(C.Structure):
    _fields_ = [("lattice", pa_lattice), ("couplings", pa_couplings), ("R", C.c_uint32),
                ("R_cap", C.c_uint32), ("ensemble", C.c_int32)]


class pa_weighted_obs(C.Structure):
    _fields_ = [("step", C.c_int32), ("n_runs", C.c_int32), ("beta", C.c_double),
                ("lnZ", C.c_double), ("minus_beta_F", C.c_double), ("w_max", C.c_double),
                ("eff_runs", C.c_double), ("e", C.c_double), ("e2", C.c_double),
                ("absm", C.c_double), ("m2", C.c_double), ("c", C.c_double), ("chi", C.c_double),
                ("c_naive", C.c_double), ("chi_naive", C.c_double), ("e_plain", C.c_double),
                ("c_plain", C.c_double), ("chi_plain", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class pa_run_row(C.Structure):
    _fields_ = [("R_i", C.c_uint32), ("R", C.c_uint32), ("sum_lnQ", C.c_double),
                ("sumE", C.c_int64), ("sumE2", C.c_int64), ("sumAbsM", C.c_int64),
                ("sumM2", C.c_int64), ("wsum", C.c_double), ("wE", C.c_double),
                ("wE2", C.c_double), ("wAM", C.c_double), ("wM2", C.c_double)]


PA_MLP_NPARAM = 4866


class pa_controller(C.Structure):
    _fields_ = [("params", C.POINTER(C.c_uint16)), ("use_mlp", C.c_int32),
                ("plain_units", C.c_int32), ("plain_theta", C.c_uint32),
                ("theta_min", C.c_uint32), ("theta_max", C.c_uint32), ("budget", C.c_uint32),
                ("u_max", C.c_int32)]


class PAError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {pa_strerror(status)} (status {status})")


def _load():
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"libpa.so is not built ({path}); run __graft_entry__.build() first")
    lib = C.CDLL(path)
    vp, sz = C.c_void_p, C.c_size_t
    lib.pa_workspace_bytes.argtypes = [C.POINTER(pa_lattice), C.c_uint32, C.c_uint32, C.c_int32,
                                       C.c_int]
    lib.pa_workspace_bytes.restype = sz
    lib.pa_init.argtypes = [C.POINTER(vp), C.POINTER(pa_lattice), C.POINTER(pa_couplings),
                            C.c_uint32, C.c_uint32, C.POINTER(pa_schedule), C.c_int, C.c_uint64,
                            vp, vp, sz]
    lib.pa_step.argtypes = [vp, C.c_int32]
    lib.pa_sync.argtypes = [vp]
    lib.pa_observables.argtypes = [vp, C.POINTER(pa_obs)]
    lib.pa_trace.argtypes = [vp, C.POINTER(pa_obs), C.c_int32, C.POINTER(C.c_int32)]
    lib.pa_free_energy.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_double)]
    lib.pa_get_array.argtypes = [vp, C.c_int, vp, sz, C.POINTER(sz)]
    lib.pa_set_state.argtypes = [vp, C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.c_uint32,
                                 C.c_int32, C.c_double]
    lib.pa_enable_timing.argtypes = [vp, C.c_int32]
    lib.pa_sweep_timing.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_int64),
                                    C.POINTER(C.c_double)]
    lib.pa_launch_count.argtypes = [vp]
    lib.pa_launch_count.restype = C.c_int64
    lib.pa_destroy.argtypes = [vp]
    lib.pa_weights_static.argtypes = [vp, C.c_uint32, C.c_uint32, C.c_int32, C.c_int32,
                                      C.c_int32, C.c_double, vp, vp, vp]
    lib.pa_batch_workspace_bytes.argtypes = [C.POINTER(pa_run_spec), C.c_int32, C.c_int32,
                                             C.c_int]
    lib.pa_batch_workspace_bytes.restype = sz
    lib.pa_batch_init.argtypes = [C.POINTER(vp), C.POINTER(pa_run_spec), C.c_int32,
                                  C.POINTER(pa_schedule), C.c_int, C.c_uint64, vp, vp, sz]
    lib.pa_batch_size.argtypes = [vp]
    lib.pa_batch_size.restype = C.c_int32
    lib.pa_run_observables.argtypes = [vp, C.c_int32, C.POINTER(pa_obs)]
    lib.pa_run_trace.argtypes = [vp, C.c_int32, C.POINTER(pa_obs), C.c_int32,
                                 C.POINTER(C.c_int32)]
    lib.pa_run_free_energy.argtypes = [vp, C.c_int32, C.POINTER(C.c_double),
                                       C.POINTER(C.c_double)]
    lib.pa_run_get_array.argtypes = [vp, C.c_int32, C.c_int, vp, sz, C.POINTER(sz)]
    lib.pa_weighted.argtypes = [vp, C.c_int32, C.POINTER(pa_weighted_obs), C.c_int32,
                                C.POINTER(C.c_int32)]
    lib.pa_set_graph.argtypes = [vp, C.c_int32]
    lib.pa_set_partial_resampling.argtypes = [vp, C.c_double]
    lib.pa_weighted_rows.argtypes = [C.POINTER(pa_run_row), C.c_int32, C.c_int32, C.c_double,
                                     C.c_int32, C.POINTER(pa_weighted_obs), vp]
    lib.pa_overlap.argtypes = [vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.c_int32,
                               vp, C.POINTER(C.c_double)]
    lib.pa_set_controller.argtypes = [vp, C.POINTER(pa_controller)]
    lib.pa_schedule_taken.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_uint32),
                                      C.c_int32, C.POINTER(C.c_int32)]
    lib.pa_run_schedule_taken.argtypes = [vp, C.c_int32, C.POINTER(C.c_double),
                                          C.POINTER(C.c_uint32), C.c_int32, C.POINTER(C.c_int32)]
    lib.pa_mlp_scratch_bytes.argtypes = [C.c_int32]
    lib.pa_mlp_scratch_bytes.restype = sz
    lib.pa_mlp_forward.argtypes = [vp, vp, C.c_int32, vp, vp]
    lib.pa_mlp_gradients.argtypes = [vp, vp, vp, vp, C.c_int32, vp, vp, vp, sz, vp]
    lib.pa_mlp_adam.argtypes = [vp, vp, vp, vp, vp, C.c_int32, C.c_float, vp]
    lib.pa_set_sweep_threads.argtypes = [vp, C.c_int32]
    lib.pa_set_sweep_queue.argtypes = [vp, C.c_int32]
    lib.pa_set_wait_test.argtypes = [vp, C.c_int32]
    lib.pa_set_sweep_groups.argtypes = [vp, C.c_int32]
    lib.pa_get_sweep_groups.argtypes = [vp]
    lib.pa_get_sweep_groups.restype = C.c_int32
    lib.pa_get_sweep_threads.argtypes = [vp]
    lib.pa_get_sweep_threads.restype = C.c_int32
    lib.pa_strerror.argtypes = [C.c_int]
    lib.pa_strerror.restype = C.c_char_p
    for name in EXPORTS:
        if name not in ("pa_workspace_bytes", "pa_launch_count", "pa_strerror",
                        "pa_get_sweep_threads", "pa_batch_workspace_bytes", "pa_batch_size",
                        "pa_mlp_scratch_bytes"):
            getattr(lib, name).restype = C.c_int
    return lib


_lib = _load()


def _check(status, where):
    if status != PA_OK:
        raise PAError(status, where)


def _lat(dim, L):
    return pa_lattice(int(dim), int(L))


def _couplings(couplings, keep):
    """('ferro',), ('ea', disorder_seed, realization) or ('explicit', J int8 array)."""
    if couplings[0] == "ferro":
        return pa_couplings(PA_COUPLING_FERRO, 0, 0, None)
    if couplings[0] == "ea":
        return pa_couplings(PA_COUPLING_EA_PM, int(couplings[2]), int(couplings[1]), None)
    if couplings[0] == "explicit":
        J = np.ascontiguousarray(couplings[1], np.int8)
        keep.append(J)
        return pa_couplings(PA_COUPLING_EXPLICIT, 0, 0, J.ctypes.data_as(C.POINTER(C.c_int8)))
    raise ValueError(f"unknown couplings {couplings[0]!r}")


def _schedule(betas, thetas, keep):
    b = np.ascontiguousarray(betas, np.float64)
    t = np.ascontiguousarray(thetas, np.uint32)
    keep += [b, t]
    return pa_schedule(len(b) - 1, b.ctypes.data_as(C.POINTER(C.c_double)),
                       t.ctypes.data_as(C.POINTER(C.c_uint32)))


def _specs(runs, keep):
    """runs: list of dicts with dim, L, R, optional R_cap, couplings, ensemble."""
    arr = (pa_run_spec * len(runs))()
    for k, r in enumerate(runs):
        arr[k] = pa_run_spec(_lat(r["dim"], r["L"]), _couplings(r.get("couplings", ("ferro",)),
                                                               keep),
                             int(r["R"]), int(r.get("R_cap", 0)), int(r.get("ensemble", 0)))
    return arr


# ---- the C entry points, one to one ---------------------------------------------------------

def pa_strerror(status: int) -> str:
    return _lib.pa_strerror(int(status)).decode()


def pa_workspace_bytes(dim, L, R, R_cap, n_steps, resampler) -> int:
    lat = _lat(dim, L)
    return int(_lib.pa_workspace_bytes(C.byref(lat), R, R_cap, n_steps, int(resampler)))


def pa_init(dim, L, couplings, R, R_cap, betas, thetas, resampler, seed, stream=0,
            workspace=0, workspace_bytes=0):
    """couplings: ('ferro',), ('ea', disorder_seed, realization) or ('explicit', J int8 array)."""
    lat = _lat(dim, L)
    keep = []
    cpl = _couplings(couplings, keep)
    sch = _schedule(betas, thetas, keep)
    ctx = C.c_void_p()
    st = _lib.pa_init(C.byref(ctx), C.byref(lat), C.byref(cpl), int(R), int(R_cap), C.byref(sch),
                      int(resampler), int(seed) & (2 ** 64 - 1), C.c_void_p(stream),
                      C.c_void_p(workspace), int(workspace_bytes))
    del keep
    _check(st, "pa_init")
    return ctx


def pa_step(ctx, n=1):
    _check(_lib.pa_step(ctx, int(n)), "pa_step")


def pa_sync(ctx):
    _check(_lib.pa_sync(ctx), "pa_sync")


def pa_observables(ctx) -> dict:
    o = pa_obs()
    _check(_lib.pa_observables(ctx, C.byref(o)), "pa_observables")
    return o.as_dict()


def pa_trace(ctx, max_rows) -> list:
    rows = (pa_obs * max_rows)()
    n = C.c_int32()
    _check(_lib.pa_trace(ctx, rows, max_rows, C.byref(n)), "pa_trace")
    return [rows[i].as_dict() for i in range(n.value)]


def pa_free_energy(ctx):
    a, b = C.c_double(), C.c_double()
    _check(_lib.pa_free_energy(ctx, C.byref(a), C.byref(b)), "pa_free_energy")
    return a.value, b.value


_ARRAY_DTYPE = {PA_ARRAY_SPINS: np.uint32, PA_ARRAY_ENERGY: np.int32, PA_ARRAY_FAMILY: np.uint32,
                PA_ARRAY_COUNTS: np.uint32, PA_ARRAY_ANCESTOR: np.uint32,
                PA_ARRAY_MAGNET: np.int32, PA_ARRAY_WEIGHT: np.float64}


def pa_get_array(ctx, which, capacity):
    out = np.zeros(int(capacity), _ARRAY_DTYPE[which])
    n = C.c_size_t()
    _check(_lib.pa_get_array(ctx, int(which), out.ctypes.data_as(C.c_void_p), out.size,
                             C.byref(n)), "pa_get_array")
    return out[: n.value]


def pa_set_state(ctx, spins_words, family, R_i, step, sum_lnQ):
    s = np.ascontiguousarray(spins_words, np.uint32)
    fam_p = None
    if family is not None:
        f = np.ascontiguousarray(family, np.uint32)
        fam_p = f.ctypes.data_as(C.POINTER(C.c_uint32))
    _check(_lib.pa_set_state(ctx, s.ctypes.data_as(C.POINTER(C.c_uint32)), fam_p, int(R_i),
                             int(step), float(sum_lnQ)), "pa_set_state")


def pa_enable_timing(ctx, on=True):
    _check(_lib.pa_enable_timing(ctx, 1 if on else 0), "pa_enable_timing")


def pa_sweep_timing(ctx):
    ms, n, u = C.c_double(), C.c_int64(), C.c_double()
    _check(_lib.pa_sweep_timing(ctx, C.byref(ms), C.byref(n), C.byref(u)), "pa_sweep_timing")
    return ms.value, n.value, u.value


def pa_launch_count(ctx) -> int:
    return int(_lib.pa_launch_count(ctx))


def pa_weights_static(E_ptr, R_prev, R, dim, L, parity, dbeta, lnQ_ptr, f_ptr, stream=0):
    """Device pointers in, device pointers out; allocates nothing (see include/pa.h)."""
    _check(_lib.pa_weights_static(C.c_void_p(E_ptr), int(R_prev), int(R), int(dim), int(L),
                                  int(parity), float(dbeta), C.c_void_p(lnQ_ptr),
                                  C.c_void_p(f_ptr), C.c_void_p(stream)), "pa_weights_static")


def pa_set_sweep_threads(ctx, threads):
    _check(_lib.pa_set_sweep_threads(ctx, int(threads)), "pa_set_sweep_threads")


def pa_set_sweep_queue(ctx, cap):
    _check(_lib.pa_set_sweep_queue(ctx, int(cap)), "pa_set_sweep_queue")


def pa_set_wait_test(ctx, on):
    _check(_lib.pa_set_wait_test(ctx, int(on)), "pa_set_wait_test")


def pa_set_sweep_groups(ctx, mult):
    _check(_lib.pa_set_sweep_groups(ctx, int(mult)), "pa_set_sweep_groups")


def pa_get_sweep_groups(ctx) -> int:
    return int(_lib.pa_get_sweep_groups(ctx))


def pa_get_sweep_threads(ctx) -> int:
    return int(_lib.pa_get_sweep_threads(ctx))


def pa_batch_workspace_bytes(runs, n_steps, resampler) -> int:
    keep = []
    specs = _specs(runs, keep)
    return int(_lib.pa_batch_workspace_bytes(specs, len(runs), n_steps, int(resampler)))


def pa_batch_init(runs, betas, thetas, resampler, seed, stream=0, workspace=0,
                  workspace_bytes=0):
    keep = []
    specs = _specs(runs, keep)
    sch = _schedule(betas, thetas, keep)
    ctx = C.c_void_p()
    _check(_lib.pa_batch_init(C.byref(ctx), specs, len(runs), C.byref(sch), int(resampler),
                              int(seed) & (2 ** 64 - 1), C.c_void_p(stream),
                              C.c_void_p(workspace), int(workspace_bytes)), "pa_batch_init")
    return ctx


def pa_batch_size(ctx) -> int:
    return int(_lib.pa_batch_size(ctx))


def pa_run_observables(ctx, run) -> dict:
    o = pa_obs()
    _check(_lib.pa_run_observables(ctx, int(run), C.byref(o)), "pa_run_observables")
    return o.as_dict()


def pa_run_trace(ctx, run, max_rows) -> list:
    rows = (pa_obs * max_rows)()
    n = C.c_int32()
    _check(_lib.pa_run_trace(ctx, int(run), rows, max_rows, C.byref(n)), "pa_run_trace")
    return [rows[i].as_dict() for i in range(n.value)]


def pa_run_free_energy(ctx, run):
    a, b = C.c_double(), C.c_double()
    _check(_lib.pa_run_free_energy(ctx, int(run), C.byref(a), C.byref(b)), "pa_run_free_energy")
    return a.value, b.value


def pa_run_get_array(ctx, run, which, capacity):
    out = np.zeros(int(capacity), _ARRAY_DTYPE[which])
    n = C.c_size_t()
    _check(_lib.pa_run_get_array(ctx, int(run), int(which), out.ctypes.data_as(C.c_void_p),
                                 out.size, C.byref(n)), "pa_run_get_array")
    return out[: n.value]


def pa_weighted(ctx, ensemble, max_rows) -> list:
    rows = (pa_weighted_obs * max_rows)()
    n = C.c_int32()
    _check(_lib.pa_weighted(ctx, int(ensemble), rows, max_rows, C.byref(n)), "pa_weighted")
    return [rows[i].as_dict() for i in range(n.value)]


def pa_set_graph(ctx, on=True):
    _check(_lib.pa_set_graph(ctx, 1 if on else 0), "pa_set_graph")


def pa_set_partial_resampling(ctx, alpha):
    _check(_lib.pa_set_partial_resampling(ctx, float(alpha)), "pa_set_partial_resampling")


def run_row(obs, R_nominal, partial=False, N=None):
    """pa_run_row from a pa_obs dict (pa_observables / pa_run_observables / a trace row)."""
    r = pa_run_row(int(obs["R_i"]), int(R_nominal), float(obs["sum_lnQ"]), int(obs["sumE"]),
                   int(obs["sumE2"]), int(obs["sumAbsM"]), int(obs["sumM2"]), 0.0, 0.0, 0.0,
                   0.0, 0.0)
    if partial:
        # the weighted averages rescaled to a weight sum of 1
        r.wsum = 1.0
        r.wE, r.wE2 = obs["e"] * N, obs["e2"] * N * N
        r.wAM, r.wM2 = obs["absm"] * N, obs["m2"] * N * N
    return r


def pa_weighted_rows(rows, N, beta, step=0, stream=0) -> dict:
    arr = (pa_run_row * len(rows))(*rows)
    out = pa_weighted_obs()
    _check(_lib.pa_weighted_rows(arr, len(rows), int(N), float(beta), int(step), C.byref(out),
                                 C.c_void_p(stream)), "pa_weighted_rows")
    return out.as_dict()


def pa_overlap(ctx, run_a, run_b, hist_dev_ptr, N, weighted=True):
    """Overlap histograms of run pairs into a device buffer (n_pairs x (N+1) uint32);
    returns the weighted P(k) as a numpy array (or None with weighted=False: asynchronous)."""
    a = np.ascontiguousarray(run_a, np.int32)
    b = np.ascontiguousarray(run_b, np.int32)
    if a.shape != b.shape:
        raise ValueError("run_a and run_b differ in length")
    P = np.zeros(int(N) + 1, np.float64) if weighted else None
    _check(_lib.pa_overlap(ctx, a.ctypes.data_as(C.POINTER(C.c_int32)),
                           b.ctypes.data_as(C.POINTER(C.c_int32)), int(a.size),
                           C.c_void_p(hist_dev_ptr),
                           P.ctypes.data_as(C.POINTER(C.c_double)) if weighted else None),
           "pa_overlap")
    return P


def pa_set_controller(ctx, params_bf16, use_mlp, plain_units, plain_theta, theta_min,
                      theta_max, budget, u_max):
    bits = None if params_bf16 is None else np.ascontiguousarray(params_bf16, np.uint16)
    cfg = pa_controller(None if bits is None else bits.ctypes.data_as(C.POINTER(C.c_uint16)),
                        int(use_mlp), int(plain_units), int(plain_theta), int(theta_min),
                        int(theta_max), int(budget), int(u_max))
    _check(_lib.pa_set_controller(ctx, C.byref(cfg)), "pa_set_controller")


def pa_schedule_taken(ctx, max_rows):
    b = np.zeros(max_rows, np.float64)
    t = np.zeros(max(max_rows - 1, 1), np.uint32)
    n = C.c_int32()
    _check(_lib.pa_schedule_taken(ctx, b.ctypes.data_as(C.POINTER(C.c_double)),
                                  t.ctypes.data_as(C.POINTER(C.c_uint32)), max_rows, C.byref(n)),
           "pa_schedule_taken")
    return b[: n.value], t[: max(n.value - 1, 0)]


def pa_run_schedule_taken(ctx, run, max_rows):
    b = np.zeros(max_rows, np.float64)
    t = np.zeros(max(max_rows - 1, 1), np.uint32)
    n = C.c_int32()
    _check(_lib.pa_run_schedule_taken(ctx, int(run), b.ctypes.data_as(C.POINTER(C.c_double)),
                                      t.ctypes.data_as(C.POINTER(C.c_uint32)), max_rows,
                                      C.byref(n)), "pa_run_schedule_taken")
    return b[: n.value], t[: max(n.value - 1, 0)]


def pa_mlp_scratch_bytes(B) -> int:
    return int(_lib.pa_mlp_scratch_bytes(int(B)))


def pa_mlp_forward(params_bf16_ptr, X_ptr, B, Y_ptr, stream=0):
    _check(_lib.pa_mlp_forward(C.c_void_p(params_bf16_ptr), C.c_void_p(X_ptr), int(B),
                               C.c_void_p(Y_ptr), C.c_void_p(stream)), "pa_mlp_forward")


def pa_mlp_gradients(params_ptr, X_ptr, Yt_ptr, mask_ptr, B, grads_ptr, loss_ptr, scratch_ptr,
                     scratch_bytes, stream=0):
    _check(_lib.pa_mlp_gradients(C.c_void_p(params_ptr), C.c_void_p(X_ptr), C.c_void_p(Yt_ptr),
                                 C.c_void_p(mask_ptr), int(B), C.c_void_p(grads_ptr),
                                 C.c_void_p(loss_ptr), C.c_void_p(scratch_ptr),
                                 int(scratch_bytes), C.c_void_p(stream)), "pa_mlp_gradients")


def pa_mlp_adam(params_ptr, grads_ptr, m_ptr, v_ptr, params_bf16_ptr, step, lr, stream=0):
    _check(_lib.pa_mlp_adam(C.c_void_p(params_ptr), C.c_void_p(grads_ptr), C.c_void_p(m_ptr),
                            C.c_void_p(v_ptr), C.c_void_p(params_bf16_ptr), int(step),
                            float(lr), C.c_void_p(stream)), "pa_mlp_adam")


def pa_destroy(ctx):
    _check(_lib.pa_destroy(ctx), "pa_destroy")


# ---- a convenience owner of one run ---------------------------------------------------------

class Population:
    """One PA run: owns a context and, optionally, a torch-allocated workspace."""

    def __init__(self, dim, L, R, betas, thetas, resampler="systematic", seed=1,
                 couplings=("ferro",), R_cap=0, use_torch_memory=True, stream=None,
                 sweep_threads=None):
        self.dim, self.L, self.N = dim, L, L ** dim
        self.W = (self.N + 31) // 32
        self.betas = np.ascontiguousarray(betas, np.float64)
        self.thetas = np.ascontiguousarray(thetas, np.uint32)
        self.n_steps = len(self.betas) - 1
        self.resampler = RESAMPLERS[resampler] if isinstance(resampler, str) else int(resampler)
        self.R = R
        self.R_cap = R_cap if R_cap else default_capacity(R, self.resampler)
        self._spec = {"dim": dim, "L": L, "R": R, "R_cap": R_cap, "couplings": couplings}
        self._stream_obj = stream
        self._ws = None
        ws_ptr, ws_bytes, stream_ptr = 0, 0, 0
        if use_torch_memory:
            import torch
            nbytes = pa_workspace_bytes(dim, L, R, R_cap, self.n_steps, self.resampler)
            if nbytes == 0:
                raise PAError(PA_ERR_ARG, "pa_workspace_bytes")
            self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
            ws_ptr = (self._ws.data_ptr() + 255) & ~255
            ws_bytes = nbytes
            s = stream if stream is not None else torch.cuda.current_stream()
            stream_ptr = s.cuda_stream
        elif stream is not None:
            stream_ptr = stream.cuda_stream
        self.ctx = pa_init(dim, L, couplings, R, R_cap, self.betas, self.thetas, self.resampler,
                           seed, stream_ptr, ws_ptr, ws_bytes)
        if sweep_threads == "auto":  # the autotuner's choice for this shape (cached)
            from . import tune
            th = int(np.median(self.thetas)) if len(self.thetas) else 0
            specs, so = self._tune_specs(), getattr(self, "_stream_obj", None)
            sweep_threads = tune.best_sweep_threads_batch(specs, theta=th, stream=so)
            groups = tune.best_sweep_groups_batch(specs, theta=th, stream=so)
            if groups > 1:
                pa_set_sweep_groups(self.ctx, groups)
        if sweep_threads:
            pa_set_sweep_threads(self.ctx, sweep_threads)

    def _tune_specs(self):
        return [dict(self._spec)] if hasattr(self, "_spec") else [dict(s) for s in self.specs]

    def close(self):
        if getattr(self, "ctx", None) is not None:
            pa_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n=1):
        pa_step(self.ctx, n)

    def observables(self):
        return pa_observables(self.ctx)

    def trace(self):
        return pa_trace(self.ctx, self.n_steps + 1)

    def free_energy(self):
        return pa_free_energy(self.ctx)

    @property
    def size(self):
        return self.observables()["R_i"]

    def spins_words(self):
        cap = self.R_cap * self.W
        w = pa_get_array(self.ctx, PA_ARRAY_SPINS, cap)
        return w.reshape(-1, self.W)

    def spins(self):
        """int8 sigma[R_i][N] unpacked from the device bits (bit 1 = -1)."""
        w = self.spins_words()
        bits = ((w[:, :, None] >> np.arange(32, dtype=np.uint32)) & 1).reshape(w.shape[0], -1)
        return (1 - 2 * bits[:, : self.N].astype(np.int8)).astype(np.int8)

    def array(self, which):
        return pa_get_array(self.ctx, which, self.R_cap)

    def energies(self):
        return self.array(PA_ARRAY_ENERGY)

    def families(self):
        return self.array(PA_ARRAY_FAMILY)

    def counts(self):
        return self.array(PA_ARRAY_COUNTS)

    def ancestors(self):
        return self.array(PA_ARRAY_ANCESTOR)

    def magnetisations(self):
        return self.array(PA_ARRAY_MAGNET)

    def weights(self):
        return self.array(PA_ARRAY_WEIGHT)

    def set_partial_resampling(self, alpha):
        pa_set_partial_resampling(self.ctx, alpha)


def default_capacity(R, resampler):
    if resampler in (PA_POISSON, PA_NEAREST, "poisson", "nearest"):
        return R + int(math.ceil(10 * math.sqrt(R))) + 64
    return R


class Batch:
    """Several PA runs advanced together (one launch per phase for all runs).

    runs: list of dicts {dim, L, R, R_cap?, couplings?, ensemble?}; all runs share the
    dimension, coupling kind, rule, schedule and seed; run m's draws carry its identity."""

    def __init__(self, runs, betas, thetas, resampler="systematic", seed=1, stream=None,
                 use_torch_memory=True, sweep_threads=None, graph=True):
        self.specs = [dict(r) for r in runs]
        self._stream_obj = stream
        self.M = len(runs)
        self.betas = np.ascontiguousarray(betas, np.float64)
        self.thetas = np.ascontiguousarray(thetas, np.uint32)
        self.n_steps = len(self.betas) - 1
        self.resampler = RESAMPLERS[resampler] if isinstance(resampler, str) else int(resampler)
        self._ws = None
        ws_ptr, ws_bytes, stream_ptr = 0, 0, 0
        if use_torch_memory:
            import torch
            nbytes = pa_batch_workspace_bytes(self.specs, self.n_steps, self.resampler)
            if nbytes == 0:
                raise PAError(PA_ERR_ARG, "pa_batch_workspace_bytes")
            self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
            ws_ptr = (self._ws.data_ptr() + 255) & ~255
            ws_bytes = nbytes
            s = stream if stream is not None else torch.cuda.current_stream()
            stream_ptr = s.cuda_stream
        elif stream is not None:
            stream_ptr = stream.cuda_stream
        self.ctx = pa_batch_init(self.specs, self.betas, self.thetas, self.resampler, seed,
                                 stream_ptr, ws_ptr, ws_bytes)
        if sweep_threads == "auto":  # the autotuner's choice for this shape (cached)
            from . import tune
            th = int(np.median(self.thetas)) if len(self.thetas) else 0
            specs, so = self._tune_specs(), getattr(self, "_stream_obj", None)
            sweep_threads = tune.best_sweep_threads_batch(specs, theta=th, stream=so)
            groups = tune.best_sweep_groups_batch(specs, theta=th, stream=so)
            if groups > 1:
                pa_set_sweep_groups(self.ctx, groups)
        if sweep_threads:
            pa_set_sweep_threads(self.ctx, sweep_threads)
        pa_set_graph(self.ctx, graph)

    def _tune_specs(self):
        return [dict(self._spec)] if hasattr(self, "_spec") else [dict(s) for s in self.specs]

    def close(self):
        if getattr(self, "ctx", None) is not None:
            pa_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n=1):
        pa_step(self.ctx, n)

    def observables(self, run):
        return pa_run_observables(self.ctx, run)

    def trace(self, run):
        return pa_run_trace(self.ctx, run, self.n_steps + 1)

    def free_energy(self, run):
        return pa_run_free_energy(self.ctx, run)

    def weighted(self, ensemble):
        return pa_weighted(self.ctx, ensemble, self.n_steps + 1)

    def set_partial_resampling(self, alpha):
        pa_set_partial_resampling(self.ctx, alpha)

    def overlap(self, pairs):
        """Overlap distribution of run pairs [(a, b), ...] at the current step:
        (hist[n_pairs][N+1] of the number of differing sites k, weighted P(k))."""
        import torch
        spec = self.specs[pairs[0][0]]
        N = spec["L"] ** spec["dim"]
        hist = torch.empty((len(pairs), N + 1), dtype=torch.int32, device="cuda")
        P = pa_overlap(self.ctx, [a for a, _ in pairs], [b for _, b in pairs], hist.data_ptr(),
                       N)
        return hist.cpu().numpy().view(np.uint32), P

    def array(self, run, which):
        spec = self.specs[run]
        cap = spec.get("R_cap") or default_capacity(spec["R"], self.resampler)
        if which == PA_ARRAY_SPINS:
            cap *= (spec["L"] ** spec["dim"] + 31) // 32
        return pa_run_get_array(self.ctx, run, which, cap)

    def spins_words(self, run):
        spec = self.specs[run]
        W = (spec["L"] ** spec["dim"] + 31) // 32
        return self.array(run, PA_ARRAY_SPINS).reshape(-1, W)

    def slot_bases(self):
        """32 x the sweep CTAs of the preceding runs: the replica-slot offset of each run."""
        out, acc = [], 0
        for spec in self.specs:
            out.append(acc)
            cap = spec.get("R_cap") or default_capacity(spec["R"], self.resampler)
            acc += 32 * ((cap + 31) // 32)
        return out
