"""ctypes wrapper of the plain CPU population-annealing oracle (pa_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg
of the benchmark use it to produce expected values.  The library's product
path never imports this module, and this module imports nothing from the
library.

The oracle follows Sec. 2 of the paper (steps 1-5) one site at a time; see the
header comment of pa_oracle.c for the discretisation it fixes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "pa_oracle.c")
BUILD_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD_DIR, "liboracle.so")
LIB_OMP = os.path.join(BUILD_DIR, "liboracle_omp.so")  # the same source with -fopenmp

MULTINOMIAL, SYSTEMATIC, RESIDUAL, POISSON, NEAREST = 0, 1, 2, 3, 4
RESAMPLERS = {"multinomial": MULTINOMIAL, "systematic": SYSTEMATIC, "residual": RESIDUAL,
              "poisson": POISSON, "nearest": NEAREST}

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile pa_oracle.c with gcc (no FMA contraction) into oracle/_build/liboracle.so
    (single thread: the parity runs) and liboracle_omp.so (-fopenmp: the replica loop of
    the sweeps on all host cores, for the multi-core CPU baseline)."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    for out, extra in ((LIB, []), (LIB_OMP, ["-fopenmp"])):
        if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(SRC):
            tmp = out + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-std=gnu99", "-fPIC", "-shared", "-ffp-contract=off",
                   "-fno-fast-math", *extra, "-o", tmp, SRC, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, out)
    return LIB


class Obs(C.Structure):
    _fields_ = [("R_i", C.c_uint32), ("lnQ", C.c_double), ("sum_lnQ", C.c_double),
                ("sumE", C.c_int64), ("sumE2", C.c_int64), ("sumAbsM", C.c_int64),
                ("sumM2", C.c_int64), ("sumC2", C.c_int64), ("entropy", C.c_double),
                ("sv", C.c_double), ("accepts", C.c_uint64), ("ess", C.c_double),
                ("resampled", C.c_int32), ("wsum", C.c_double), ("wE", C.c_double),
                ("wE2", C.c_double), ("wAM", C.c_double), ("wM2", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib_omp = None


def lib():
    """The single-thread oracle library."""
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _declare(C.CDLL(LIB))
    return _lib


def lib_omp():
    """The same oracle built with -fopenmp (replica loop of the sweeps on all cores)."""
    global _lib_omp
    with _lock:
        if _lib_omp is None:
            build()
            _lib_omp = _declare(C.CDLL(LIB_OMP))
    return _lib_omp


def _declare(L):
    """Argument and result types of the oracle's C entry points."""
    u32p, u64p, i8p, i32p, dp = (C.POINTER(C.c_uint32), C.POINTER(C.c_uint64),
                                 C.POINTER(C.c_int8), C.POINTER(C.c_int32),
                                 C.POINTER(C.c_double))
    L.or_philox.argtypes = [u32p, u32p, u32p]
    L.or_exp.argtypes = [C.c_double]
    L.or_exp.restype = C.c_double
    L.or_energy.argtypes = [C.c_int, C.c_int, i8p, i8p]
    L.or_energy.restype = C.c_int32
    L.or_disorder.argtypes = [C.c_int, C.c_int, C.c_uint64, C.c_uint32, i8p]
    L.or_init_replica.argtypes = [C.c_int, C.c_int, C.c_uint64, C.c_uint32, i8p]
    L.or_thresholds.argtypes = [C.c_double, u32p]
    L.or_sweeps.argtypes = [C.c_int, C.c_int, i8p, i8p, i32p, C.c_uint64, C.c_uint32,
                            C.c_uint32, C.c_uint32, u32p]
    L.or_sweeps.restype = C.c_uint64
    L.or_u_less.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_int,
                            C.c_int, C.c_uint32]
    L.or_u_less.restype = C.c_int
    L.or_resample.argtypes = [i32p, C.c_uint32, C.c_uint32, C.c_double, C.c_int,
                              C.c_uint64, C.c_uint32, C.c_uint32, u32p, u64p, dp, u64p]
    L.or_resample.restype = C.c_int
    L.or_run_create.argtypes = [C.c_int, C.c_int, i8p, C.c_uint32, C.c_uint32, C.c_int,
                                dp, u32p, C.c_int, C.c_uint64]
    L.or_run_create.restype = C.c_void_p
    L.or_run_create_ex.argtypes = [C.c_int, C.c_int, i8p, C.c_uint32, C.c_uint32,
                                   C.c_int, dp, u32p, C.c_int, C.c_uint64, C.c_uint32,
                                   C.c_uint32]
    L.or_run_create_ex.restype = C.c_void_p
    L.or_run_destroy.argtypes = [C.c_void_p]
    L.or_run_step.argtypes = [C.c_void_p]
    L.or_run_step.restype = C.c_int
    for name, rt in [("or_run_status", C.c_int), ("or_run_step_index", C.c_int),
                     ("or_run_size", C.c_uint32), ("or_run_prev_size", C.c_uint32),
                     ("or_run_sum_lnQ", C.c_double), ("or_run_minus_beta_F", C.c_double),
                     ("or_run_spins", C.c_void_p), ("or_run_energies", C.c_void_p),
                     ("or_run_families", C.c_void_p), ("or_run_counts", C.c_void_p),
                     ("or_run_fixed_weights", C.c_void_p),
                     ("or_run_ancestors", C.c_void_p),
                     ("or_run_weights", C.c_void_p)]:
        f = getattr(L, name)
        f.argtypes = [C.c_void_p]
        f.restype = rt
    L.or_run_obs.argtypes = [C.c_void_p, C.POINTER(Obs)]
    L.or_run_set_partial.argtypes = [C.c_void_p, C.c_double]
    L.or_run_set_partial.restype = C.c_int
    return L


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def philox(ctr, key):
    """Philox4x32-10 of counter (4 x uint32) under key (2 x uint32)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib().or_philox(_p(c, C.c_uint32), _p(k, C.c_uint32), _p(out, C.c_uint32))
    return out


def exp(x: float) -> float:
    return lib().or_exp(float(x))


def ferro_couplings(d: int, L: int) -> np.ndarray:
    return np.ones(d * L ** d, np.int8)


def disorder(d: int, L: int, seed: int, realization: int) -> np.ndarray:
    J = np.zeros(d * L ** d, np.int8)
    lib().or_disorder(d, L, seed, realization, _p(J, C.c_int8))
    return J


def energy(d, L, J, sig) -> int:
    J = np.ascontiguousarray(J, np.int8)
    s = np.ascontiguousarray(sig, np.int8)
    return int(lib().or_energy(d, L, _p(J, C.c_int8), _p(s, C.c_int8)))


def init_replica(d, L, seed, j) -> np.ndarray:
    s = np.zeros(L ** d, np.int8)
    lib().or_init_replica(d, L, seed, j, _p(s, C.c_int8))
    return s


def u_less(seed, slot, step, sweep, colour, site, thr) -> bool:
    """The Metropolis test u < thr of one (replica slot, site, sweep, colour, step)."""
    return bool(lib().or_u_less(seed, slot, step, sweep, colour, site, thr))


def thresholds(beta: float) -> np.ndarray:
    t = np.zeros(4, np.uint32)
    lib().or_thresholds(float(beta), _p(t, C.c_uint32))
    return t


def sweeps(d, L, J, sig, seed, step, slot, theta, beta):
    """theta checkerboard rounds of one replica; returns (sig', E', accepted)."""
    J = np.ascontiguousarray(J, np.int8)
    s = np.array(sig, np.int8, copy=True)
    E = np.array([energy(d, L, J, s)], np.int32)
    thr = thresholds(beta)
    acc = lib().or_sweeps(d, L, _p(J, C.c_int8), _p(s, C.c_int8), _p(E, C.c_int32), seed, step,
                          slot, theta, _p(thr, C.c_uint32))
    return s, int(E[0]), int(acc)


def resample(E, R, dbeta, method, seed, step, run_id=0):
    """Weights, ln Q and copy counts from energies E at one temperature step."""
    E = np.ascontiguousarray(E, np.int32)
    n = len(E)
    counts = np.zeros(n, np.uint32)
    f = np.zeros(n, np.uint64)
    lnQ = np.zeros(1, np.float64)
    Rnew = np.zeros(1, np.uint64)
    st = lib().or_resample(_p(E, C.c_int32), n, R, float(dbeta), int(method), seed, step,
                           run_id, _p(counts, C.c_uint32), _p(f, C.c_uint64), _p(lnQ, C.c_double),
                           _p(Rnew, C.c_uint64))
    return {"status": st, "counts": counts, "f": f, "lnQ": float(lnQ[0]), "R_new": int(Rnew[0])}


class Run:
    """A whole PA run of the oracle: Run(...).step() advances one temperature step."""

    def __init__(self, d, L, J, R, betas, thetas, method, seed, R_cap=0, slot_base=0, run_id=0,
                 alpha=None, parallel=False):
        """parallel=True runs the replica loop of the sweeps on all host cores (OpenMP
        build, OMP_NUM_THREADS threads); the results are the same."""
        self._L = lib_omp() if parallel else lib()
        self.d, self.L, self.N = d, L, L ** d
        self.J = np.ascontiguousarray(J, np.int8)
        self.betas = np.ascontiguousarray(betas, np.float64)
        self.thetas = np.ascontiguousarray(thetas, np.uint32)
        self._h = self._L.or_run_create_ex(d, L, _p(self.J, C.c_int8), R, R_cap,
                                         len(self.betas) - 1, _p(self.betas, C.c_double),
                                         _p(self.thetas, C.c_uint32), int(method), seed,
                                         slot_base, run_id)
        if not self._h:
            raise ValueError("oracle: invalid run arguments")
        self.R = R
        if alpha is not None and self._L.or_run_set_partial(self._h, float(alpha)) != 0:
            raise ValueError("oracle: invalid partial-resampling threshold")
        self.partial = alpha is not None

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._L.or_run_destroy(h)
            self._h = None

    def step(self) -> int:
        return self._L.or_run_step(self._h)

    @property
    def status(self):
        return self._L.or_run_status(self._h)

    @property
    def size(self) -> int:
        return self._L.or_run_size(self._h)

    @property
    def prev_size(self) -> int:
        return self._L.or_run_prev_size(self._h)

    def _arr(self, fn, ct, n, dt):
        ptr = getattr(lib(), fn)(self._h)
        return np.ctypeslib.as_array(C.cast(ptr, C.POINTER(ct)), shape=(n,)).astype(dt, copy=True)

    def spins(self):
        return self._arr("or_run_spins", C.c_int8, self.size * self.N, np.int8).reshape(
            self.size, self.N)

    def energies(self):
        return self._arr("or_run_energies", C.c_int32, self.size, np.int32)

    def families(self):
        return self._arr("or_run_families", C.c_uint32, self.size, np.uint32)

    def counts(self):
        return self._arr("or_run_counts", C.c_uint32, self.prev_size, np.uint32)

    def fixed_weights(self):
        return self._arr("or_run_fixed_weights", C.c_uint64, self.prev_size, np.uint64)

    def ancestors(self):
        return self._arr("or_run_ancestors", C.c_uint32, self.size, np.uint32)

    def weights(self):
        """Per-replica weights under partial resampling (ones otherwise)."""
        if not self.partial:
            return np.ones(self.size)
        return self._arr("or_run_weights", C.c_double, self.size, np.float64)

    def obs(self) -> dict:
        o = Obs()
        self._L.or_run_obs(self._h, C.byref(o))
        return o.as_dict()

    def sum_lnQ(self) -> float:
        return self._L.or_run_sum_lnQ(self._h)

    def minus_beta_F(self) -> float:
        return self._L.or_run_minus_beta_F(self._h)


def pack_spins(sig: np.ndarray) -> np.ndarray:
    """int8 sigma[R][N] -> uint32 words [R][ceil(N/32)], bit (s&31) of word s>>5 set for -1."""
    R, N = sig.shape
    W = (N + 31) // 32
    bits = np.zeros((R, W * 32), np.uint8)
    bits[:, :N] = (sig < 0)
    b = bits.reshape(R, W, 32).astype(np.uint64)
    w = (b << np.arange(32, dtype=np.uint64)).sum(axis=2)
    return w.astype(np.uint32)
