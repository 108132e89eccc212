"""Exact reference results for the pins of the oracle (test infrastructure only).

* kaufman_lnZ: Kaufman's closed form (Phys. Rev. 76, 1232 (1949)) of the
  partition function of the L x L periodic Ising ferromagnet,
      Z = 1/2 (2 sinh 2K)^(N/2) (Z1 + Z2 + Z3 + Z4),
      Z1 = prod_{r<L} 2 cosh(L g_{2r+1}/2),  Z2 = prod 2 sinh(L g_{2r+1}/2),
      Z3 = prod_{r<L} 2 cosh(L g_{2r}/2),    Z4 = prod 2 sinh(L g_{2r}/2),
      cosh g_k = cosh 2K coth 2K - cos(pi k / L)  (k > 0),
      g_0 = 2K + ln tanh K,
  evaluated with mpmath at 50 digits.  The paper's free-energy estimator
  (Eq. free-energy-estimator) is checked against it.
* transfer_lnZ: the same partition function by the row-to-row transfer matrix
  (an independent exact method, L <= 12).
* brute_force: full enumeration of the 2^N states of a small lattice with any
  couplings (2D L <= 4, 3D L = 2), giving the exact density of states.
* onsager_minus_beta_f: Onsager's infinite-lattice free energy per spin.

The Hamiltonian is Eq. (Hamiltonian) with k_B = 1 and K = beta J.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

try:
    import mpmath as _mp
except ImportError:  # the GPU host has no mpmath; only the CPU pins need it
    _mp = None


def kaufman_lnZ(L: int, beta: float, dps: int = 50) -> float:
    if _mp is None:
        raise RuntimeError("mpmath is required for kaufman_lnZ")
    mp = _mp.mp
    with _mp.workdps(dps):
        K = _mp.mpf(beta)
        if K == 0:
            return float(L * L * _mp.log(2))
        N = L * L
        c2, s2 = _mp.cosh(2 * K), _mp.sinh(2 * K)
        base = c2 * c2 / s2  # cosh 2K coth 2K

        def gamma(k):
            if k == 0:
                return 2 * K + _mp.log(_mp.tanh(K))
            return _mp.acosh(base - _mp.cos(_mp.pi * k / L))

        odd = [gamma(2 * r + 1) for r in range(L)]
        even = [gamma(2 * r) for r in range(L)]
        Z1 = _mp.fprod(2 * _mp.cosh(L * g / 2) for g in odd)
        Z2 = _mp.fprod(2 * _mp.sinh(L * g / 2) for g in odd)
        Z3 = _mp.fprod(2 * _mp.cosh(L * g / 2) for g in even)
        Z4 = _mp.fprod(2 * _mp.sinh(L * g / 2) for g in even)
        Z = (Z1 + Z2 + Z3 + Z4) / 2 * (2 * s2) ** (N // 2)
        del mp
        return float(_mp.log(Z))


def transfer_lnZ(L: int, beta: float) -> float:
    """ln Z of the L x L periodic ferromagnet as ln Tr(T^L), T the 2^L x 2^L row transfer matrix."""
    n = 1 << L
    states = np.array([[1 - 2 * ((c >> x) & 1) for x in range(L)] for c in range(n)], np.float64)
    row_e = -(states * np.roll(states, -1, axis=1)).sum(axis=1)      # bonds inside a row
    inter = -(states @ states.T)                                        # bonds between rows
    # T[a, b] = exp(-beta (E_row(a) + E_between(a, b))); scale by the largest exponent
    expo = -beta * (row_e[:, None] + inter)
    shift = expo.max()
    T = np.exp(expo - shift)
    # ln Tr(T^L) via eigenvalues of the symmetric form D^1/2 ... use a stable power
    # product with rescaling (exact up to float64 rounding).
    M = np.eye(n)
    logscale = 0.0
    for _ in range(L):
        M = M @ T
        m = np.abs(M).max()
        M /= m
        logscale += math.log(m)
    return float(math.log(np.trace(M)) + logscale + L * shift)


def _neighbours(d: int, L: int):
    N = L ** d
    idx = np.arange(N)
    coords = [(idx // L ** a) % L for a in range(d)]
    nbs = []
    for a in range(d):
        c = coords[a]
        nbs.append(np.where(c == L - 1, idx - (L - 1) * L ** a, idx + L ** a))
    return nbs


def brute_force(d: int, L: int, J=None):
    """Exact density of states {E: g(E)} and magnetisation moments by enumeration."""
    N = L ** d
    if N > 24:
        raise ValueError("brute force limited to N <= 24 sites")
    if J is None:
        J = np.ones(d * N, np.int64)
    J = np.asarray(J, np.int64)
    nbs = _neighbours(d, L)
    codes = np.arange(1 << N, dtype=np.int64)
    sig = 1 - 2 * ((codes[:, None] >> np.arange(N)) & 1)                # [2^N, N]
    E = np.zeros(1 << N, np.int64)
    for a in range(d):
        E -= (sig * sig[:, nbs[a]] * J[a * N:(a + 1) * N]).sum(axis=1)
    M = sig.sum(axis=1)
    return E, M


def exact_thermo(E: np.ndarray, M: np.ndarray, beta: float, N: int):
    """ln Z, <E>, <E^2>, <|M|>, <M^2> from enumerated energies (float64, log-shifted)."""
    x = -beta * E.astype(np.float64)
    xm = x.max()
    w = np.exp(x - xm)
    Z = w.sum()
    lnZ = math.log(Z) + xm
    e1 = (w * E).sum() / Z
    e2 = (w * E.astype(np.float64) ** 2).sum() / Z
    am = (w * np.abs(M)).sum() / Z
    m2 = (w * M.astype(np.float64) ** 2).sum() / Z
    return {"lnZ": lnZ, "E": e1, "E2": e2, "absM": am, "M2": m2}


def onsager_minus_beta_f(beta: float) -> float:
    """-beta f per spin of the infinite square-lattice ferromagnet (Onsager 1944)."""
    from scipy import integrate
    K = beta
    c, s = math.cosh(2 * K), math.sinh(2 * K)

    def inner(t1):
        return integrate.quad(lambda t2: math.log(c * c - s * (math.cos(t1) + math.cos(t2))),
                              0, math.pi, limit=200)[0]

    val = integrate.quad(inner, 0, math.pi, limit=200)[0]
    return math.log(2) + val / (2 * math.pi ** 2)


def mattis_gauge(d, L, J, gauge):
    """Couplings J'_{s,s+e} = g_s J g_{s+e} of the gauge g (+-1 per site)."""
    N = L ** d
    nbs = _neighbours(d, L)
    g = np.asarray(gauge, np.int64)
    Jp = np.asarray(J, np.int64).copy()
    for a in range(d):
        Jp[a * N:(a + 1) * N] = g * Jp[a * N:(a + 1) * N] * g[nbs[a]]
    return Jp.astype(np.int8)
