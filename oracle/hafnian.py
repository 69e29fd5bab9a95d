"""Brute-force hafnian amplitudes: the exact Fock amplitudes of a pure
Gaussian state that the MPS approximates (Sec. I; the hafnian formula of
Hamilton et al. 2017 cited there).  For |psi> proportional to
exp(1/2 a^dag Q a^dag)|0> (Eq. (paired-form)), expanding the exponential gives

    <n|psi> / <0|psi> = haf(Q_n) / sqrt(prod_i n_i!),
    |<0|psi>|^2 = det(1 - Q Q^*)^{1/2},

where Q_n repeats row/column i n_i times.  Only for tiny instances."""
from __future__ import annotations

import math

import numpy as np


def hafnian(A: np.ndarray) -> complex:
    """Sum over perfect matchings, by recursion on the lowest free index with
    memoisation over subsets (exact up to rounding)."""
    n = A.shape[0]
    if n == 0:
        return 1.0 + 0j
    if n % 2:
        return 0j
    memo = {0: 1.0 + 0j}

    def f(mask):
        if mask in memo:
            return memo[mask]
        i = (mask & -mask).bit_length() - 1
        rest = mask & ~(1 << i)
        tot = 0j
        m = rest
        while m:
            j = (m & -m).bit_length() - 1
            tot += A[i, j] * f(rest & ~(1 << j))
            m &= m - 1
        memo[mask] = tot
        return tot

    return f((1 << n) - 1)


def expand(Q: np.ndarray, n) -> np.ndarray:
    idx = np.repeat(np.arange(len(n)), np.asarray(n, dtype=np.int64))
    return Q[np.ix_(idx, idx)]


def relative_amplitude(Q: np.ndarray, n) -> complex:
    """<n|psi>/<0|psi> = haf(Q_n)/sqrt(prod n_i!)."""
    n = np.asarray(n, dtype=np.int64)
    if n.sum() % 2:
        return 0j
    den = math.sqrt(float(np.prod([math.factorial(int(k)) for k in n])))
    return hafnian(expand(Q, n)) / den


def vacuum_amplitude(Q: np.ndarray) -> float:
    """<0|psi> > 0 for the normalised state: det(1 - Q Q^*)^{1/4}."""
    m = np.eye(Q.shape[0]) - Q @ Q.conj()
    return float(np.real(np.linalg.det(m))) ** 0.25


def amplitude(Q: np.ndarray, n) -> complex:
    return vacuum_amplitude(Q) * relative_amplitude(Q, n)


def local_entry(Q: np.ndarray, occ) -> complex:
    """Coefficient of prod_z (d_z^dag)^{k_z}/sqrt(k_z!)|0> in
    exp(1/2 d^dag Q d^dag)|0>: haf(Q_k)/sqrt(prod k!).  This is the plain
    definition of an unscaled PCO tensor entry, Eq. (Am_apb)."""
    return relative_amplitude(Q, occ)
