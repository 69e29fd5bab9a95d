"""Whole-state build, normalisation, amplitudes, sampling and fidelity.

Build: GSVD chain (Sec. II B), kept bases per bond (Sec. II C), PCO local
tensors (Sec. II C, App. B); the bond state |I_m> = prod exp(l^dag r^dag)|0>
(Eq. (bond)) contracts l_m and r_m Fock states index by index, so the MPS is
the chain of tensors A^m[alpha, p, beta] with shared bond bases (Eq. (GMPS)).

Readings where the paper is silent (it defers sampling to standard MPS
routines and normalises only "up to an unimportant factor"):
* normalisation and phase: A^1 is divided by sqrt(<psi|psi>) computed with
  right environments R_m = sum_p A^m[p] R_{m+1} A^m[p]^dag, R_{N+1} = 1, and
  multiplied by the phase that makes the all-vacuum amplitude real positive;
* sampling: exact sequential conditional sampling of the truncated MPS.
  Given uniforms u[s, m]: v = [1]; for m = 1..N: w_p = v A^m[p],
  q_p = max(0, Re w_p R_{m+1} w_p^dag), Z = sum q, C = prefix sums,
  p* = min{p : u Z < C_p} (if none, the largest p with q_p > 0),
  v = w_{p*}/sqrt(q_{p*}).  A draw with |u Z - C_p| <= 1e-12 Z for some p is
  flagged as a boundary case.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import gaussian
from .basis import Basis, kept_basis
from .pco import local_tensor


@dataclass
class MPS:
    tensors: list                 # A^m, shape (D_{m-1}, d, D_m), complex128
    bases: list                   # Basis of bonds 0..N (bond 0 and N: vacuum)
    cuts: list = field(default_factory=list)
    eps: list = field(default_factory=list)   # eps_m for bonds 1..N-1

    @property
    def N(self):
        return len(self.tensors)

    @property
    def bond_dims(self):
        return [1] + [t.shape[2] for t in self.tensors]

    @property
    def n_e(self):
        return [b.ne for b in self.bases[1:-1]]


def vacuum_basis() -> Basis:
    return Basis(occ=np.zeros((1, 0), dtype=np.int64), E=np.zeros(1), eps=0.0, index={(): 0})


def build_mps(gamma: np.ndarray, d: int, chi: int, eps: float = 0.0,
              lambda2_freeze: float = 1e-13, sites=None, route=None) -> MPS:
    """Unnormalised MPS of the pure Gaussian state with covariance gamma.
    ``sites`` restricts the PCO build to a subset of site indices (the others
    are left as None), for bounded-cost checks on large states; ``route``
    picks the Williamson construction of the GSVD chain (default: Cholesky)."""
    cuts = gaussian.gsvd_chain(gamma, lambda2_freeze=lambda2_freeze, route=route)
    N = len(cuts)
    bases = [vacuum_basis()]
    epss = []
    for m in range(N - 1):
        b = kept_basis(cuts[m].lam2, chi, eps)
        bases.append(b)
        epss.append(b.eps)
    bases.append(vacuum_basis())
    tensors = []
    for m in range(N):
        if sites is not None and m not in sites:
            tensors.append(None)
            continue
        tensors.append(local_tensor(cuts[m].Q, bases[m], bases[m + 1], d, cuts[m].c))
    return MPS(tensors=tensors, bases=bases, cuts=cuts, eps=epss)


def build_from_q(Q: np.ndarray, d: int, chi: int, eps: float = 0.0,
                 lambda2_freeze: float = 1e-13) -> MPS:
    """A-matrix / paired-form input: convert to the covariance first."""
    return build_mps(gaussian.gamma_from_q(Q), d, chi, eps, lambda2_freeze)


def environments(tensors) -> list:
    """R[m] for m = 0..N: R[N] = [[1]], R[m] = sum_p A^m[p] R[m+1] A^m[p]^dag;
    R[0] is the squared norm."""
    N = len(tensors)
    R = [None] * (N + 1)
    R[N] = np.ones((1, 1), dtype=np.complex128)
    for m in range(N - 1, -1, -1):
        A = tensors[m]
        acc = np.zeros((A.shape[0], A.shape[0]), dtype=np.complex128)
        for p in range(A.shape[1]):
            acc += A[:, p, :] @ R[m + 1] @ A[:, p, :].conj().T
        R[m] = acc
    return R


def contract(tensors, pattern) -> complex:
    v = np.ones(1, dtype=np.complex128)
    for m, A in enumerate(tensors):
        p = int(pattern[m])
        if p >= A.shape[1]:
            return 0j
        v = v @ A[:, p, :]
    return complex(v[0])


def normalise(tensors) -> list:
    """Divide A^1 by the norm and fix the global phase (vacuum amplitude > 0)."""
    R = environments(tensors)
    nrm = np.sqrt(R[0][0, 0].real)
    out = [t.copy() for t in tensors]
    out[0] = out[0] / nrm
    a0 = contract(out, np.zeros(len(out), dtype=np.int64))
    if abs(a0) > 0:
        out[0] = out[0] * (np.conj(a0) / abs(a0))
    return out


def amplitudes(tensors, patterns) -> np.ndarray:
    """<n_1..n_N|psi> for each pattern (rows), by the matrix chain; patterns
    with any n_i >= d give 0."""
    return np.array([contract(tensors, p) for p in patterns], dtype=np.complex128)


def sample(tensors, u: np.ndarray, R=None):
    """Conditional sampling with given uniforms u (S, N).  Returns
    (patterns uint8 (S, N), boundary flags bool (S,))."""
    if R is None:
        R = environments(tensors)
    S, N = u.shape
    v = np.ones((S, 1), dtype=np.complex128)
    out = np.zeros((S, N), dtype=np.uint8)
    flag = np.zeros(S, dtype=bool)
    rows = np.arange(S)
    for m in range(N):
        A = tensors[m]
        d = A.shape[1]
        Dl, Dr = A.shape[0], A.shape[2]
        W = (v @ A.reshape(Dl, d * Dr)).reshape(S, d, Dr)      # w_p = v A^m[p]
        Y = (W.reshape(S * d, Dr) @ R[m + 1]).reshape(S, d, Dr)
        q = np.maximum(0.0, np.real(np.sum(Y * W.conj(), axis=2)))
        Z = q.sum(axis=1)
        Cp = np.cumsum(q, axis=1)
        t = u[:, m] * Z
        hit = t[:, None] < Cp
        pstar = np.where(hit.any(axis=1), np.argmax(hit, axis=1),
                         d - 1 - np.argmax((q > 0)[:, ::-1], axis=1))
        flag |= np.any(np.abs(t[:, None] - Cp) <= 1e-12 * Z[:, None], axis=1)
        out[:, m] = pstar
        w = W[rows, pstar, :]
        v = w / np.sqrt(q[rows, pstar])[:, None]
    return out, flag


def overlap(ta, tb) -> complex:
    """<a|b> by the transfer-matrix sweep E <- sum_p A_a[p]^dag E A_b[p]."""
    E = np.ones((1, 1), dtype=np.complex128)
    for A, B in zip(ta, tb):
        acc = np.zeros((A.shape[2], B.shape[2]), dtype=np.complex128)
        for p in range(min(A.shape[1], B.shape[1])):
            acc += A[:, p, :].conj().T @ E @ B[:, p, :]
        E = acc
    return complex(E[0, 0])


def fidelity(ta, tb) -> float:
    """|<a|b>|^2 / (<a|a><b|b>), gauge and phase invariant."""
    ab = overlap(ta, tb)
    return float(abs(ab) ** 2 / (overlap(ta, ta).real * overlap(tb, tb).real))


def left_environments(tensors) -> list:
    """L[m] for m = 0..N: L[0] = [[1]], L[m+1] = sum_p A^m[p]^dag L[m] A^m[p]."""
    L = [np.ones((1, 1), dtype=np.complex128)]
    for A in tensors:
        acc = np.zeros((A.shape[2], A.shape[2]), dtype=np.complex128)
        for p in range(A.shape[1]):
            acc += A[:, p, :].conj().T @ L[-1] @ A[:, p, :]
        L.append(acc)
    return L


def site_marginals(tensors) -> np.ndarray:
    """P(n_m = p) for every site (N, d): L[m] and R[m+1] around one site."""
    L = left_environments(tensors)
    R = environments(tensors)
    nrm = R[0][0, 0].real
    out = []
    for m, A in enumerate(tensors):
        row = []
        for p in range(A.shape[1]):
            row.append(np.real(np.trace(L[m] @ A[:, p, :] @ R[m + 1] @ A[:, p, :].conj().T)))
        out.append(np.array(row) / nrm)
    return np.array(out)
