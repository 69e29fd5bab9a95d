"""Kept virtual subspace and the index maps of the PCO mapping (FP64, numpy).

Sec. II C "The kept subspace and projection" (entanglement Hamiltonian
Eq. (HE), partition function Eq. (Z), the D(eps) rule), Sec. III A (truncation
error eps_m), App. B Alg. 1 (vector set of one mode) and Alg. 3 (composition
of two vector sets).

Readings where the paper is silent:
* ties in the entanglement energy are resolved by grouping energies within
  1e-12 * max(1, E) of the first member of a group and ordering each group
  lexicographically by occupation vector (smaller first);
* the kept dimension is D_m = min(chi, D(eps)); eps = 0 means chi alone.
"""
from __future__ import annotations

import heapq
import math
from dataclasses import dataclass

import numpy as np

TIE_TOL = 1e-12


@dataclass
class Basis:
    occ: np.ndarray       # (D, n_e) int64 occupation vectors, index 0 = vacuum
    E: np.ndarray         # (D,) entanglement energies
    eps: float            # discarded weight 1 - (1/Z) sum_kept e^{-E}
    index: dict           # occupation tuple -> basis index

    @property
    def D(self) -> int:
        return self.occ.shape[0]

    @property
    def ne(self) -> int:
        return self.occ.shape[1]


def weights(lam2: np.ndarray) -> np.ndarray:
    """Single-quantum entanglement energies w_q = -2 log Lambda_q, Eq. (HE)."""
    return -np.log(np.asarray(lam2, dtype=np.float64))


def tie_order(E: np.ndarray, occ: np.ndarray) -> np.ndarray:
    """Order by E with the tie reading above; returns a permutation."""
    keys = sorted(range(len(E)), key=lambda i: (E[i], tuple(occ[i])))
    out = []
    i = 0
    while i < len(keys):
        e0 = E[keys[i]]
        j = i
        while j < len(keys) and E[keys[j]] - e0 <= TIE_TOL * max(1.0, abs(e0)):
            j += 1
        grp = sorted(keys[i:j], key=lambda k: tuple(occ[k]))
        out.extend(grp)
        i = j
    return np.asarray(out, dtype=np.int64)


def kept_basis(lam2: np.ndarray, chi: int, eps: float = 0.0,
               max_states: int | None = None) -> Basis:
    """Sec. II C steps 1-3: enumerate virtual Fock states |n_1..n_ne>, compute
    E = sum_q n_q w_q, sort ascending and keep the first D = min(chi, D(eps)).
    Enumeration is best-first from the vacuum with a binary heap (each state
    is reached from every predecessor; a set removes duplicates)."""
    lam2 = np.asarray(lam2, dtype=np.float64)
    ne = lam2.size
    w = weights(lam2)
    logZ = -np.sum(np.log1p(-lam2))        # Z = prod 1/(1 - L^2), Eq. (Z)
    if ne == 0:
        occ = np.zeros((1, 0), dtype=np.int64)
        return Basis(occ=occ, E=np.zeros(1), eps=0.0, index={(): 0})
    start = (0,) * ne
    heap = [(0.0, start)]
    seen = {start}
    popped_E, popped = [], []
    acc = 0.0
    target = (1.0 - eps) if eps > 0 else None
    limit = chi if max_states is None else min(chi, max_states)
    Dcut = None
    while heap:
        e, s = heapq.heappop(heap)
        if Dcut is not None and e - popped_E[Dcut - 1] > TIE_TOL * max(1.0, abs(popped_E[Dcut - 1])) * 4:
            break
        popped_E.append(e)
        popped.append(s)
        if Dcut is None:
            acc += math.exp(-e - logZ)
            if len(popped) >= limit or (target is not None and acc >= target):
                Dcut = len(popped)
        for q in range(ne):
            t = list(s)
            t[q] += 1
            t = tuple(t)
            if t not in seen:
                seen.add(t)
                et = float(np.dot(np.asarray(t, dtype=np.float64), w))
                heapq.heappush(heap, (et, t))
    occ = np.asarray(popped, dtype=np.int64).reshape(-1, ne)
    E = occ.astype(np.float64) @ w
    perm = tie_order(E, occ)
    D = Dcut if Dcut is not None else len(popped)
    occ, E = occ[perm][:D], E[perm][:D]
    kept = float(np.sum(np.exp(-E - logZ)))
    eps_m = 1.0 - kept                       # Sec. III A, eps_m
    index = {tuple(int(x) for x in row): i for i, row in enumerate(occ)}
    return Basis(occ=occ, E=E, eps=eps_m, index=index)


def single_mode_basis(d: int) -> Basis:
    """Physical Fock basis {|0>..|d-1>} of a_m as a one-mode space."""
    occ = np.arange(d, dtype=np.int64).reshape(d, 1)
    return Basis(occ=occ, E=np.arange(d, dtype=np.float64), eps=0.0,
                 index={(i,): i for i in range(d)})


@dataclass
class VectorSet:
    vin: np.ndarray
    vout: np.ndarray
    vord: np.ndarray


def vector_set(b: Basis, q: int) -> VectorSet:
    """App. B Alg. 1: for beta = D-1 down to 0 and kappa = 1..n_{beta,q}, record
    (alpha, beta, kappa) with |v_alpha> the state with kappa fewer quanta in
    mode q, so that |v_beta> = sqrt(n_alpha,q!/n_beta,q!) (d_q^dag)^kappa |v_alpha>."""
    vin, vout, vord = [], [], []
    for beta in range(b.D - 1, -1, -1):
        n = b.occ[beta]
        for kappa in range(1, int(n[q]) + 1):
            s = list(int(x) for x in n)
            s[q] -= kappa
            vin.append(b.index[tuple(s)])
            vout.append(beta)
            vord.append(kappa)
    return VectorSet(np.asarray(vin, dtype=np.int64), np.asarray(vout, dtype=np.int64),
                     np.asarray(vord, dtype=np.int64))


def compose(vq: VectorSet, vqp: VectorSet) -> VectorSet:
    """App. B Alg. 3: all pairs (l, r) with (vout_q[l], vord_q[l]) =
    (vin_q'[r], vord_q'[r]), sorted by r; record (vin_q[l], vout_q'[r], vord_q'[r]).
    The composite maps a state to the one with kappa more quanta in both q and q'."""
    lut = {}
    for l in range(vq.vin.size):
        lut[(int(vq.vout[l]), int(vq.vord[l]))] = l
    vin, vout, vord = [], [], []
    for r in range(vqp.vin.size):
        key = (int(vqp.vin[r]), int(vqp.vord[r]))
        if key in lut:
            l = lut[key]
            vin.append(int(vq.vin[l]))
            vout.append(int(vqp.vout[r]))
            vord.append(int(vqp.vord[r]))
    return VectorSet(np.asarray(vin, dtype=np.int64), np.asarray(vout, dtype=np.int64),
                     np.asarray(vord, dtype=np.int64))
