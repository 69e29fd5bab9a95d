"""Projected-creation-operator (PCO) construction of one local tensor.

Sec. II C "The core algorithm": the projected state P_V exp(1/2 d^dag Q d^dag)|0>
equals the product over zeta <= zeta' of the PCOs
    PP_{zeta zeta'} = P_V sum_kappa [(1 - delta/2) Q_{zeta zeta'} d^dag_zeta d^dag_zeta']^kappa / kappa!
applied to the vacuum, by the closure identity P d^dag = P d^dag P.
App. B: cross-type PCOs (Alg. 2), intra-type PCOs through composed vector
sets (Alg. 3, Alg. 4), duplicate-type PCOs (Alg. 5); the physical-mode PCOs
r^dag a^dag, a^dag a^dag, a^dag l^dag are applied first, then the virtual-only
PCOs act on every physical sector (the sectors are independent).

Each PCO is applied out of place, which is the definition of the operator
product; the paper's in-place loop with reverse-ordered vector sets gives the
same coefficients (every source index precedes every target index it feeds).
Tensor layout: C[alpha, p, beta] over (basis_{m-1}) x (0..d-1) x (basis_m).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import gammaln

from .basis import Basis, VectorSet, compose, single_mode_basis, vector_set


def _log_sqrt_fact_ratio(n_hi: np.ndarray, k: int) -> np.ndarray:
    """log sqrt(n_hi! / (n_hi - k)!)"""
    n_hi = np.asarray(n_hi, dtype=np.float64)
    return 0.5 * (gammaln(n_hi + 1.0) - gammaln(n_hi - k + 1.0))


def _gk_over_kfact(g: complex, k: int):
    """(log |g^k / k!|, phase of g^k); -inf when g = 0."""
    if g == 0:
        return -np.inf, 1.0
    return k * math.log(abs(g)) - math.lgamma(k + 1.0), np.exp(1j * k * np.angle(g))


def apply_cross(C, ax1, vs1: VectorSet, occ1, ax2, vs2: VectorSet, occ2, g):
    """Alg. 2 generalised to any two distinct index spaces of C: for every
    pair of vector-set entries with equal kappa,
    C[mu, nu] += g^kappa/kappa! sqrt(n_mu! n_nu! / (n_sigma! n_gamma!)) C[sigma, gamma]."""
    Cn = C.copy()
    src = np.moveaxis(C, (ax1, ax2), (0, 1))
    dst = np.moveaxis(Cn, (ax1, ax2), (0, 1))
    if vs1.vord.size == 0 or vs2.vord.size == 0:
        return Cn
    kmax = int(min(vs1.vord.max(), vs2.vord.max()))
    for k in range(1, kmax + 1):
        s1, s2 = vs1.vord == k, vs2.vord == k
        if not s1.any() or not s2.any():
            continue
        o1, i1 = vs1.vout[s1], vs1.vin[s1]
        o2, i2 = vs2.vout[s2], vs2.vin[s2]
        lg, ph = _gk_over_kfact(g, k)
        if lg == -np.inf:
            continue
        l1 = _log_sqrt_fact_ratio(occ1[o1], k)
        l2 = _log_sqrt_fact_ratio(occ2[o2], k)
        coef = ph * np.exp(lg + l1[:, None] + l2[None, :])
        blk = src[np.ix_(i1, i2)]
        coef = coef.reshape(coef.shape + (1,) * (blk.ndim - 2))
        dst[np.ix_(o1, o2)] += coef * blk
    return Cn


def apply_intra(C, ax, comp: VectorSet, occ_q, occ_qp, g):
    """Alg. 4: distinct modes q, q' of the same space through the composed
    vector set: C[.., nu] += g^kappa/kappa! sqrt(n_nu,q! n_nu,q'! /
    (n_gamma,q! n_gamma,q'!)) C[.., gamma]."""
    Cn = C.copy()
    src = np.moveaxis(C, ax, 0)
    dst = np.moveaxis(Cn, ax, 0)
    if comp.vord.size == 0:
        return Cn
    for k in range(1, int(comp.vord.max()) + 1):
        s = comp.vord == k
        if not s.any():
            continue
        o, i = comp.vout[s], comp.vin[s]
        lg, ph = _gk_over_kfact(g, k)
        if lg == -np.inf:
            continue
        lc = lg + _log_sqrt_fact_ratio(occ_q[o], k) + _log_sqrt_fact_ratio(occ_qp[o], k)
        coef = ph * np.exp(lc)
        blk = src[i]
        dst[o] += coef.reshape((-1,) + (1,) * (blk.ndim - 1)) * blk
    return Cn


def apply_duplicate(C, ax, vs: VectorSet, occ_q, g):
    """Alg. 5: the same mode twice, PP = P exp[(g/2) d_q^dag d_q^dag]; only even
    kappa: C[.., nu] += (g/2)^(kappa/2)/(kappa/2)! sqrt(n_nu! / n_gamma!) C[.., gamma]."""
    Cn = C.copy()
    src = np.moveaxis(C, ax, 0)
    dst = np.moveaxis(Cn, ax, 0)
    if vs.vord.size == 0:
        return Cn
    for k in range(2, int(vs.vord.max()) + 1, 2):
        s = vs.vord == k
        if not s.any():
            continue
        o, i = vs.vout[s], vs.vin[s]
        j = k // 2
        lg, ph = _gk_over_kfact(g / 2.0, j)
        if lg == -np.inf:
            continue
        coef = ph * np.exp(lg + _log_sqrt_fact_ratio(occ_q[o], k))
        blk = src[i]
        dst[o] += coef.reshape((-1,) + (1,) * (blk.ndim - 1)) * blk
    return Cn


def pco_order(nl: int, nr: int):
    """The fixed PCO order used here: physical-mode PCOs (r_q a, a a, a l_q'),
    then cross (r_q, l_q'), intra left, intra right, duplicate left,
    duplicate right, each lexicographic.  Mode indices refer to
    c_m = (r_1..r_nl, a, l_1..l_nr)."""
    a = nl
    out = [(q, a) for q in range(nl)] + [(a, a)] + [(a, nl + 1 + q) for q in range(nr)]
    out += [(q, nl + 1 + qp) for q in range(nl) for qp in range(nr)]
    out += [(q, qp) for q in range(nl) for qp in range(q + 1, nl)]
    out += [(nl + 1 + q, nl + 1 + qp) for q in range(nr) for qp in range(q + 1, nr)]
    out += [(q, q) for q in range(nl)]
    out += [(nl + 1 + q, nl + 1 + q) for q in range(nr)]
    return out


def local_tensor(Q: np.ndarray, bl: Basis, br: Basis, d: int, c: float = 1.0,
                 order=None) -> np.ndarray:
    """Coefficients of P_V |A^m> on V_m = basis_l x {0..d-1} x basis_r,
    Eq. (Am_apb), multiplied by the scale c.  ``order`` may permute the PCOs
    (the result is order independent, Sec. II C)."""
    nl, nr = bl.ne, br.ne
    assert Q.shape == (nl + 1 + nr, nl + 1 + nr)
    bp = single_mode_basis(d)
    spaces = []   # (axis, basis, local mode index) for each mode of c_m
    spaces += [(0, bl, q) for q in range(nl)]
    spaces += [(1, bp, 0)]
    spaces += [(2, br, q) for q in range(nr)]
    vsets = {}

    def vs(z):
        if z not in vsets:
            ax, b, q = spaces[z]
            vsets[z] = vector_set(b, q)
        return vsets[z]

    C = np.zeros((bl.D, d, br.D), dtype=np.complex128)
    C[0, 0, 0] = 1.0
    for (z1, z2) in (order if order is not None else pco_order(nl, nr)):
        if z1 > z2:
            z1, z2 = z2, z1
        ax1, b1, q1 = spaces[z1]
        ax2, b2, q2 = spaces[z2]
        if z1 == z2:
            C = apply_duplicate(C, ax1, vs(z1), b1.occ[:, q1], Q[z1, z1])
        elif ax1 != ax2:
            C = apply_cross(C, ax1, vs(z1), b1.occ[:, q1], ax2, vs(z2), b2.occ[:, q2],
                            Q[z1, z2])
        else:
            comp = compose(vs(z1), vs(z2))
            C = apply_intra(C, ax1, comp, b1.occ[:, q1], b1.occ[:, q2], Q[z1, z2])
    return c * C
