"""Seeded synthetic inputs shared by the FP64 oracle and the GPU path.

This module generates *inputs only*: covariance matrices of pure Gaussian
states made of single-mode squeezed vacua sent through a passive linear-optical
network, the paired-form matrix of the same state, photon-number patterns and
the uniform draws consumed by conditional sampling.  It contains none of the
arithmetic of the state-to-MPS method itself, so that both the oracle and the
GPU path can depend on it without sharing any method code.

Conventions (the paper fixes the quadratures, Sec. II A; the workload shapes
stand in for the lossy-experiment data of Sec. III, which is not available):

* a_j = (x_j + i p_j)/sqrt(2); covariance Gamma = (1/2)<{dR, dR}> in the
  ordering R = (x_1..x_N, p_1..p_N); the vacuum has Gamma = I/2.
* an x-squeezed input of strength r has Gamma = diag(e^{-2r}, e^{2r})/2 and
  paired-form coefficient -tanh(r).
* a passive unitary U maps a -> U a; on the quadratures it acts as
  S_U = [[Re U, -Im U], [Im U, Re U]].
* brick-wall networks: layer l couples modes (2k, 2k+1) for even l and
  (2k+1, 2k+2) for odd l (0-based), each with the beamsplitter
  [[cos t, -e^{-i f} sin t], [e^{i f} sin t, cos t]], t ~ U(0, pi/2),
  f ~ U(0, 2 pi).
* Haar unitaries: complex Ginibre matrix, QR, phases of R's diagonal divided
  out (Mezzadri, Notices AMS 54, 2007).
* all draws come from one numpy Philox stream per seed, in the order:
  squeezing strengths, then gates layer by layer (theta, phi per gate).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Workload", "haar_unitary", "brickwall_unitary", "squeezed_state",
    "config", "CONFIGS", "uniforms", "random_patterns", "rng", "lossy",
]


def rng(seed: int) -> np.random.Generator:
    """Counter-based (Philox) generator: identical streams on x86 and Arm."""
    return np.random.Generator(np.random.Philox(int(seed)))


def haar_unitary(n: int, g: np.random.Generator) -> np.ndarray:
    z = (g.standard_normal((n, n)) + 1j * g.standard_normal((n, n))) / math.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diagonal(r)
    return q * (d / np.abs(d))[None, :]


def brickwall_unitary(n: int, depth: int, g: np.random.Generator) -> np.ndarray:
    u = np.eye(n, dtype=np.complex128)
    for layer in range(depth):
        start = layer % 2
        for j in range(start, n - 1, 2):
            t = g.uniform(0.0, math.pi / 2)
            f = g.uniform(0.0, 2 * math.pi)
            c, s = math.cos(t), math.sin(t)
            bs = np.array([[c, -np.exp(-1j * f) * s], [np.exp(1j * f) * s, c]])
            u[j:j + 2, :] = bs @ u[j:j + 2, :]
    return u


@dataclass
class Workload:
    """One synthetic pure Gaussian state plus the MPS parameters to build."""
    name: str
    N: int
    gamma: np.ndarray          # (2N, 2N) float64, xxpp
    Q: np.ndarray              # (N, N) complex128 paired-form matrix
    r: np.ndarray              # squeezing strengths
    U: np.ndarray              # passive unitary
    d: int
    chi: int
    eps: float = 1e-12
    freeze: float = 1e-13     # lambda2_freeze (the D* tolerance of Sec. II A)
    seed: int = 0
    meta: dict = field(default_factory=dict)


def squeezed_state(r: np.ndarray, U: np.ndarray):
    """Covariance and paired-form matrix of x-squeezed vacua r through U."""
    r = np.asarray(r, dtype=np.float64)
    n = r.size
    g_in = 0.5 * np.diag(np.concatenate([np.exp(-2 * r), np.exp(2 * r)]))
    s_u = np.block([[U.real, -U.imag], [U.imag, U.real]])
    gamma = s_u @ g_in @ s_u.T
    gamma = 0.5 * (gamma + gamma.T)
    q = U @ np.diag(-np.tanh(r)) @ U.T
    q = 0.5 * (q + q.T)
    return gamma, q


def _make(name, N, rlo, rhi, depth, d, chi, seed, eps=1e-12, haar=False, freeze=1e-13):
    g = rng(seed)
    r = g.uniform(rlo, rhi, size=N)
    U = haar_unitary(N, g) if haar else brickwall_unitary(N, depth, g)
    gamma, q = squeezed_state(r, U)
    return Workload(name=name, N=N, gamma=gamma, Q=q, r=r, U=U, d=d, chi=chi,
                    eps=eps, freeze=freeze, seed=seed,
                    meta={"depth": depth, "r_range": [rlo, rhi], "haar": haar})


#: Workload recipes.  Seeds are 20251210 + index.
CONFIGS = {
    # 8 modes, squeezed vacua r~U(0.3,0.8) through an 8x8 Haar unitary, d=8, chi=64
    "pr1_n8": dict(N=8, rlo=0.3, rhi=0.8, depth=0, d=8, chi=64, seed=20251210, haar=True,
                   eps=0.0),
    # 144 modes, r~U(0.1,0.4), brick-wall depth 12, d=6, chi=256
    # (eps = 1e-12 and freeze = 1e-9: chi binds at the central bonds; modes with
    # Lambda^2 <= 1e-9 are frozen)
    "n144_d6_chi256": dict(N=144, rlo=0.1, rhi=0.4, depth=12, d=6, chi=256, seed=20251211,
                           eps=1e-12, freeze=1e-9),
    # 1024 modes, r~U(0.05,0.25), brick-wall depth 32, d=4, chi=512
    "n1024_d4_chi512": dict(N=1024, rlo=0.05, rhi=0.25, depth=32, d=4, chi=512, seed=20251213,
                            eps=1e-12, freeze=1e-9),
}


def config(name: str, **over) -> Workload:
    """Build a named workload; keyword overrides (N, chi, d, depth, ...) allowed."""
    kw = dict(CONFIGS[name])
    kw.update(over)
    return _make(name, **kw)


def small(N: int, seed: int, d: int = 4, chi: int = 32, depth: int = 4,
          rlo: float = 0.1, rhi: float = 0.5, eps: float = 1e-12,
          haar: bool = False) -> Workload:
    """Small brick-wall (or Haar) state for parity tests."""
    return _make(f"small_n{N}_s{seed}", N, rlo, rhi, depth, d, chi, seed,
                 eps=eps, haar=haar)


def batch(count: int, seed: int = 20251212):
    """Many independent states of uneven size: N~U{16..144}, r~U(0.1,0.5),
    depth N/8, d=6, chi in {32,64,128,256} (eps 1e-12, freeze 1e-9)."""
    g = rng(seed)
    out = []
    for i in range(count):
        N = int(g.integers(16, 145))
        chi = int(g.choice([32, 64, 128, 256]))
        out.append(_make(f"batch{i}", N, 0.1, 0.5, max(1, N // 8), 6, chi,
                         seed * 1000 + i, eps=1e-12, freeze=1e-9))
    return out


def serving(count: int, rate_hz: float, seed: int = 20251214, n_range=(32, 512),
            chis=(64, 128, 256, 512), ds=(4, 6), s_range=(1000, 100000)):
    """A stream of build + sampling requests: Poisson arrivals at rate_hz;
    N log-uniform in n_range, r~U(0.05,0.4), brick-wall depth N/16, d from
    ds, chi from chis, sample count uniform in s_range.  Returns a list of
    (arrival time in s, Workload, samples); the Workload's Gamma is built when
    the item is generated."""
    g = rng(seed)
    t = 0.0
    out = []
    for i in range(count):
        t += float(g.exponential(1.0 / rate_hz))
        N = int(round(math.exp(g.uniform(math.log(n_range[0]), math.log(n_range[1])))))
        d = int(g.choice(ds))
        chi = int(g.choice(chis))
        S = int(g.integers(s_range[0], s_range[1] + 1))
        w = _make(f"req{i}", N, 0.05, 0.4, max(1, N // 16), d, chi, seed * 1000 + i,
                  eps=1e-12, freeze=1e-9)
        out.append((t, w, S))
    return out


def lossy(N: int, seed: int, eta: float, depth: int = 4, rlo: float = 0.3, rhi: float = 0.8,
          haar: bool = False):
    """Mixed covariance of a lossy experiment: the pure brick-wall (or Haar)
    state of ``small`` after uniform loss of transmission eta on every mode,
    Gamma_th = eta Gamma + (1 - eta) I / 2 (loss mixes each mode with
    vacuum, Gamma = I/2).  Returns (Gamma_th, the pure Workload)."""
    w = _make(f"lossy_n{N}_s{seed}", N, rlo, rhi, depth, 4, 32, seed, haar=haar)
    return eta * w.gamma + (1.0 - eta) * 0.5 * np.eye(2 * N), w


def uniforms(S: int, N: int, seed: int) -> np.ndarray:
    """(S, N) float64 uniforms in [0,1) for conditional sampling."""
    return rng(seed).random((S, N))


def random_patterns(P: int, N: int, d: int, seed: int, max_total=None,
                    even=True) -> np.ndarray:
    """(P, N) uint8 photon patterns with entries < d (low occupations
    favoured); optionally even total photon number."""
    g = rng(seed)
    pats = np.zeros((P, N), dtype=np.uint8)
    for i in range(P):
        # geometric-like low occupations
        x = np.minimum(g.geometric(0.75, size=N) - 1, d - 1)
        if max_total is not None:
            while x.sum() > max_total:
                j = int(np.argmax(x))
                x[j] -= 1
        if even and x.sum() % 2 == 1:
            nz = np.nonzero(x)[0]
            if nz.size:
                x[nz[0]] -= 1
        pats[i] = x
    return pats
