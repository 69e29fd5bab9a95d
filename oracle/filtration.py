"""Mixed -> pure decomposition of a Gaussian covariance matrix (FP64, numpy).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. III, Eq. (decompose): an experimentally produced mixed covariance
Gamma_th is split as Gamma_th = Gamma_p + W with Gamma_p the covariance of a
pure state and W >= 0 classical noise; the best split has the smallest
tr(Gamma_p).  App. C, Eq. (loss): with Gamma_p = S S^T / 2, S symplectic,
minimise L(S) = -lambda_min(Gamma_th - S S^T / 2) by Riemannian gradient
descent on Sp(2N), starting from S = I and stopping once L <= eps:

* the directional derivative along X in sp(2N) at S is
  dL = (1/2) <v0| S (X + X^T) S^T |v0>,  v0 the lowest eigenvector of W;
* the gradient G is the unit X in sp(2N) that maximises it (Eq. (gradient));
* the retraction is S <- S exp(-alpha G).

Readings where the appendix is silent:
* the norm on sp(2N) is the Frobenius norm (the appendix names "the two-form
  norm" without defining it); sp(2N) = {Omega H : H = H^T}, so with
  u = S^T v0 the maximiser is G = Omega H / ||H||_F, H = sym(Omega^T u u^T);
* the step alpha is a fixed step length along the unit gradient;
* when the lowest eigenvalue is degenerate the eigenvector numpy's eigh
  returns first is used (the appendix notes the gradient is then only
  approximate);
* the loop also stops after max_iter steps.
Every step is taken in the appendix's order with library primitives (eigh,
expm, matmul); nothing is fused.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
from scipy.linalg import expm

from .gaussian import omega


@dataclass
class Filtered:
    S: np.ndarray          # symplectic, Gamma_p = S S^T / 2
    iters: int             # gradient steps taken
    loss: float            # L(S) at the end (<= eps when converged)
    converged: bool

    @property
    def gamma_p(self) -> np.ndarray:
        return 0.5 * self.S @ self.S.T

    @property
    def n_eff(self) -> float:
        """N_eff = tr(Gamma_p)/2 - N/2 (reading A1: the vacuum is Gamma = I/2)."""
        n = self.S.shape[0] // 2
        return float(0.5 * np.trace(self.gamma_p) - 0.5 * n)


def loss_and_vector(gamma_th: np.ndarray, S: np.ndarray):
    """L(S) = -lambda_min(W), W = Gamma_th - S S^T / 2, and the eigenvector."""
    W = gamma_th - 0.5 * S @ S.T
    ev, V = np.linalg.eigh(W)
    return -float(ev[0]), V[:, 0]


def directional_derivative(S: np.ndarray, v0: np.ndarray, X: np.ndarray) -> float:
    """dL along X at S, first-order perturbation of the lowest eigenvalue."""
    return float(0.5 * v0 @ S @ (X + X.T) @ S.T @ v0)


def gradient(S: np.ndarray, v0: np.ndarray) -> np.ndarray:
    """The unit X in sp(2N) (Frobenius norm) maximising dL: with X = Omega H,
    dL = <H, sym(Omega^T u u^T)>_F for u = S^T v0."""
    n = S.shape[0] // 2
    Om = omega(n)
    u = S.T @ v0
    H = Om.T @ np.outer(u, u)
    H = 0.5 * (H + H.T)
    return Om @ H / np.linalg.norm(H)


def filtration(gamma_th: np.ndarray, alpha: float, eps: float = 0.0, max_iter: int = 100000,
               S0: np.ndarray | None = None) -> Filtered:
    """Gradient descent of App. C from S0 (identity by default)."""
    n = gamma_th.shape[0]
    S = np.eye(n) if S0 is None else np.array(S0, dtype=np.float64)
    for k in range(max_iter):
        L, v0 = loss_and_vector(gamma_th, S)
        if L <= eps:
            return Filtered(S=S, iters=k, loss=L, converged=True)
        S = S @ expm(-alpha * gradient(S, v0))
    L, _ = loss_and_vector(gamma_th, S)
    return Filtered(S=S, iters=max_iter, loss=L, converged=L <= eps)
