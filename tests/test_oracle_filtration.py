"""Pins of the oracle's mixed -> pure decomposition (Sec. III Eq. (decompose),
App. C) against closed forms and first-order perturbation theory.  CPU only."""
import math

import numpy as np
import pytest

import workloads as wl
from oracle import filtration as F
from oracle import gaussian as G


def _single_mode(r, eta, phi=0.0):
    """Lossy x-squeezed vacuum, rotated by the phase phi: Gamma_th =
    R diag(a, b) R^T, a = (eta e^{-2r} + 1 - eta)/2, b = (eta e^{2r} + 1 - eta)/2."""
    a = 0.5 * (eta * math.exp(-2 * r) + 1 - eta)
    b = 0.5 * (eta * math.exp(2 * r) + 1 - eta)
    c, s = math.cos(phi), math.sin(phi)
    R = np.array([[c, -s], [s, c]])
    return R @ np.diag([a, b]) @ R.T, a, b, R


@pytest.mark.parametrize("r,eta,phi,alpha", [(0.5, 0.6, 0.0, 0.01), (0.9, 0.3, 0.7, 0.02),
                                             (0.2, 0.8, -1.1, 0.005)])
def test_single_mode_trajectory_closed_form(r, eta, phi, alpha):
    """From S = I the lowest eigenvector of W is the squeezed quadrature R e_x,
    u is parallel to it, and the unit gradient is G = R diag(1, -1) R^T/sqrt 2,
    so S_k = R diag(e^{-k beta}, e^{k beta}) R^T with beta = alpha/sqrt 2; the
    descent stops at the first k with a - e^{-2 k beta}/2 >= -eps."""
    gth, a, b, R = _single_mode(r, eta, phi)
    eps = 1e-12
    beta = alpha / math.sqrt(2)
    k = 0
    while a - 0.5 * math.exp(-2 * k * beta) < -eps:
        k += 1
    res = F.filtration(gth, alpha, eps=eps)
    assert res.converged and res.iters == k
    want = R @ np.diag([math.exp(-k * beta), math.exp(k * beta)]) @ R.T
    assert np.abs(res.S - want).max() < 1e-12
    # the optimum of the trace problem: e^{-2 s*}/2 = a; the descent stops
    # within one step above it
    s_star = -0.5 * math.log(2 * a)
    assert s_star <= k * beta < s_star + beta + 1e-12


def test_product_state_neff_between_optimum_and_one_step():
    """Independent lossy modes: each mode's squeezing ends within one step of
    its optimum s_i* = -ln(2 a_i)/2, so sum sinh^2 s_i* <= N_eff <
    sum sinh^2(s_i* + beta); the result is symplectic and W >= -eps."""
    r = np.array([0.3, 0.6, 0.9, 0.45])
    eta, alpha, eps = 0.5, 0.01, 1e-12
    gpure, _ = wl.squeezed_state(r, np.eye(4, dtype=np.complex128))
    gth = eta * gpure + (1 - eta) * 0.5 * np.eye(8)
    res = F.filtration(gth, alpha, eps=eps)
    assert res.converged
    a = 0.5 * (eta * np.exp(-2 * r) + 1 - eta)
    s_star = -0.5 * np.log(2 * a)
    beta = alpha / math.sqrt(2)
    lo, hi = np.sum(np.sinh(s_star) ** 2), np.sum(np.sinh(s_star + beta) ** 2)
    assert lo - 1e-12 <= res.n_eff < hi
    Om = G.omega(4)
    assert np.abs(res.S @ Om @ res.S.T - Om).max() < 1e-12
    assert np.linalg.eigvalsh(gth - res.gamma_p).min() >= -eps


def test_directional_derivative_and_gradient():
    """First-order perturbation theory (App. C): the loss along S exp(t X)
    changes at the rate (1/2) v0^T S (X + X^T) S^T v0 (finite differences,
    non-degenerate lowest eigenvalue), and the unit gradient G maximises that
    rate over unit X in sp(2N) = {Omega H : H = H^T}."""
    gth, w = wl.lossy(4, 7, eta=0.5)
    res = F.filtration(gth, 0.02, max_iter=15)          # a generic S on the path
    S = res.S
    L0, v0 = F.loss_and_vector(gth, S)
    ev = np.linalg.eigvalsh(gth - 0.5 * S @ S.T)
    assert ev[1] - ev[0] > 1e-3                          # non-degenerate here
    rng = np.random.default_rng(0)
    Om = G.omega(4)
    Gm = F.gradient(S, v0)
    assert abs(np.linalg.norm(Gm) - 1) < 1e-14
    assert np.abs(Gm @ Om + Om @ Gm.T).max() < 1e-14   # G in sp(2N)
    dG = F.directional_derivative(S, v0, Gm)
    for _ in range(50):
        H = rng.standard_normal((8, 8))
        X = Om @ (H + H.T)
        X /= np.linalg.norm(X)
        t = 1e-6
        L1, _ = F.loss_and_vector(gth, S @ (np.eye(8) + t * X))
        Lm, _ = F.loss_and_vector(gth, S @ (np.eye(8) - t * X))
        fd = (L1 - Lm) / (2 * t)
        assert abs(fd - F.directional_derivative(S, v0, X)) < 1e-6
        assert F.directional_derivative(S, v0, X) <= dG + 1e-14
    # the first steps lower the loss
    Ls = [F.loss_and_vector(gth, F.filtration(gth, 0.02, max_iter=k).S)[0] for k in range(4)]
    assert all(Ls[i + 1] < Ls[i] for i in range(3))


def test_lossy_brickwall_feasible_and_near_optimum():
    """A lossy brick-wall state (uniform loss commutes with the passive
    network): the optimum is the lossy inputs' product optimum, N_eff* =
    sum_i sinh^2 s_i*; the descent ends feasible (W >= -eps), symplectic,
    with N_eff above N_eff* and within a few percent of it."""
    gth, w = wl.lossy(8, 3, eta=0.5, depth=4)
    res = F.filtration(gth, 0.01, eps=1e-12)
    assert res.converged
    a = 0.5 * (0.5 * np.exp(-2 * w.r) + 0.5)
    n_opt = np.sum(np.sinh(-0.5 * np.log(2 * a)) ** 2)
    assert n_opt - 1e-12 <= res.n_eff <= 1.1 * n_opt
    Om = G.omega(8)
    assert np.abs(res.S @ Om @ res.S.T - Om).max() < 1e-11
    assert np.linalg.eigvalsh(gth - res.gamma_p).min() >= -1e-12
