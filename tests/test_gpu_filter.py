"""Mixed -> pure decomposition on the GPU (gbsmps_filter; Sec. III
Eq. (decompose), App. C) against the FP64 oracle on the same lossy inputs.

The descent is deterministic given the lowest eigenvector of W at every step,
so while that eigenvalue stays separated from the next one the GPU follows
the oracle's trajectory step for step: S after K steps agrees entrywise
(1e-9 of the largest entry), the loss values agree, and runs to convergence
take the same number of steps.  Whatever the path: the result is
symplectic, W = Gamma_th - S S^T / 2 >= -eps, and N_eff lies between the
optimum of the trace problem and the descent's last step above it."""
import math

import numpy as np
import pytest

import workloads as wl
from oracle import filtration as F
from oracle import gaussian as G

pytestmark = pytest.mark.gpu

g = pytest.importorskip("paper_2512_10643_gb300")


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = g.Context(0)
    yield c
    c.close()


def min_gap_along(gth, alpha, iters):
    """Smallest relative gap lambda_1 - lambda_0 of W along the oracle's path."""
    S = np.eye(gth.shape[0])
    worst = np.inf
    for _ in range(iters + 1):
        ev, V = np.linalg.eigh(gth - 0.5 * S @ S.T)
        worst = min(worst, (ev[1] - ev[0]) / np.abs(ev).max())
        from scipy.linalg import expm
        S = S @ expm(-alpha * F.gradient(S, V[:, 0]))
    return worst


@pytest.mark.parametrize("K", [0, 1, 5, 30])
def test_first_steps_follow_the_oracle(ctx, K):
    gth, w = wl.lossy(8, 3, eta=0.5, depth=4)
    alpha = 0.01
    ref = F.filtration(gth, alpha, eps=0.0, max_iter=K)
    S, it, loss = g.gbsmps_filter(ctx.h, gth[None], alpha, eps=0.0, max_iter=K)
    assert it[0] == K
    assert np.abs(S[0] - ref.S).max() <= 1e-9 * np.abs(ref.S).max()
    assert abs(loss[0] - ref.loss) <= 1e-12 * max(1.0, abs(ref.loss))


@pytest.mark.parametrize("N,seed,eta,alpha", [(4, 7, 0.5, 0.01), (8, 3, 0.5, 0.01), (12, 5, 0.4, 0.02)])
def test_converged_decomposition(ctx, N, seed, eta, alpha):
    gth, w = wl.lossy(N, seed, eta=eta, depth=max(1, N // 2))
    eps = 1e-10
    ref = F.filtration(gth, alpha, eps=eps)
    assert ref.converged
    S, it, loss = g.gbsmps_filter(ctx.h, gth[None], alpha, eps=eps, max_iter=100000)
    S = S[0]
    Om = G.omega(N)
    assert np.abs(S @ Om @ S.T - Om).max() < 1e-10              # symplectic
    assert np.linalg.eigvalsh(gth - 0.5 * S @ S.T).min() >= -eps - 1e-12
    assert loss[0] <= eps
    a = 0.5 * (eta * np.exp(-2 * w.r) + 1 - eta)
    n_opt = np.sum(np.sinh(-0.5 * np.log(2 * a)) ** 2)
    n_eff = 0.5 * np.trace(0.5 * S @ S.T) - 0.5 * N
    assert n_opt - 1e-9 <= n_eff <= 1.1 * n_opt
    if min_gap_along(gth, alpha, ref.iters) > 1e-6:              # the paths cannot part
        assert it[0] == ref.iters
        assert np.abs(S - ref.S).max() <= 1e-8 * np.abs(ref.S).max()
        assert abs(n_eff - ref.n_eff) <= 1e-9 * ref.n_eff


def test_single_mode_closed_form(ctx):
    """S_k = R diag(e^{-k b}, e^{k b}) R^T with b = alpha / sqrt 2 (App. C
    steps for one lossy squeezed mode), stopping at the first k with
    a - e^{-2 k b}/2 >= -eps."""
    r, eta, phi, alpha, eps = 0.7, 0.5, 0.4, 0.01, 1e-12
    a = 0.5 * (eta * math.exp(-2 * r) + 1 - eta)
    bq = 0.5 * (eta * math.exp(2 * r) + 1 - eta)
    c, s = math.cos(phi), math.sin(phi)
    R = np.array([[c, -s], [s, c]])
    gth = R @ np.diag([a, bq]) @ R.T
    beta = alpha / math.sqrt(2)
    k = 0
    while a - 0.5 * math.exp(-2 * k * beta) < -eps:
        k += 1
    S, it, loss = g.gbsmps_filter(ctx.h, gth[None], alpha, eps=eps)
    assert it[0] == k
    want = R @ np.diag([math.exp(-k * beta), math.exp(k * beta)]) @ R.T
    assert np.abs(S[0] - want).max() < 1e-11


def test_batch_equals_single_launches_and_edge_cases(ctx):
    torch = pytest.importorskip("torch")
    gs = np.stack([wl.lossy(6, s, eta=0.5)[0] for s in (1, 2, 3)])
    Sb, itb, lb = g.gbsmps_filter(ctx.h, gs, 0.01, eps=1e-10)
    for k in range(3):
        S1, it1, l1 = g.gbsmps_filter(ctx.h, gs[k:k + 1], 0.01, eps=1e-10)
        assert np.array_equal(S1[0], Sb[k]) and it1[0] == itb[k] and l1[0] == lb[k]
    # device buffers give the same result
    Sd, itd, ld = g.gbsmps_filter(ctx.h, torch.from_numpy(gs).cuda(), 0.01, eps=1e-10)
    assert np.array_equal(Sd.cpu().numpy(), Sb) and np.array_equal(itd, itb)
    # max_iter = 0: S = I and the initial loss 1/2 - lambda_min(Gamma_th)
    S0, it0, l0 = g.gbsmps_filter(ctx.h, gs[:1], 0.01, max_iter=0)
    assert it0[0] == 0 and np.array_equal(S0[0], np.eye(12))
    assert abs(l0[0] - (0.5 - np.linalg.eigvalsh(gs[0]).min())) < 1e-13
    # a pure input needs no step (W = Gamma - I/2 >= 0 is not the point: the
    # vacuum is the only state with W >= 0 at S = I)
    vac = 0.5 * np.eye(4)
    Sv, itv, lv = g.gbsmps_filter(ctx.h, vac[None], 0.01, eps=1e-12)
    assert itv[0] == 0 and np.array_equal(Sv[0], np.eye(4))
    # count = 0 is a no-op; N above the limit is rejected
    g.gbsmps_filter(ctx.h, np.zeros((0, 4, 4)), 0.01)
    with pytest.raises(g.GbsmpsError) as e:
        g.gbsmps_filter(ctx.h, np.eye(130)[None] * 0.5, 0.01)
    assert e.value.code == g.ERR_BOUNDS
