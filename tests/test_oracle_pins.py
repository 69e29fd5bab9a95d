"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics
(closed forms, brute-force hafnians, identities), independent of the oracle's
own code paths.  CPU only."""
import itertools
import math

import numpy as np
import pytest
from scipy.linalg import expm

import workloads as wl
from oracle import basis as B
from oracle import gaussian as G
from oracle import hafnian as H
from oracle import mps as M
from oracle import pco as P


def tmsv_gamma(r):
    """Two-mode squeezed vacuum as a 50:50 beamsplitter on an x- and a
    p-squeezed vacuum (input convention of the workloads module)."""
    U = np.array([[1, -1], [1, 1]], dtype=np.complex128) / math.sqrt(2)
    gamma, q = wl.squeezed_state(np.array([r, -r]), U)
    return gamma, q


# ---------------------------------------------------------------- P10
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_williamson_bogoliubov_identities(seed):
    w = wl.small(6, seed, depth=6, rlo=0.2, rhi=0.7)
    sub = [0, 1, 2, 6, 7, 8]
    g = w.gamma[np.ix_(sub, sub)]          # mixed 3-mode reduced state
    D, S = G.williamson(g)
    Om = G.omega(3)
    assert np.abs(S @ Om @ S.T - Om).max() < 1e-12
    assert np.abs(0.5 * S @ np.diag(np.r_[D, D]) @ S.T - g).max() < 1e-12
    assert np.all(np.diff(D) <= 1e-12) and D.min() > 1 - 1e-12
    # symplectic spectrum = |eigenvalues of i Omega V| (independent route)
    ev = np.sort(np.abs(np.linalg.eigvals(1j * Om @ (2 * g))))[::2]
    assert np.allclose(np.sort(D), ev, rtol=1e-10)
    U, V = G.uv_from_s(S)
    I3 = np.eye(3)
    # constraints of Eq. (UV)
    assert np.abs(U.conj().T @ U - V.conj().T @ V - I3).max() < 1e-12
    assert np.abs(U.T @ V - V.T @ U).max() < 1e-12
    assert np.abs(U.conj() @ U.T - V @ V.conj().T - I3).max() < 1e-12
    assert np.abs(G.sinv_rows_from_uv(U, V) @ S - np.eye(6)).max() < 1e-12


def test_q_two_routes_and_roundtrip():
    w = wl.small(7, 5, depth=5, rlo=0.2, rhi=0.6)
    # route 1: moments (O2); route 2: the generator's U diag(-tanh r) U^T
    assert np.abs(G.q_from_gamma(w.gamma) - w.Q).max() < 1e-12
    # route 3: Williamson of the full pure state (all D = 1), Q = U^-dag V^dag
    D, S = G.williamson(w.gamma)
    assert np.abs(D - 1).max() < 1e-10
    U, V = G.uv_from_s(S)
    Q3 = np.linalg.inv(U.conj().T) @ V.conj().T
    assert np.abs(Q3 - w.Q).max() < 1e-10
    assert np.abs(Q3 - Q3.T).max() < 1e-10          # Q symmetric
    assert np.abs(G.gamma_from_q(w.Q) - w.gamma).max() < 1e-12
    assert G.purity_defect(w.gamma) < 1e-12


def test_q_left_annihilation_conditions():
    """|phi_L> = prod exp(b^dag l^dag)|0> is annihilated by l_q - b_q^dag and
    b_q - l_q^dag; with a = Q c^dag on the paired form these read Q alpha = -beta."""
    w = wl.small(5, 9, depth=5)
    sub = [0, 1, 5, 6]
    D, S = G.williamson(w.gamma[np.ix_(sub, sub)])
    U, V = G.uv_from_s(S)
    Q = G.q_left(U, V, 2)
    n = 2
    for q in range(n):
        e = np.zeros(n); e[q] = 1
        # l_q - b_q^dag = l_q + sum V_jq a_j - sum U_jq a_j^dag
        alpha = np.r_[V[:, q], e]
        beta = np.r_[-U[:, q], np.zeros(n)]
        assert np.abs(Q @ alpha + beta).max() < 1e-12
        # b_q - l_q^dag = sum U*_jq a_j - V*_jq a_j^dag - l_q^dag
        alpha = np.r_[U[:, q].conj(), np.zeros(n)]
        beta = np.r_[-V[:, q].conj(), -e]
        assert np.abs(Q @ alpha + beta).max() < 1e-12


# ---------------------------------------------------------------- P2
@pytest.mark.parametrize("r", [0.2, 0.5, 0.9])
def test_tmsv_closed_forms(r):
    gamma, q = tmsv_gamma(r)
    cuts = G.gsvd_chain(gamma)
    lam = math.tanh(r)
    assert abs(cuts[0].D[0] - math.cosh(2 * r)) < 1e-12          # D = cosh 2r
    assert abs(cuts[0].lam2[0] - lam ** 2) < 1e-12                 # Lambda = tanh r
    # entropy of Sec. II A vs -sum p log p of the Schmidt weights (1-L^2) L^{2n}
    p = (1 - lam ** 2) * lam ** (2 * np.arange(400))
    p = p[p > 0]
    assert abs(G.entropy_q(np.array([lam ** 2]))[0] + np.sum(p * np.log(p))) < 1e-10
    mps = M.build_mps(gamma, d=90, chi=90)
    T = M.normalise(mps.tensors)
    for n in range(8):
        a = M.contract(T, [n, n])
        assert abs(abs(a) ** 2 - (1 - lam ** 2) * lam ** (2 * n)) < 1e-12
        assert abs(M.contract(T, [n, n + 1])) < 1e-14


# ---------------------------------------------------------------- P1
def test_product_state_closed_forms():
    r = np.array([0.3, 0.5, 0.7, 0.2])
    gamma, q = wl.squeezed_state(r, np.eye(4, dtype=np.complex128))
    mps = M.build_mps(gamma, d=12, chi=8)
    assert mps.n_e == [0, 0, 0] and mps.bond_dims == [1, 1, 1, 1, 1]
    T = M.normalise(mps.tensors)
    pv = abs(M.contract(T, [0, 0, 0, 0])) ** 2
    # the cutoff d=12 drops weight; compare the vacuum amplitude ratio exactly
    for i, ri in enumerate(r):
        for k in range(3):
            pat = [0] * 4
            pat[i] = 2 * k
            ratio = abs(M.contract(T, pat)) ** 2 / pv
            exact = math.tanh(ri) ** (2 * k) * math.factorial(2 * k) / (4 ** k * math.factorial(k) ** 2)
            assert abs(ratio - exact) < 1e-13
    # with a large cutoff, P(vac) = prod 1/cosh r
    T2 = M.normalise(M.build_mps(gamma, d=60, chi=4).tensors)
    assert abs(abs(M.contract(T2, [0] * 4)) ** 2 - np.prod(1 / np.cosh(r))) < 1e-12


# ---------------------------------------------------------------- P4
@pytest.mark.parametrize("N,seed", [(3, 11), (4, 12), (5, 1)])
def test_amplitudes_vs_hafnian(N, seed):
    """All patterns with n_i <= 3 and even total <= N+2: MPS amplitude ratios
    to the vacuum equal haf(Q_n)/sqrt(n!) when the truncation is negligible."""
    w = wl.small(N, seed, d=8, depth=N, rlo=0.1, rhi=0.3, haar=True)
    mps = M.build_mps(w.gamma, d=8, chi=300)
    assert max(mps.eps) < 1e-14
    T = mps.tensors
    a0 = M.contract(T, [0] * N)
    worst = 0.0
    for n in itertools.product(range(4), repeat=N):
        if sum(n) % 2 or sum(n) > N + 2:
            continue
        ex = H.relative_amplitude(w.Q, n)
        got = M.contract(T, n) / a0
        worst = max(worst, abs(ex - got) / max(abs(ex), 1e-3))
    assert worst < 1e-10


def test_pr1_fidelity_vs_hafnian_within_truncation():
    """8 modes through a Haar unitary, d=8, chi=64: amplitudes over all
    patterns with total <= 8 and n_i <= 7 agree with hafnians up to the
    truncation error (|1-F| bounded by a small multiple of sum eps_m)."""
    w = wl.config("pr1_n8")
    mps = M.build_mps(w.gamma, d=8, chi=64)
    T = M.normalise(mps.tensors)
    pats = [n for n in itertools.product(range(8), repeat=8) if sum(n) <= 6 and sum(n) % 2 == 0]
    ex = np.array([H.amplitude(w.Q, n) for n in pats])
    got = M.amplitudes(T, pats)
    f = abs(np.vdot(ex, got)) ** 2 / (np.vdot(ex, ex).real * np.vdot(got, got).real)
    assert 1 - f < 10 * sum(mps.eps) + 1e-12


# ---------------------------------------------------------------- P5
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_local_tensor_entries_are_hafnians(seed):
    """Every entry of the PCO tensor equals haf(Q_k)/sqrt(k!) of its occupation
    k = (n_alpha, p, n_beta), for an arbitrary symmetric complex Q."""
    g = np.random.default_rng(seed)
    nl, nr, d = 2, 3, 4
    n = nl + 1 + nr
    Q = (g.standard_normal((n, n)) + 1j * g.standard_normal((n, n))) * 0.4
    Q = 0.5 * (Q + Q.T)
    bl = B.kept_basis(np.array([0.3, 0.1]), 12)
    br = B.kept_basis(np.array([0.4, 0.2, 0.05]), 15)
    C = P.local_tensor(Q, bl, br, d, c=1.0)
    for a in range(bl.D):
        for p in range(d):
            for b in range(br.D):
                k = np.r_[bl.occ[a], p, br.occ[b]]
                ex = H.local_entry(Q, k)
                assert abs(C[a, p, b] - ex) <= 1e-12 * max(1, abs(ex))


# ---------------------------------------------------------------- P6
def test_parity_odd_entries_vanish():
    w = wl.small(8, 3, depth=6)
    mps = M.build_mps(w.gamma, d=5, chi=40)
    for m, A in enumerate(mps.tensors):
        nl = mps.bases[m].occ.sum(axis=1)
        nr = mps.bases[m + 1].occ.sum(axis=1)
        tot = nl[:, None, None] + np.arange(5)[None, :, None] + nr[None, None, :]
        assert np.all(A[tot % 2 == 1] == 0)


# ---------------------------------------------------------------- P9
def test_norm_equals_sum_over_patterns():
    w = wl.small(4, 4, depth=4, d=4)
    T = M.build_mps(w.gamma, d=4, chi=10).tensors
    R = M.environments(T)
    tot = sum(abs(M.contract(T, n)) ** 2 for n in itertools.product(range(4), repeat=4))
    assert abs(tot - R[0][0, 0].real) < 1e-12 * tot


# ---------------------------------------------------------------- P3
def test_photon_numbers_and_vacuum_from_covariance():
    w = wl.small(5, 21, depth=4, rlo=0.05, rhi=0.25)
    T = M.normalise(M.build_mps(w.gamma, d=14, chi=200).tensors)
    marg = M.site_marginals(T)
    N = 5
    nbar = 0.5 * (np.diag(w.gamma)[:N] + np.diag(w.gamma)[N:]) - 0.5
    assert np.abs(marg @ np.arange(14) - nbar).max() < 1e-10
    pvac = np.linalg.det(w.gamma + 0.5 * np.eye(2 * N)) ** -0.5
    assert abs(abs(M.contract(T, [0] * N)) ** 2 - pvac) < 1e-10
    assert abs(pvac - H.vacuum_amplitude(w.Q) ** 2) < 1e-12


# ---------------------------------------------------------------- P11
def _dense_ops(bl, d, br):
    """Creation operators of every mode of c_m as dense matrices on V_m,
    projected (P d^dag P)."""
    dims = (bl.D, d, br.D)
    dim = bl.D * d * br.D
    idx = lambda a, p, b: (a * d + p) * br.D + b
    ops = []
    for side, basis, ne in ((0, bl, bl.ne), (1, None, 1), (2, br, br.ne)):
        for q in range(ne):
            Op = np.zeros((dim, dim))
            for a in range(dims[0]):
                for p in range(d):
                    for b in range(dims[2]):
                        if side == 1:
                            if p + 1 < d:
                                Op[idx(a, p + 1, b), idx(a, p, b)] = math.sqrt(p + 1)
                            continue
                        occ = (bl if side == 0 else br).occ[a if side == 0 else b].copy()
                        occ[q] += 1
                        t = basis.index.get(tuple(int(x) for x in occ))
                        if t is None:
                            continue
                        if side == 0:
                            Op[idx(t, p, b), idx(a, p, b)] = math.sqrt(occ[q])
                        else:
                            Op[idx(a, p, t), idx(a, p, b)] = math.sqrt(occ[q])
            ops.append(Op)
    return ops


def test_pco_matches_dense_exponential_and_is_order_free():
    g = np.random.default_rng(7)
    bl = B.kept_basis(np.array([0.3, 0.2]), 7)
    br = B.kept_basis(np.array([0.25]), 5)
    d = 4
    n = 4
    Q = (g.standard_normal((n, n)) + 1j * g.standard_normal((n, n))) * 0.5
    Q = 0.5 * (Q + Q.T)
    ops = _dense_ops(bl, d, br)
    X = sum(0.5 * Q[i, j] * ops[i] @ ops[j] for i in range(n) for j in range(n))
    vac = np.zeros(X.shape[0], dtype=np.complex128)
    vac[0] = 1
    # the projected creation operators commute on V and X is nilpotent here,
    # so P exp(X)|0> is the plain matrix exponential of the projected X
    ref = (expm(X) @ vac).reshape(bl.D, d, br.D)
    C1 = P.local_tensor(Q, bl, br, d)
    assert np.abs(C1 - ref).max() < 1e-12
    order = P.pco_order(2, 1)
    C2 = P.local_tensor(Q, bl, br, d, order=list(reversed(order)))
    assert np.abs(C1 - C2).max() < 1e-13


# ---------------------------------------------------------------- P12
def test_truncation_error_identity_and_d_eps():
    lam2 = 0.3
    b = B.kept_basis(np.array([lam2]), 10)
    # one mode: kept weight (1 - L^2) sum_{n<D} L^{2n} = 1 - L^{2D}
    assert abs(b.eps - lam2 ** 10) < 1e-15
    b2 = B.kept_basis(np.array([lam2]), 1000, eps=1e-6)
    # D(eps) = smallest D with L^{2D} <= eps
    assert b2.D == math.ceil(math.log(1e-6) / math.log(lam2))
    # two modes: kept set is down-closed and sorted by energy
    b3 = B.kept_basis(np.array([0.4, 0.1]), 30)
    assert np.all(np.diff(b3.E) >= -1e-12)
    for occ in b3.occ:
        for q in range(2):
            if occ[q]:
                s = occ.copy(); s[q] -= 1
                assert tuple(int(x) for x in s) in b3.index
    # brute force: the 30 lowest energies among all vectors with n_q <= 40
    allv = np.array(list(itertools.product(range(41), range(41))))
    E = allv @ B.weights(np.array([0.4, 0.1]))
    assert np.allclose(np.sort(E)[:30], b3.E, atol=1e-12)


def test_tie_break_is_lexicographic():
    # w_1 = 2 w_2 exactly: E(1,0) = E(0,2)
    lam2 = np.array([0.04, 0.2])
    b = B.kept_basis(lam2, 6)
    assert [tuple(x) for x in b.occ] == [(0, 0), (0, 1), (0, 2), (1, 0), (0, 3), (1, 1)]


def test_vector_set_relation():
    b = B.kept_basis(np.array([0.3, 0.15, 0.1]), 40)
    for q in range(3):
        vs = B.vector_set(b, q)
        for a, bb, k in zip(vs.vin, vs.vout, vs.vord):
            diff = b.occ[bb] - b.occ[a]
            assert diff[q] == k and np.all(np.delete(diff, q) == 0)
        # every (state, kappa <= n_q) appears exactly once
        assert vs.vin.size == int(b.occ[:, q].sum())
    comp = B.compose(B.vector_set(b, 0), B.vector_set(b, 1))
    for a, bb, k in zip(comp.vin, comp.vout, comp.vord):
        diff = b.occ[bb] - b.occ[a]
        assert diff[0] == k and diff[1] == k and diff[2] == 0


# ---------------------------------------------------------------- P13
def test_sampling_rule_and_statistics():
    w = wl.small(4, 8, depth=4, d=4, rlo=0.3, rhi=0.6)
    T = M.normalise(M.build_mps(w.gamma, d=4, chi=20).tensors)
    pats = list(itertools.product(range(4), repeat=4))
    prob = np.array([abs(M.contract(T, n)) ** 2 for n in pats])
    prob /= prob.sum()
    S = 40000
    u = wl.uniforms(S, 4, seed=3)
    out, flag = M.sample(T, u)
    assert not flag.any()
    assert np.all(out.astype(int).sum(axis=1) % 2 == 0)       # P6 on samples
    counts = np.zeros(len(pats))
    lut = {p: i for i, p in enumerate(pats)}
    for row in out:
        counts[lut[tuple(int(x) for x in row)]] += 1
    keep = prob * S > 5
    chi2 = np.sum((counts[keep] - S * prob[keep]) ** 2 / (S * prob[keep]))
    dof = keep.sum() - 1
    assert chi2 < dof + 6 * math.sqrt(2 * dof)
    # the selection rule itself on a hand-made first site: p* = min{p: uZ < C_p}
    marg = M.site_marginals(T)[0]
    cdf = np.cumsum(marg)
    for uu in (0.0, 0.3, cdf[0] - 1e-9, cdf[0] + 1e-9, 0.999):
        o, _ = M.sample(T, np.array([[uu, 0.5, 0.5, 0.5]]))
        assert o[0, 0] == int(np.argmax(uu < cdf))


def test_gsvd_chain_reproduces_state_on_random_instances():
    """Fidelity of the oracle MPS with the exact state over all patterns of a
    6-mode state (brute force over the full truncated Fock space)."""
    w = wl.small(6, 31, depth=6, rlo=0.1, rhi=0.3, d=5)
    mps = M.build_mps(w.gamma, d=5, chi=200)
    T = M.normalise(mps.tensors)
    pats = [n for n in itertools.product(range(5), repeat=6) if sum(n) % 2 == 0 and sum(n) <= 8]
    ex = np.array([H.amplitude(w.Q, n) for n in pats])
    got = M.amplitudes(T, pats)
    # compare ratios to the vacuum (normalisation-free)
    assert np.abs(got / got[0] - ex / ex[0]).max() < 1e-9
