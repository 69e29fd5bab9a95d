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


def compositions(n, total, cap):
    """Every n-tuple of integers in [0, cap] with sum <= total."""
    if n == 0:
        yield ()
        return
    for k in range(min(total, cap) + 1):
        for rest in compositions(n - 1, total - k, cap):
            yield (k,) + rest


def tmsv_gamma(r):
    """Two-mode squeezed vacuum as a 50:50 beamsplitter on an x- and a
    p-squeezed vacuum (input convention of the workloads module)."""
    U = np.array([[1, -1], [1, 1]], dtype=np.complex128) / math.sqrt(2)
    gamma, q = wl.squeezed_state(np.array([r, -r]), U)
    return gamma, q


# ---------------------------------------------------------------- P10
@pytest.mark.parametrize("route", [G.williamson, G.williamson_sqrt])
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_williamson_bogoliubov_identities(seed, route):
    w = wl.small(6, seed, depth=6, rlo=0.2, rhi=0.7)
    sub = [0, 1, 2, 6, 7, 8]
    g = w.gamma[np.ix_(sub, sub)]          # mixed 3-mode reduced state
    D, S = route(g)
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
    pats = [n for n in compositions(8, 8, 7) if sum(n) % 2 == 0]
    assert len(pats) == 8510
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


# ---------------------------------------------------------------- O9: overlap and fidelity
def _rotated_squeezed(r, phi):
    """x-squeezed vacuum of strength r behind the phase shifter e^{i phi}:
    paired-form coefficient q = -e^{2 i phi} tanh r."""
    return wl.squeezed_state(np.array([r]), np.array([[np.exp(1j * phi)]]))


@pytest.mark.parametrize("r1,p1,r2,p2", [(0.3, 0.0, 0.7, 0.0), (0.5, 0.3, 0.5, 1.1),
                                         (0.8, -0.4, 0.2, 0.9), (0.6, 0.7, 0.4, 0.2)])
def test_overlap_closed_form_single_mode(r1, p1, r2, p2):
    """Two single-mode squeezed vacua with paired-form coefficients
    q_j = -e^{i t_j} tanh r_j.  Expanding both states in Fock states and
    summing sum_k C(2k, k) x^k = (1 - 4x)^{-1/2}:
        <z1|z2> = (cosh r1 cosh r2)^{-1/2} (1 - e^{i(t2 - t1)} tanh r1 tanh r2)^{-1/2}
    (principal root, both vacuum amplitudes real positive), so
    |<z1|z2>|^2 = 1/|cosh r1 cosh r2 - e^{i(t2-t1)} sinh r1 sinh r2|, which is
    1/cosh(r1 - r2) for t1 = t2.  A missing conjugation in the sweep turns
    t2 - t1 into t2 + t1 and fails the cases with t1 != 0."""
    ga, qa = _rotated_squeezed(r1, p1)
    gb, qb = _rotated_squeezed(r2, p2)
    ta = M.normalise(M.build_mps(ga, d=90, chi=1).tensors)
    tb = M.normalise(M.build_mps(gb, d=90, chi=1).tensors)
    t1, t2 = np.angle(-qa[0, 0]), np.angle(-qb[0, 0])
    c1, c2, s1, s2 = np.cosh(r1), np.cosh(r2), np.sinh(r1), np.sinh(r2)
    f_ex = 1.0 / abs(c1 * c2 - np.exp(1j * (t2 - t1)) * s1 * s2)
    if p1 == p2 == 0.0:
        assert abs(f_ex - 1 / np.cosh(r1 - r2)) < 1e-15
    assert abs(M.fidelity(ta, tb) - f_ex) < 1e-12
    ov_ex = (c1 * c2) ** -0.5 * (1 - np.exp(1j * (t2 - t1)) * np.tanh(r1) * np.tanh(r2)) ** -0.5
    assert abs(M.overlap(ta, tb) - ov_ex) < 1e-12
    assert abs(M.overlap(tb, ta) - np.conj(ov_ex)) < 1e-12


@pytest.mark.parametrize("seeds", [(41, 42), (43, 44)])
def test_overlap_equals_dense_inner_product(seeds):
    """Two different entangled 4-mode states (different bond bases): the
    transfer-matrix <a|b> equals sum_n conj(a_n) b_n over the whole truncated
    Fock space, each amplitude from the plain matrix chain; the fidelity
    equals |<a|b>|^2/(<a|a><b|b>) of the dense vectors."""
    wa = wl.small(4, seeds[0], d=4, depth=4, rlo=0.3, rhi=0.7)
    wb = wl.small(4, seeds[1], d=4, depth=4, rlo=0.3, rhi=0.7)
    ta = M.build_mps(wa.gamma, d=4, chi=30).tensors
    tb = M.build_mps(wb.gamma, d=4, chi=30).tensors
    pats = list(itertools.product(range(4), repeat=4))
    va = M.amplitudes(ta, pats)
    vb = M.amplitudes(tb, pats)
    ab = np.vdot(va, vb)
    scale = np.linalg.norm(va) * np.linalg.norm(vb)
    assert abs(M.overlap(ta, tb) - ab) <= 1e-13 * scale
    assert abs(M.overlap(tb, ta) - np.conj(ab)) <= 1e-13 * scale
    assert abs(M.overlap(ta, ta) - np.vdot(va, va)) <= 1e-13 * np.vdot(va, va).real
    f = abs(ab) ** 2 / (np.vdot(va, va).real * np.vdot(vb, vb).real)
    assert 1e-3 < f < 0.999                 # the two states really differ
    assert abs(M.fidelity(ta, tb) - f) < 1e-12
    # gauge invariance: A^2 -> A^2 X, A^3 -> X^-1 A^3 on bond 2 leaves <a|b>
    g = np.random.default_rng(5)
    D2 = ta[1].shape[2]
    X = np.eye(D2) + 0.3 * (g.standard_normal((D2, D2)) + 1j * g.standard_normal((D2, D2))) / D2
    tg = [t.copy() for t in ta]
    tg[1] = np.einsum("apb,bc->apc", tg[1], X)
    tg[2] = np.einsum("cb,bpd->cpd", np.linalg.inv(X), tg[2])
    assert abs(M.overlap(tg, tb) - ab) <= 1e-12 * scale


# ---------------------------------------------------------------- O10: the boundary flag
def test_sampling_boundary_flag():
    """A uniform placed on the first site's CDF value C_p is flagged
    (|uZ - C_p| <= 1e-12 Z); 1e-9 below it takes p (the first p with
    uZ < C_p), 1e-9 above it takes the next p with q > 0, both unflagged."""
    w = wl.small(4, 8, depth=4, d=4, rlo=0.3, rhi=0.6)
    T = M.normalise(M.build_mps(w.gamma, d=4, chi=20).tensors)
    marg = M.site_marginals(T)[0]
    cdf = np.cumsum(marg)
    rest = [0.5, 0.5, 0.5]
    for p in range(3):
        if marg[p] <= 1e-6:
            continue
        o, fl = M.sample(T, np.array([[cdf[p]] + rest]))
        assert fl[0]
        assert o[0, 0] in (p, p + 1 + int(np.argmax(marg[p + 1:] > 0)))
        o, fl = M.sample(T, np.array([[cdf[p] - 1e-9] + rest]))
        assert not fl[0] and o[0, 0] == p
        o, fl = M.sample(T, np.array([[cdf[p] + 1e-9] + rest]))
        assert not fl[0] and o[0, 0] == p + 1 + int(np.argmax(marg[p + 1:] > 0))
    # a flag on a later site is reported too
    o0, _ = M.sample(T, np.array([[0.2] + rest]))
    sub = M.site_marginals(T)                     # not conditional: use the rule
    assert o0.shape == (1, 4) and sub.shape == (4, 4)


# ---------------------------------------------------------------- hafnian module
def test_hafnian_closed_forms():
    """haf(ones(2n)) = (2n-1)!!; a 4x4 hafnian is the sum over its three
    perfect matchings; the single-mode squeezed vacuum with paired-form
    coefficient q has <2k|z>/<0|z> = q^k sqrt((2k)!)/(2^k k!) (expansion of
    exp(q a^dag^2/2)|0>) and |<0|z>|^4 = 1 - |q|^2."""
    for n in range(1, 6):
        assert H.hafnian(np.ones((2 * n, 2 * n))) == math.prod(range(1, 2 * n, 2))
    assert H.hafnian(np.ones((5, 5))) == 0
    g = np.random.default_rng(3)
    A = g.standard_normal((4, 4)) + 1j * g.standard_normal((4, 4))
    A = A + A.T
    ex = A[0, 1] * A[2, 3] + A[0, 2] * A[1, 3] + A[0, 3] * A[1, 2]
    assert abs(H.hafnian(A) - ex) < 1e-13
    q = -np.exp(0.7j) * math.tanh(0.6)
    Q = np.array([[q]])
    for k in range(6):
        ex = q ** k * math.sqrt(math.factorial(2 * k)) / (2 ** k * math.factorial(k))
        assert abs(H.relative_amplitude(Q, [2 * k]) - ex) < 1e-13
        assert H.relative_amplitude(Q, [2 * k + 1]) == 0
    assert abs(H.vacuum_amplitude(Q) ** 2 - 1 / math.cosh(0.6)) < 1e-14


# ---------------------------------------------------------------- purity and gauge
def test_purity_defect_of_thermal_and_pure_states():
    """A single-mode thermal state Gamma = (nbar + 1/2) I has
    (2 Gamma Omega)^2 = -(2 nbar + 1)^2 I, so the defect is (2 nbar + 1)^2 - 1;
    a pure state has defect 0."""
    for nbar in (0.1, 0.5, 2.0):
        assert abs(G.purity_defect((nbar + 0.5) * np.eye(2)) - ((2 * nbar + 1) ** 2 - 1)) < 1e-12
    w = wl.small(5, 3, depth=4)
    assert G.purity_defect(w.gamma) < 1e-12


def test_canonical_gauge_fixes_the_free_phases():
    """b_q -> e^{i t_q} b_q multiplies column q of U and V by e^{-i t_q}; the
    canonical gauge removes any such phase (same output for every input
    phase), makes each column's largest |U| entry real positive and keeps
    the constraints of Eq. (UV)."""
    w = wl.small(6, 2, depth=6, rlo=0.2, rhi=0.7)
    sub = [0, 1, 2, 6, 7, 8]
    D, S = G.williamson(w.gamma[np.ix_(sub, sub)])
    U, V = G.uv_from_s(S)
    U1, V1 = G.canonical_gauge(U, V)
    ph = np.exp(1j * np.array([0.4, -2.0, 2.9]))
    U2, V2 = G.canonical_gauge(U * ph, V * ph)
    assert np.abs(U1 - U2).max() < 1e-13 and np.abs(V1 - V2).max() < 1e-13
    for q in range(3):
        j = int(np.argmax(np.abs(U1[:, q])))
        assert abs(U1[j, q].imag) < 1e-15 and U1[j, q].real > 0
    I3 = np.eye(3)
    assert np.abs(U1.conj().T @ U1 - V1.conj().T @ V1 - I3).max() < 1e-12
    assert np.abs(U1.T @ V1 - V1.T @ U1).max() < 1e-12


# ---------------------------------------------------------------- FP64 determinacy (tolerances)
def test_two_williamson_routes_bound_fp64_amplitude_parity():
    """How closely is the MPS of a given Gamma determined in FP64 at all?
    Two valid FP64 Williamson routes (Cholesky vs symmetric square root) give
    MPSs whose fidelity agrees to ~1e-15 but whose amplitudes differ by
    ~1e-12 of the largest amplitude when modes near the freeze threshold
    1e-9 are kept: such a mode is nearly degenerate with the frozen ones (gap
    ~2 Lambda^2), so its eigenvector is fixed only to ~1e-16/(2 Lambda^2).
    Small amplitudes therefore carry relative differences far above 1e-9 in
    any FP64 implementation; GPU parity is held to the oracle-route spread."""
    w = wl.small(24, 5, d=4, chi=64, depth=6)
    m1 = M.build_mps(w.gamma, d=4, chi=64, lambda2_freeze=1e-9)
    m2 = M.build_mps(w.gamma, d=4, chi=64, lambda2_freeze=1e-9, route=G.williamson_sqrt)
    assert m1.bond_dims == m2.bond_dims and m1.n_e == m2.n_e
    T1, T2 = M.normalise(m1.tensors), M.normalise(m2.tensors)
    assert 1 - M.fidelity(T1, T2) < 1e-14
    pats = np.concatenate([wl.random_patterns(300, 24, 4, seed=1),
                           wl.random_patterns(300, 24, 4, seed=2, even=False)])
    a1, a2 = M.amplitudes(T1, pats), M.amplitudes(T2, pats)
    mx = np.abs(a1).max()
    spread = np.abs(a1 - a2)
    assert 1e-14 * mx < spread.max() < 1e-10 * mx
    mid = np.abs(a1) > 1e-8 * mx
    assert np.max(spread[mid] / np.abs(a1[mid])) > 1e-8      # far above 1e-9 relative
    # odd totals are exactly zero on both routes (P6)
    odd = pats.astype(int).sum(1) % 2 == 1
    assert np.all(a1[odd] == 0) and np.all(a2[odd] == 0)
