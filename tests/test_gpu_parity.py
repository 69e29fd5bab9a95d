"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the same
seeded inputs.  Tolerances (FP64 path): amplitude relative error <= 1e-9 for
|a| >= 1e-10 max|a| (absolute below), state fidelity >= 1 - 1e-10, tensor
entries 1e-11 of the largest entry, samples bit-exact except draws flagged
within 1e-12 Z of a CDF boundary."""
import itertools

import numpy as np
import pytest

import workloads as wl
from oracle import basis as B
from oracle import gaussian as G
from oracle import hafnian as H
from oracle import mps as M
from oracle import pco as P

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


def amp_close(a_gpu, a_ref, rtol=1e-9, floor=1e-12):
    """|a_gpu - a_ref| <= rtol |a_ref| + floor max|a_ref|.  The floor is the
    FP64 noise of an N-site matrix chain (rounding of each product relative
    to the largest amplitude); above it the bound is relative 1e-9."""
    a_gpu = np.asarray(a_gpu)
    a_ref = np.asarray(a_ref)
    scale = np.abs(a_ref).max()
    return bool(np.all(np.abs(a_gpu - a_ref) <= rtol * np.abs(a_ref) + floor * scale))


def route_floor(a_ref, a_alt, N, Dmax):
    """Relative floor for amp_close: ten times the largest difference between
    the amplitudes of two valid FP64 oracle routes (Cholesky and symmetric
    square-root Williamson forms) plus the forward rounding bound of an
    N-site chain of products of length <= Dmax (N Dmax eps of the largest
    amplitude).  Modes kept just above the freeze threshold make the MPS
    itself undetermined in FP64 at the first level (their eigenvectors are
    fixed only to ~1e-16/(2 Lambda^2))."""
    scale = np.abs(a_ref).max()
    spread = np.abs(np.asarray(a_alt) - np.asarray(a_ref)).max() / scale
    return 10 * spread + N * Dmax * np.finfo(np.float64).eps


def all_kinds_of_patterns(N, d, seed, full=False):
    """Even and odd totals (odd ones are exactly zero, P6) and patterns with
    some n_i >= d (zero by the cutoff); every low pattern for tiny N."""
    if full:
        pats = np.array([p for p in itertools.product(range(min(d, 4)), repeat=N)
                         if sum(p) <= 8], dtype=np.uint8)
    else:
        pats = np.concatenate([wl.random_patterns(200, N, d, seed=seed),
                               wl.random_patterns(100, N, d, seed=seed + 1, even=False)])
    over = np.zeros((3, N), dtype=np.uint8)
    over[0, 0], over[1, N - 1], over[2, N // 2] = d, 255, d + 1
    return np.concatenate([pats, over])


def unambiguous(cuts, freeze, rel=1e-3):
    """True when no symplectic eigenvalue puts Lambda^2 within rounding
    distance of the freeze threshold (the active-mode count is then the same
    for any FP64 eigensolver)."""
    for c in cuts[:-1]:
        l2 = (c.D - 1) / (c.D + 1)
        if np.any(np.abs(l2 - freeze) <= 1e-14 + rel * freeze):
            return False
    return True


# ---------------------------------------------------------------- PCO kernel
@pytest.mark.parametrize("seed,nl,nr,d,chil,chir", [
    (0, 2, 3, 4, 12, 15), (1, 0, 2, 5, 1, 20), (2, 3, 0, 3, 25, 1), (3, 4, 4, 6, 70, 90),
    (4, 1, 1, 8, 33, 47), (5, 0, 0, 7, 1, 1)])
def test_build_site_matches_oracle(ctx, seed, nl, nr, d, chil, chir):
    r = np.random.default_rng(seed)
    n = nl + 1 + nr
    Q = (r.standard_normal((n, n)) + 1j * r.standard_normal((n, n))) * 0.35
    Q = 0.5 * (Q + Q.T)
    bl = B.kept_basis(np.sort(r.uniform(0.05, 0.4, nl))[::-1], chil) if nl else M.vacuum_basis()
    br = B.kept_basis(np.sort(r.uniform(0.05, 0.4, nr))[::-1], chir) if nr else M.vacuum_basis()
    ref = P.local_tensor(Q, bl, br, d, c=0.7)
    got = g.gbsmps_build_site(ctx.h, Q, 0.7, bl.occ.astype(np.uint8).reshape(bl.D, nl),
                              br.occ.astype(np.uint8).reshape(br.D, nr), d)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    # parity (P6): odd-total entries are exactly zero on the GPU too
    tot = bl.occ.sum(1)[:, None, None] + np.arange(d)[None, :, None] + br.occ.sum(1)[None, None, :]
    assert np.all(got[tot % 2 == 1] == 0)


def test_build_site_vs_hafnian(ctx):
    r = np.random.default_rng(11)
    n = 4
    Q = (r.standard_normal((n, n)) + 1j * r.standard_normal((n, n))) * 0.5
    Q = 0.5 * (Q + Q.T)
    bl = B.kept_basis(np.array([0.3]), 6)
    br = B.kept_basis(np.array([0.35, 0.12]), 10)
    got = g.gbsmps_build_site(ctx.h, Q, 1.0, bl.occ.astype(np.uint8), br.occ.astype(np.uint8), 5)
    for a in range(bl.D):
        for p in range(5):
            for b in range(br.D):
                ex = H.local_entry(Q, np.r_[bl.occ[a], p, br.occ[b]])
                assert abs(got[a, p, b] - ex) <= 1e-12 * max(1.0, abs(ex))


# ---------------------------------------------------------------- whole build
SMALL = [  # (N, seed, d, chi, depth, rlo, rhi, haar)
    (2, 1, 6, 20, 1, 0.3, 0.6, False),
    (6, 2, 4, 30, 4, 0.1, 0.5, False),
    (12, 3, 4, 40, 6, 0.1, 0.5, False),
    (20, 4, 5, 64, 6, 0.1, 0.4, False),
    (8, 20251210, 8, 64, 0, 0.3, 0.8, True),
]


def _oracle(w, chi, d, eps=0.0, freeze=1e-13):
    mps = M.build_mps(w.gamma, d=d, chi=chi, eps=eps, lambda2_freeze=freeze)
    return mps, M.normalise(mps.tensors)


@pytest.mark.parametrize("case", SMALL)
def test_build_parity(ctx, case):
    N, seed, d, chi, depth, rlo, rhi, haar = case
    w = wl.small(N, seed, d=d, chi=chi, depth=depth, rlo=rlo, rhi=rhi, haar=haar)
    # the workloads' freeze threshold 1e-9, or the first one above it that no
    # symplectic eigenvalue sits on (the active-mode count is then the same
    # for any FP64 eigensolver).  An active mode with Lambda^2 ~ freeze is
    # nearly degenerate with the frozen ones (gap ~ 2 Lambda^2), so any FP64
    # eigensolver fixes its eigenvector only to ~1e-16 / (2 Lambda^2); the
    # amplitude floor is measured as the spread of two valid oracle routes.
    for freeze in (1e-9, 1e-8, 1e-7):
        omps, oT = _oracle(w, chi, d, freeze=freeze)
        if unambiguous(omps.cuts, freeze):
            break
    assert unambiguous(omps.cuts, freeze)
    alt = M.normalise(M.build_mps(w.gamma, d=d, chi=chi, lambda2_freeze=freeze,
                                  route=G.williamson_sqrt).tensors)
    m = g.MPS.from_cov(ctx, np.ascontiguousarray(w.gamma), d=d, chi_max=chi, lambda2_freeze=freeze)
    try:
        info = m.info
        assert list(info["n_e"]) == omps.n_e
        assert list(info["bond_dims"]) == omps.bond_dims
        assert np.allclose(info["eps"], omps.eps, rtol=1e-6, atol=1e-13)
        lam2, Qm, cm = g.gbsmps_get_gsvd(m.h)
        for k, cut in enumerate(omps.cuts[:-1]):
            assert np.allclose(lam2[k, :cut.n_out], cut.lam2, rtol=1e-9, atol=1e-13)
        gT = m.tensors()
        # gauge-invariant state fidelity
        f = M.fidelity(gT, oT)
        assert f >= 1 - 1e-10
        # amplitudes on all low patterns (tiny N) or sampled patterns, odd
        # totals and n_i >= d included
        pats = all_kinds_of_patterns(N, d, seed, full=N <= 8)
        ref = M.amplitudes(oT, pats)
        fl = route_floor(ref, M.amplitudes(alt, pats), N, max(omps.bond_dims))
        got = m.amplitudes(pats)
        assert amp_close(got, ref, floor=fl)
        zero = (pats.astype(int).sum(1) % 2 == 1) | (pats >= d).any(1)
        assert zero.sum() >= 3 and np.all(got[zero] == 0)
        # oracle amplitudes from the GPU's own tensors agree too
        assert amp_close(M.amplitudes(gT, pats), ref, floor=fl)
    finally:
        m.release()


def test_tensors_entrywise_canonical_gauge(ctx):
    """With well-separated symplectic spectra the canonical gauge makes the
    tensors themselves comparable entry by entry."""
    w = wl.small(10, 7, d=4, chi=48, depth=4, rlo=0.3, rhi=0.6)
    omps, oT = _oracle(w, 48, 4, freeze=1e-6)
    m = g.MPS.from_cov(ctx, np.ascontiguousarray(w.gamma), d=4, chi_max=48, lambda2_freeze=1e-6)
    try:
        for site in range(10):
            a = m.tensor(site)
            b = oT[site]
            assert a.shape == b.shape
            assert np.abs(a - b).max() <= 1e-9 * np.abs(b).max()
    finally:
        m.release()


def tie_state():
    """Two two-mode squeezed pairs, (0, 2) with Lambda^2 = 0.04 and (1, 3)
    with Lambda^2 = 0.2, both crossing the cut after mode 1.  Their
    entanglement energies w = -ln Lambda^2 satisfy w(0.04) = 2 w(0.2), so
    E(0,1) = E(2,0), E(1,1) = E(3,0) and E(0,2) = E(2,1) = E(4,0) on bond 2:
    exact ties, ordered lexicographically by occupation (reading A3)."""
    r1, r2 = np.arctanh(0.2), np.arctanh(np.sqrt(0.2))
    U = np.zeros((4, 4), dtype=np.complex128)
    for a, b in ((0, 2), (1, 3)):
        U[np.ix_([a, b], [a, b])] = np.array([[1, -1], [1, 1]]) / np.sqrt(2)
    gamma, q = wl.squeezed_state(np.array([r1, r2, -r1, -r2]), U)
    return gamma, q


@pytest.mark.parametrize("chi", [3, 4, 5, 7, 9])
def test_exact_energy_ties(ctx, chi):
    """chi cuts inside or at the edge of a tie group on bond 2: the GPU keeps
    the same occupation vectors in the same order as the oracle (checked
    through the tensor entries, which depend on which states are kept and
    where), with equal bond dimensions and truncation errors."""
    gamma, q = tie_state()
    d = 6
    omps = M.build_mps(gamma, d=d, chi=chi)
    lam = omps.cuts[1].lam2
    assert abs(lam[0] - 0.2) < 1e-12 and abs(lam[1] - 0.04) < 1e-12
    oT = M.normalise(omps.tensors)
    occ = [tuple(int(x) for x in o) for o in omps.bases[2].occ]
    assert occ[:3] == [(0, 0), (1, 0), (0, 1)]          # the tie (0,1) vs (2,0)
    m = g.MPS.from_cov(ctx, np.ascontiguousarray(gamma), d=d, chi_max=chi)
    try:
        assert list(m.info["bond_dims"]) == omps.bond_dims
        assert list(m.info["n_e"]) == omps.n_e
        assert np.allclose(m.info["eps"], omps.eps, rtol=1e-12, atol=1e-15)
        for site in range(4):
            a, b = m.tensor(site), oT[site]
            assert a.shape == b.shape
            assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max(), site
        pats = np.array(list(itertools.product(range(d), repeat=4)), dtype=np.uint8)
        ref = M.amplitudes(oT, pats)
        assert amp_close(m.amplitudes(pats), ref, floor=1e-13)
    finally:
        m.release()


def test_hafnian_pin_through_gpu(ctx):
    w = wl.small(4, 12, d=8, depth=4, rlo=0.1, rhi=0.3, haar=True)
    m = g.MPS.from_cov(ctx, np.ascontiguousarray(w.gamma), d=8, chi_max=300)
    try:
        pats = np.array([p for p in itertools.product(range(4), repeat=4) if sum(p) % 2 == 0],
                        dtype=np.uint8)
        got = m.amplitudes(pats)
        ex = np.array([H.amplitude(w.Q, p) for p in pats])
        r_got = got / got[0]
        r_ex = ex / ex[0]
        assert np.abs(r_got - r_ex).max() <= 1e-10 * np.abs(r_ex).max()
    finally:
        m.release()


def test_build_from_q_matches_cov(ctx):
    w = wl.small(10, 5, d=4, chi=40, depth=5)
    m1 = g.MPS.from_cov(ctx, np.ascontiguousarray(w.gamma), d=4, chi_max=40)
    m2 = g.MPS.from_Q(ctx, np.ascontiguousarray(w.Q), d=4, chi_max=40)
    try:
        assert list(m1.info["bond_dims"]) == list(m2.info["bond_dims"])
        f = M.fidelity(m1.tensors(), m2.tensors())
        assert f >= 1 - 1e-10
    finally:
        m1.release()
        m2.release()


@pytest.mark.parametrize("N,seed,chi", [(6, 2, 30), (16, 9, 48)])
def test_samples_bit_exact(ctx, N, seed, chi):
    w = wl.small(N, seed, d=4, chi=chi, depth=4, rlo=0.2, rhi=0.6)
    omps, oT = _oracle(w, chi, 4)
    m = g.MPS.from_cov(ctx, np.ascontiguousarray(w.gamma), d=4, chi_max=chi)
    try:
        S = 3000
        u = wl.uniforms(S, N, seed=seed + 100)
        flags = np.zeros(S, dtype=np.uint8)
        got = m.sample(S, uniforms=u, flags=flags)
        ref, rflag = M.sample(oT, u)
        ok = (flags == 0) & (~rflag)
        assert ok.mean() > 0.99
        assert np.array_equal(got[ok], ref[ok])
        assert np.all(got.astype(int).sum(1) % 2 == 0)       # P6 on samples
    finally:
        m.release()


def test_rejects_mixed_and_asymmetric(ctx):
    w = wl.small(6, 3, d=4, chi=20, depth=4)
    mixed = 0.8 * w.gamma + 0.2 * 0.5 * np.eye(12)
    with pytest.raises(g.GbsmpsError) as e:
        g.MPS.from_cov(ctx, np.ascontiguousarray(mixed), d=4, chi_max=20)
    assert e.value.code == g.ERR_NOT_PURE
    asym = w.gamma.copy()
    asym[0, 1] += 1e-6
    with pytest.raises(g.GbsmpsError) as e:
        g.MPS.from_cov(ctx, np.ascontiguousarray(asym), d=4, chi_max=20)
    assert e.value.code == g.ERR_NOT_SYMMETRIC
    # the context stays usable after an error
    m = g.MPS.from_cov(ctx, np.ascontiguousarray(w.gamma), d=4, chi_max=20)
    m.release()


def test_edge_cases(ctx):
    # single mode: no cut at all
    gam, q = wl.squeezed_state(np.array([0.4]), np.eye(1, dtype=np.complex128))
    m = g.MPS.from_cov(ctx, np.ascontiguousarray(gam), d=10, chi_max=4)
    try:
        a = m.tensor(0)[0, :, 0]
        t = np.tanh(0.4)
        for k in range(5):
            ex = np.sqrt(1 / np.cosh(0.4)) * (-t) ** k * np.sqrt(float(np.prod(range(1, 2 * k + 1)))) / (2 ** k * float(np.prod(range(1, k + 1))))
            assert abs(a[2 * k] / a[0] - ex / np.sqrt(1 / np.cosh(0.4))) < 1e-12
        assert np.all(a[1::2] == 0)
    finally:
        m.release()
    # product state: every bond dimension 1
    gam, q = wl.squeezed_state(np.array([0.3, 0.5, 0.2]), np.eye(3, dtype=np.complex128))
    m = g.MPS.from_cov(ctx, np.ascontiguousarray(gam), d=6, chi_max=16)
    try:
        assert list(m.info["bond_dims"]) == [1, 1, 1, 1]
    finally:
        m.release()
    # empty batches are no-ops
    w = wl.small(5, 1, d=4, chi=16, depth=3)
    m = g.MPS.from_cov(ctx, np.ascontiguousarray(w.gamma), d=4, chi_max=16)
    try:
        assert m.amplitudes(np.zeros((0, 5), dtype=np.uint8)).shape == (0,)
        assert m.sample(0).shape == (0, 5)
        # patterns with n_i >= d give 0
        assert m.amplitudes(np.array([[4, 0, 0, 0, 0]], dtype=np.uint8))[0] == 0
    finally:
        m.release()


def test_full_size_n144(ctx):
    """The 144-mode brick-wall workload at d=6, chi=256: GSVD spectra and
    bond dimensions equal the oracle's; sampled sites' tensors equal the
    oracle's PCO build from the GPU's own Q^m and bases (gauge-free); the
    state is normalised and the vacuum amplitude positive."""
    w = wl.config("n144_d6_chi256")
    cuts = G.gsvd_chain(w.gamma, lambda2_freeze=w.freeze)
    assert unambiguous(cuts, w.freeze)
    m = g.MPS.from_cov(ctx, np.ascontiguousarray(w.gamma), d=6, chi_max=256, eps_trunc=w.eps,
                       lambda2_freeze=w.freeze)
    try:
        info = m.info
        assert list(info["n_e"]) == [c.n_out for c in cuts[:-1]]
        bases = [M.vacuum_basis()] + [B.kept_basis(c.lam2, 256, w.eps) for c in cuts[:-1]] + [M.vacuum_basis()]
        assert list(info["bond_dims"]) == [b.D for b in bases]
        lam2, Qm, cm = g.gbsmps_get_gsvd(m.h)
        for k, cut in enumerate(cuts[:-1]):
            assert np.allclose(lam2[k, :cut.n_out], cut.lam2, rtol=1e-9, atol=1e-13)
        for site in (0, 5, 71, 143):
            nl, nr = bases[site].ne, bases[site + 1].ne
            nq = nl + 1 + nr
            ref = P.local_tensor(Qm[site, :nq, :nq], bases[site], bases[site + 1], 6, cm[site])
            got = m.tensor(site)
            if site == 0:      # A^1 carries the global normalisation and phase
                k = np.argmax(np.abs(ref))
                ref = ref * (got.flat[k] / ref.flat[k])
            assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max()
        a0 = m.amplitudes(np.zeros((1, 144), dtype=np.uint8))[0]
        assert abs(a0.imag) < 1e-14 and a0.real > 0
        # physical sanity (not parity): the cutoff d = 6 and the truncation
        # renormalise the state, raising P(vac) by the discarded weight (~1e-3)
        pvac = np.linalg.det(w.gamma + 0.5 * np.eye(288)) ** -0.5
        assert abs(a0.real ** 2 - pvac) < 2e-2 * pvac
    finally:
        m.release()
