"""Mixed-precision path (FP32 PCO passes with FP64 plane sums, environments in
the energy gauge on the tensor cores with exact accumulation of bf16 integer
slices, split-FP16 tensor-core sampler in right-canonical form, FP64 Gaussian
SVD) against the FP64 oracle.
Tolerances: amplitude error <= 1e-5 relative (floor 1e-8 of the largest
amplitude), fidelity >= 1 - 1e-8, samples bit-exact except draws flagged
within 1e-5 Z of a CDF boundary."""
import numpy as np
import pytest

import workloads as wl
from oracle import basis as B
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


def mixed_close(a, b, rtol=1e-5, floor=1e-8):
    a, b = np.asarray(a), np.asarray(b)
    return bool(np.all(np.abs(a - b) <= rtol * np.abs(b) + floor * np.abs(b).max()))


@pytest.mark.parametrize("seed,nl,nr,d,chil,chir", [(0, 2, 3, 4, 12, 15), (3, 4, 4, 6, 70, 90)])
def test_fp32_pco_matches_oracle(ctx, seed, nl, nr, d, chil, chir):
    r = np.random.default_rng(seed)
    n = nl + 1 + nr
    Q = (r.standard_normal((n, n)) + 1j * r.standard_normal((n, n))) * 0.35
    Q = 0.5 * (Q + Q.T)
    bl = B.kept_basis(np.sort(r.uniform(0.05, 0.4, nl))[::-1], chil)
    br = B.kept_basis(np.sort(r.uniform(0.05, 0.4, nr))[::-1], chir)
    ref = P.local_tensor(Q, bl, br, d, c=1.0)
    got = g.gbsmps_build_site(ctx.h, Q, 1.0, bl.occ.astype(np.uint8), br.occ.astype(np.uint8), d,
                              precision=g.PREC_MIXED)
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()


@pytest.mark.parametrize("N,seed,chi,d", [(12, 3, 40, 4), (24, 4, 64, 5)])
def test_mixed_build_amplitudes_and_samples(ctx, N, seed, chi, d):
    w = wl.small(N, seed, d=d, chi=chi, depth=6, rlo=0.1, rhi=0.45)
    omps = M.build_mps(w.gamma, d=d, chi=chi, eps=1e-12, lambda2_freeze=1e-9)
    oT = M.normalise(omps.tensors)
    m = g.MPS.from_cov(ctx, np.ascontiguousarray(w.gamma), d=d, chi_max=chi, eps_trunc=1e-12,
                       lambda2_freeze=1e-9, precision=g.PREC_MIXED)
    try:
        assert list(m.info["bond_dims"]) == omps.bond_dims
        gT = m.tensors()
        assert M.fidelity(gT, oT) >= 1 - 1e-8
        pats = wl.random_patterns(300, N, d, seed=seed)
        assert mixed_close(m.amplitudes(pats), M.amplitudes(oT, pats))
        S = 4000
        u = wl.uniforms(S, N, seed=seed + 7)
        flags = np.zeros(S, dtype=np.uint8)
        got = m.sample(S, uniforms=u, flags=flags)
        ref, rflag = M.sample(oT, u)
        ok = flags == 0
        assert ok.mean() > 0.98
        assert np.array_equal(got[ok], ref[ok])
        assert np.all(got.astype(int).sum(1) % 2 == 0)
    finally:
        m.release()


def test_mixed_vs_fp64_gpu_full_size(ctx):
    """144 modes, d=6, chi=256: the mixed build and the FP64 build agree on
    the bond dimensions, amplitudes (1e-5) and, with shared uniforms, on the
    samples away from flagged boundaries."""
    w = wl.config("n144_d6_chi256")
    kw = dict(d=6, chi_max=256, eps_trunc=w.eps, lambda2_freeze=w.freeze)
    m64 = g.MPS.from_cov(ctx, np.ascontiguousarray(w.gamma), **kw)
    mmx = g.MPS.from_cov(ctx, np.ascontiguousarray(w.gamma), precision=g.PREC_MIXED, **kw)
    try:
        assert list(m64.info["bond_dims"]) == list(mmx.info["bond_dims"])
        pats = wl.random_patterns(200, 144, 6, seed=5)
        pats[0] = 0
        assert mixed_close(mmx.amplitudes(pats), m64.amplitudes(pats))
        S = 500
        u = wl.uniforms(S, 144, seed=11)
        f64 = np.zeros(S, dtype=np.uint8)
        fmx = np.zeros(S, dtype=np.uint8)
        s64 = m64.sample(S, uniforms=u, flags=f64)
        smx = mmx.sample(S, uniforms=u, flags=fmx)
        ok = (fmx == 0) & (f64 == 0)
        assert ok.mean() > 0.9
        assert np.array_equal(s64[ok], smx[ok])
    finally:
        m64.release()
        mmx.release()


def test_tcgen05_gemm_matches_simt_reference(ctx, monkeypatch):
    """The tcgen05/TMA sampler GEMM and a SIMT GEMM over the same packed
    split-FP16 planes draw the same samples from the same uniforms (only draws
    within the mixed boundary window may differ)."""
    w = wl.small(20, 6, d=5, chi=96, depth=6, rlo=0.2, rhi=0.5)
    m = g.MPS.from_cov(ctx, np.ascontiguousarray(w.gamma), d=5, chi_max=96, eps_trunc=1e-12,
                       lambda2_freeze=1e-9, precision=g.PREC_MIXED)
    try:
        S = 3000
        u = wl.uniforms(S, 20, seed=21)
        f_tc = np.zeros(S, dtype=np.uint8)
        f_rf = np.zeros(S, dtype=np.uint8)
        monkeypatch.setenv("GBSMPS_TC", "1")
        s_tc = m.sample(S, uniforms=u, flags=f_tc)
        monkeypatch.setenv("GBSMPS_TC", "0")
        s_rf = m.sample(S, uniforms=u, flags=f_rf)
        ok = (f_tc == 0) & (f_rf == 0)
        assert ok.mean() > 0.98
        assert np.array_equal(s_tc[ok], s_rf[ok])
        # in-kernel Philox path draws valid patterns too
        monkeypatch.setenv("GBSMPS_TC", "1")
        s_ph = m.sample(S, seed=5)
        assert np.all(s_ph.astype(int).sum(1) % 2 == 0)
    finally:
        m.release()



def test_p0_prepass_draws_the_full_pass_patterns(ctx, monkeypatch):
    """The p = 0 pre-pass multiplies only block 0 of every sample and decides
    p = 0 when u < q_0 - 1e-5 (sum_p q_p = |vt|^2 = 1 in right-canonical
    form); everything else goes through the full pass.  From the same
    uniforms it must draw exactly the patterns of the single full pass,
    except draws the full pass flags."""
    w = wl.small(30, 12, d=6, chi=96, depth=6, rlo=0.1, rhi=0.45)
    m = g.MPS.from_cov(ctx, np.ascontiguousarray(w.gamma), d=6, chi_max=96, eps_trunc=1e-12,
                       lambda2_freeze=1e-9, precision=g.PREC_MIXED)
    try:
        S = 6000
        u = wl.uniforms(S, 30, seed=44)
        f_full = np.zeros(S, dtype=np.uint8)
        f_pre = np.zeros(S, dtype=np.uint8)
        monkeypatch.setenv("GBSMPS_P0PASS", "0")
        s_full = m.sample(S, uniforms=u, flags=f_full)
        monkeypatch.setenv("GBSMPS_P0PASS", "1")
        s_pre = m.sample(S, uniforms=u, flags=f_pre)
        ok = (f_full == 0) & (f_pre == 0)
        assert ok.mean() > 0.98
        assert np.array_equal(s_full[ok], s_pre[ok])
        assert np.all(s_pre.astype(int).sum(1) % 2 == 0)
        # the in-kernel Philox path as well, twice in a row
        a = m.sample(S, seed=9)
        b = m.sample(S, seed=9)
        assert np.array_equal(a, b)
        monkeypatch.setenv("GBSMPS_P0PASS", "0")
        c = m.sample(S, seed=9)
        assert (a == c).all(axis=1).mean() > 0.98
    finally:
        m.release()


def test_factor_paths_agree(ctx, monkeypatch):
    """The Cholesky factors and inverses of the environments' parity blocks
    come from one shared-memory double-float kernel when the blocks fit and
    from the FP64 global-memory kernels otherwise (GBSMPS_CHOL_SMEM=0 forces
    those): the same regulariser is chosen and the same samples are drawn
    from the same uniforms, except draws flagged at a CDF boundary."""
    w = wl.small(28, 17, d=6, chi=96, depth=6, rlo=0.1, rhi=0.45)
    opts = dict(d=6, chi_max=96, eps_trunc=1e-12, lambda2_freeze=1e-9, precision=g.PREC_MIXED)
    S = 4000
    u = wl.uniforms(S, 28, seed=71)
    res = []
    for flag in ("1", "0"):
        monkeypatch.setenv("GBSMPS_CHOL_SMEM", flag)
        m = g.MPS.from_cov(ctx, np.ascontiguousarray(w.gamma), **opts)
        try:
            f = np.zeros(S, dtype=np.uint8)
            res.append((m.sample(S, uniforms=u, flags=f), f))
        finally:
            m.release()
    (s1, f1), (s0, f0) = res
    ok = (f1 == 0) & (f0 == 0)
    assert ok.mean() > 0.98
    assert np.array_equal(s1[ok], s0[ok])
    assert np.all(s1.astype(int).sum(1) % 2 == 0)
