"""The 1024-mode workload (r~U(0.05,0.25), brick-wall depth 32, d=4, chi=512)
in mixed precision, at full size: the GSVD spectra, active-mode counts and
bond dimensions equal the oracle's for every cut; sampled sites' tensors equal
the oracle's PCO build from the GPU's own Q^m and bases; the state is
normalised with a positive vacuum amplitude; and the samples obey what holds
at any size: even total photon number, and per-mode mean photon numbers that
match the covariance, <n_i> = (Gamma_{x_i x_i} + Gamma_{p_i p_i} - 1) / 2."""
import numpy as np
import pytest

import paper_2512_10643_gb300 as g
import workloads as wl
from oracle import basis as B
from oracle import gaussian as G
from oracle import mps as M
from oracle import pco as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = g.Context(0)
    yield c
    c.close()


def test_full_size_n1024(ctx):
    w = wl.config("n1024_d4_chi512")
    N, d, chi = w.N, w.d, w.chi
    freeze = None
    for f in (w.freeze, 1e-8, 1e-7):
        cuts = G.gsvd_chain(w.gamma, lambda2_freeze=f)
        if all(not np.any(np.abs((c.D - 1) / (c.D + 1) - f) <= 1e-14 + 1e-3 * f) for c in cuts[:-1]):
            freeze = f
            break
    assert freeze is not None
    m = g.MPS.from_cov(ctx, np.ascontiguousarray(w.gamma), d=d, chi_max=chi, eps_trunc=w.eps,
                       lambda2_freeze=freeze, precision=g.PREC_MIXED)
    try:
        info = m.info
        assert list(info["n_e"]) == [c.n_out for c in cuts[:-1]]
        bases = ([M.vacuum_basis()] + [B.kept_basis(c.lam2, chi, w.eps) for c in cuts[:-1]]
                 + [M.vacuum_basis()])
        assert list(info["bond_dims"]) == [b.D for b in bases]
        lam2, Qm, cm = g.gbsmps_get_gsvd(m.h)
        for k, cut in enumerate(cuts[:-1]):
            assert np.allclose(lam2[k, :cut.n_out], cut.lam2, rtol=1e-9, atol=1e-13)
        for site in (0, 1, 511, 1022, 1023):
            nl, nr = bases[site].ne, bases[site + 1].ne
            nq = nl + 1 + nr
            ref = P.local_tensor(Qm[site, :nq, :nq], bases[site], bases[site + 1], d, cm[site])
            got = m.tensor(site)
            if site == 0:      # A^1 carries the global normalisation and phase
                k = np.argmax(np.abs(ref))
                ref = ref * (got.flat[k] / ref.flat[k])
            assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()   # mixed: FP32 PCO products
        a0 = m.amplitudes(np.zeros((1, N), dtype=np.uint8))[0]
        assert abs(a0.imag) < 1e-14 and a0.real > 0
        # sampling: properties that hold at any size
        S = 20000
        s = m.sample(S, seed=2026).astype(np.int64)
        assert np.all(s.sum(1) % 2 == 0)
        n_exp = 0.5 * (np.diag(w.gamma)[:N] + np.diag(w.gamma)[N:] - 1.0)
        mean = s.mean(0)
        # n_i takes mostly 0 and 2 here (pairs), so var(n_i) >= <n_i>
        se = np.sqrt(np.maximum(s.var(0), n_exp) / S)
        z = (mean - n_exp) / se
        assert np.abs(z).max() < 6.0
        tot_se = s.sum(1).std() / np.sqrt(S)
        assert abs(s.sum(1).mean() - n_exp.sum()) < 6 * tot_se + 1e-3 * n_exp.sum()
    finally:
        m.release()
