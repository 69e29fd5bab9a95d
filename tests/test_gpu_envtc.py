"""Environment products on the tensor cores (exact accumulation of bf16
integer slices) against the double-float products on the FP32 pipes: the same
mixed-precision single build with GBSMPS_ENV_TC=1 (the default) and =0.

Both compute R_m = sum_p Ahat[p] R_{m+1} Ahat[p]^dag (Sec. II B, the
normalisation of the MPS) to about 44 bits per step, so their difference is a
rounding-level spread, far below the FP32 PCO passes that set the mixed path's
error against FP64 (7e-9 of the largest amplitude at N = 144): canonical
tensors, amplitudes and samples drawn from shared uniforms are compared."""
import numpy as np
import pytest

import paper_2512_10643_gb300 as g
import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = g.Context(0)
    yield c
    c.close()


def _states():
    rs = np.random.default_rng(11)
    out = []
    for i in range(7):
        N = int(rs.integers(8, 41))
        d = int(rs.choice([4, 6]))
        chi = int(rs.choice([16, 32, 64]))
        w = wl.small(N, 700 + i, d=d, chi=chi, depth=max(1, N // 8), rlo=0.1, rhi=0.5)
        out.append((w, dict(d=d, chi_max=chi, eps_trunc=1e-12, lambda2_freeze=1e-8,
                            precision=g.PREC_MIXED)))
    w = wl.config("n144_d6_chi256")
    out.append((w, dict(d=w.d, chi_max=w.chi, eps_trunc=w.eps, lambda2_freeze=w.freeze,
                        precision=g.PREC_MIXED)))
    w1 = wl.small(1, 5, d=4, chi=4, depth=1)          # one mode: no environment product
    out.append((w1, dict(d=4, chi_max=4, precision=g.PREC_MIXED)))
    return out


def _build(ctx, w, opts, monkeypatch, tc):
    monkeypatch.setenv("GBSMPS_ENV_TC", "1" if tc else "0")
    return g.MPS.from_cov(ctx, np.ascontiguousarray(w.gamma), **opts)


def test_tensor_core_environments_match_double_float(ctx, monkeypatch):
    worst = {"tensor": 0.0, "amp": 0.0}
    for k, (w, opts) in enumerate(_states()):
        mt = _build(ctx, w, opts, monkeypatch, True)
        md = _build(ctx, w, opts, monkeypatch, False)
        try:
            assert np.array_equal(mt.info["bond_dims"], md.info["bond_dims"])
            for m in range(0, w.N, max(1, w.N // 24)):
                tt, td = mt.tensor(m), md.tensor(m)
                err = np.abs(tt - td).max() / max(np.abs(td).max(), 1e-300)
                worst["tensor"] = max(worst["tensor"], err)
                assert err <= 1e-8, (w.N, m, err)
            pats = wl.random_patterns(200, w.N, opts["d"], seed=k, max_total=8)
            pats[0] = 0
            at, ad = mt.amplitudes(pats), md.amplitudes(pats)
            at = at.cpu().numpy() if hasattr(at, "cpu") else np.asarray(at)
            ad = ad.cpu().numpy() if hasattr(ad, "cpu") else np.asarray(ad)
            err = np.abs(at - ad).max() / np.abs(ad).max()
            worst["amp"] = max(worst["amp"], err)
            assert err <= 1e-10, (w.N, err)
            u = wl.uniforms(2000, w.N, seed=50 + k)
            ft = np.zeros(2000, np.uint8)
            fd = np.zeros(2000, np.uint8)
            st = mt.sample(2000, uniforms=u, flags=ft)
            sd = md.sample(2000, uniforms=u, flags=fd)
            st = st.cpu().numpy() if hasattr(st, "cpu") else np.asarray(st)
            sd = sd.cpu().numpy() if hasattr(sd, "cpu") else np.asarray(sd)
            ok = (ft == 0) & (fd == 0)
            assert ok.mean() > 0.95
            assert np.array_equal(st[ok], sd[ok])
        finally:
            mt.release()
            md.release()
    print("tensor-core vs double-float environments, largest relative differences:", worst)


@pytest.mark.parametrize("mode,bound", [("0", 5e-13), ("1", 1e-11), ("2", 3e-11)])
def test_chain_accuracy_against_fp64(ctx, monkeypatch, mode, bound):
    """The environment chain's own error: a mixed build whose PCO passes run
    in FP64 (GBSMPS_PCO_FP64=1) against the FP64 build of the 144-mode
    workload, largest amplitude difference over the largest amplitude
    (the vacuum amplitude carries the norm).  Measured: double-float products
    6.8e-14, tensor cores 1.2e-12 (48-column tiles) and 5.3e-12 (64-column
    tiles); the FP32 PCO passes of a default mixed build add 7.0e-9 on top."""
    w = wl.config("n144_d6_chi256")
    base = dict(d=w.d, chi_max=w.chi, eps_trunc=w.eps, lambda2_freeze=w.freeze)
    pats = wl.random_patterns(300, w.N, w.d, seed=11, max_total=8)
    pats[0] = 0
    m64 = g.MPS.from_cov(ctx, np.ascontiguousarray(w.gamma), **dict(base, precision=g.PREC_FP64))
    try:
        a64 = np.asarray(m64.amplitudes(pats))
    finally:
        m64.release()
    monkeypatch.setenv("GBSMPS_PCO_FP64", "1")
    monkeypatch.setenv("GBSMPS_ENV_TC", mode)
    m = g.MPS.from_cov(ctx, np.ascontiguousarray(w.gamma), **dict(base, precision=g.PREC_MIXED))
    try:
        a = np.asarray(m.amplitudes(pats))
    finally:
        m.release()
    err = np.abs(a - a64).max() / np.abs(a64).max()
    print(f"environment products mode {mode}: mixed (FP64 PCO) vs FP64 amplitudes {err:.3e}")
    assert err <= bound


@pytest.mark.parametrize("N,d,chi,seed", [(2, 2, 1, 1), (2, 3, 2, 2), (3, 8, 4, 3), (4, 2, 8, 4),
                                          (5, 3, 3, 5), (6, 8, 8, 6), (6, 4, 5, 7)])
def test_tiny_and_odd_shapes(ctx, monkeypatch, N, d, chi, seed):
    """Products far below a tile (one or two rows and columns, K of 1 to a
    few dozen, odd K), photon cutoffs 2, 3 and 8 and bond dimension 1: the
    tensor-core environments agree with the double-float ones like the
    larger states (amplitudes within 1e-10 of the largest)."""
    w = wl.small(N, 900 + seed, d=d, chi=chi, depth=2, rlo=0.2, rhi=0.6)
    opts = dict(d=d, chi_max=chi, eps_trunc=1e-12, lambda2_freeze=1e-8, precision=g.PREC_MIXED)
    mt = _build(ctx, w, opts, monkeypatch, True)
    md = _build(ctx, w, opts, monkeypatch, False)
    try:
        pats = wl.random_patterns(64, N, d, seed=seed, max_total=6)
        pats[0] = 0
        at, ad = np.asarray(mt.amplitudes(pats)), np.asarray(md.amplitudes(pats))
        assert np.abs(at - ad).max() <= 1e-10 * np.abs(ad).max()
        for m in range(N):
            assert np.abs(mt.tensor(m) - md.tensor(m)).max() <= 1e-8 * np.abs(md.tensor(m)).max()
    finally:
        mt.release()
        md.release()
