"""Batched build (gbsmps_build_batch): every state of a batch of uneven N,
chi, d and precision must match the same state built alone (the GSVD and PCO
stages run the same per-state arithmetic; only the environment products are
summed in another order) and the oracle.  A batch runs its environment chains
in double-float arithmetic, so the single builds it is compared with take the
double-float products too (GBSMPS_ENV_TC=0); test_gpu_envtc.py compares those
with the tensor-core products of a default single build."""
import numpy as np
import pytest

import paper_2512_10643_gb300 as g
import workloads as wl
from oracle import mps as OM

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = g.Context(0)
    yield c
    c.close()


def _freeze_for(w):
    """First freeze threshold that no symplectic eigenvalue sits on (the
    active-mode count is then the same for any FP64 eigensolver)."""
    from oracle import gaussian as G
    for freeze in (1e-8, 1e-7, 1e-6):
        cuts = G.gsvd_chain(w.gamma, lambda2_freeze=freeze)
        if all(not np.any(np.abs((c.D - 1) / (c.D + 1) - freeze) <= 1e-14 + 1e-3 * freeze)
               for c in cuts[:-1]):
            return freeze
    raise AssertionError("no unambiguous freeze threshold")


def _batch_states(precisions=(g.PREC_MIXED,)):
    rs = np.random.default_rng(11)
    out = []
    for i in range(7):
        N = int(rs.integers(8, 41))
        d = int(rs.choice([4, 6]))
        chi = int(rs.choice([16, 32, 64]))
        w = wl.small(N, 700 + i, d=d, chi=chi, depth=max(1, N // 8), rlo=0.1, rhi=0.5)
        opts = dict(d=d, chi_max=chi, eps_trunc=1e-12, lambda2_freeze=1e-8,
                    precision=precisions[i % len(precisions)])
        out.append((w, opts))
    # a one-mode state rides along
    w1 = wl.small(1, 5, d=4, chi=4, depth=1)
    out.append((w1, dict(d=4, chi_max=4, precision=precisions[0])))
    return out


@pytest.mark.parametrize("precisions", [(g.PREC_MIXED,), (g.PREC_MIXED, g.PREC_FP64)])
def test_batch_matches_single_builds(ctx, precisions, monkeypatch):
    monkeypatch.setenv("GBSMPS_ENV_TC", "0")
    states = _batch_states(precisions)
    batch = g.MPS.batch(ctx, [np.ascontiguousarray(w.gamma) for w, _ in states],
                        [o for _, o in states])
    try:
        for k, ((w, opts), mb) in enumerate(zip(states, batch)):
            ms = g.MPS.from_cov(ctx, np.ascontiguousarray(w.gamma), **opts)
            try:
                assert np.array_equal(mb.info["bond_dims"], ms.info["bond_dims"])
                assert np.array_equal(mb.info["n_e"], ms.info["n_e"])
                for m in range(w.N):
                    tb, ts = mb.tensor(m), ms.tensor(m)
                    assert np.abs(tb - ts).max() <= 1e-12 * max(np.abs(ts).max(), 1e-300)
                pats = wl.random_patterns(64, w.N, opts["d"], seed=k)
                pats[0] = 0
                ab, as_ = mb.amplitudes(pats), ms.amplitudes(pats)
                assert np.abs(ab - as_).max() <= 1e-11 * np.abs(as_).max()
                u = wl.uniforms(400, w.N, seed=50 + k)
                fb = np.zeros(400, np.uint8)
                fs = np.zeros(400, np.uint8)
                sb = mb.sample(400, uniforms=u, flags=fb)
                ss = ms.sample(400, uniforms=u, flags=fs)
                ok = (fb == 0) & (fs == 0)
                assert ok.mean() > 0.97
                assert np.array_equal(sb[ok], ss[ok])
            finally:
                ms.release()
    finally:
        for m in batch:
            m.release()


@pytest.mark.parametrize("prec", [g.PREC_MIXED, g.PREC_FP64])
def test_batch_against_oracle(ctx, prec):
    """FP64 states: fidelity 1e-10 and amplitudes 1e-9 of the largest.  Mixed
    states run the PCO products in FP32 (Eq. 17 with FP32 sums), so they are
    held to the mixed contract: amplitudes within 1e-6 of the largest (the
    contract allows 1e-5), fidelity 1 - 1e-8."""
    states = _batch_states((prec,))[:4]
    for w, o in states:
        o["lambda2_freeze"] = _freeze_for(w)
    batch = g.MPS.batch(ctx, [np.ascontiguousarray(w.gamma) for w, _ in states],
                        [o for _, o in states])
    try:
        for k, ((w, opts), mb) in enumerate(zip(states, batch)):
            ref = OM.build_mps(w.gamma, d=opts["d"], chi=opts["chi_max"], eps=opts["eps_trunc"],
                               lambda2_freeze=opts["lambda2_freeze"])
            assert list(mb.info["bond_dims"]) == ref.bond_dims
            T = OM.normalise(ref.tensors)
            fid_tol, amp_tol = (1e-10, 1e-9) if prec == g.PREC_FP64 else (1e-8, 1e-6)
            assert OM.fidelity(mb.tensors(), T) >= 1 - fid_tol
            pats = wl.random_patterns(48, w.N, opts["d"], seed=90 + k)
            pats[0] = 0
            got = mb.amplitudes(pats)
            want = OM.amplitudes(T, pats)
            assert np.abs(got - want).max() <= amp_tol * np.abs(want).max()
    finally:
        for m in batch:
            m.release()


def test_batch_edge_cases(ctx):
    assert g.gbsmps_build_batch(ctx.h, [], []) == []
    w = wl.small(10, 3, d=4, chi=16)
    bad = np.array(w.gamma)
    bad[0, 1] += 1e-3
    with pytest.raises(g.GbsmpsError) as e:
        g.MPS.batch(ctx, [np.ascontiguousarray(w.gamma), bad], [dict(d=4, chi_max=16)] * 2)
    assert e.value.code == g.ERR_NOT_SYMMETRIC
    # the context stays usable
    m = g.MPS.from_cov(ctx, np.ascontiguousarray(w.gamma), d=4, chi_max=16)
    m.release()


def test_env_tile_shapes_give_identical_results(ctx, monkeypatch):
    """The persistent environment chain sums every output in the same k order
    whatever its tile shape, so the autotuner's choice cannot change a bit."""
    states = _batch_states()[:5]
    gams = [np.ascontiguousarray(w.gamma) for w, _ in states]
    opts = [o for _, o in states]
    results = []
    for cfg in ("0", "1", "2"):
        monkeypatch.setenv("GBSMPS_ENV_TILE", cfg)
        batch = g.MPS.batch(ctx, gams, opts)
        try:
            res = []
            for k, ((w, o), m) in enumerate(zip(states, batch)):
                u = wl.uniforms(300, w.N, seed=7 + k)
                res.append((m.tensor(0), m.sample(300, uniforms=u)))
            results.append(res)
        finally:
            for m in batch:
                m.release()
    for other in results[1:]:
        for (t0, s0), (t1, s1) in zip(results[0], other):
            assert np.array_equal(t0, t1)
            assert np.array_equal(s0, s1)


def test_df64_tile_shapes_give_identical_results(ctx, monkeypatch):
    """The tile shape and the k depth of a shared-memory stage of the
    environment chain's grouped double-float launches (GBSMPS_ENV_TC=0)
    cannot change a bit: every output sums k in the same order, and the k
    split follows a fixed reference tiling, not the tile."""
    monkeypatch.setenv("GBSMPS_ENV_TC", "0")
    w = wl.small(24, 31, d=5, chi=64, depth=4, rlo=0.1, rhi=0.5)
    opts = dict(d=5, chi_max=64, eps_trunc=1e-12, lambda2_freeze=1e-8, precision=g.PREC_MIXED)
    u = wl.uniforms(300, 24, seed=3)
    res = []
    for cfg, sk in (("16", "16"), ("16", "8"), ("32", "8"), ("64", "8")):
        monkeypatch.setenv("GBSMPS_DFG_TILE", cfg)
        monkeypatch.setenv("GBSMPS_DFG_SK", sk)
        m = g.MPS.from_cov(ctx, np.ascontiguousarray(w.gamma), **opts)
        try:
            amp = m.amplitudes(np.zeros((1, 24), dtype=np.uint8))
            res.append((m.tensor(0), amp, m.sample(300, uniforms=u)))
        finally:
            m.release()
    for t, a, smp in res[1:]:
        assert np.array_equal(t, res[0][0])
        assert np.array_equal(a, res[0][1])
        assert np.array_equal(smp, res[0][2])
