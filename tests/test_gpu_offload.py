"""Out-of-core sampling (gbsmps_offload): the sampler planes of a
mixed-precision MPS move to pinned host memory and stream through a ring of
three device slots site by site.  The same kernels read the same numbers in
the same order, so the patterns and boundary flags must equal those of the
resident MPS byte for byte, from given uniforms and from in-kernel Philox,
for states shorter than the ring and at full size."""
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


@pytest.mark.parametrize("N,seed,chi,d", [(1, 3, 8, 4), (2, 4, 16, 6), (30, 12, 96, 6)])
def test_offloaded_sampling_equals_resident(ctx, N, seed, chi, d):
    w = wl.small(N, seed, d=d, chi=chi, depth=max(1, N // 5), rlo=0.1, rhi=0.45)
    opts = dict(d=d, chi_max=chi, eps_trunc=1e-12, lambda2_freeze=1e-9, precision=g.PREC_MIXED)
    m = g.MPS.from_cov(ctx, np.ascontiguousarray(w.gamma), **opts)
    try:
        S = 5000
        u = wl.uniforms(S, N, seed=seed + 1)
        f0 = np.zeros(S, dtype=np.uint8)
        a0 = m.sample(S, uniforms=u, flags=f0)
        p0 = m.sample(S, seed=21, counter0=7)
        info = dict(m.info)
        m.offload()
        m.offload()                                    # a second call is a no-op
        f1 = np.zeros(S, dtype=np.uint8)
        a1 = m.sample(S, uniforms=u, flags=f1)
        p1 = m.sample(S, seed=21, counter0=7)
        assert np.array_equal(a0, a1) and np.array_equal(f0, f1)
        assert np.array_equal(p0, p1)
        assert np.array_equal(m.info["bond_dims"], info["bond_dims"])
        with pytest.raises(g.GbsmpsError) as e:
            m.tensor(0)
        assert e.value.code == g.ERR_STATE
        with pytest.raises(g.GbsmpsError) as e:
            m.amplitudes(np.zeros((1, N), dtype=np.uint8))
        assert e.value.code == g.ERR_STATE
    finally:
        m.release()


def test_offloaded_sampling_full_size(ctx):
    """144-mode workload, 100,000 samples: byte-identical patterns."""
    torch = pytest.importorskip("torch")
    w = wl.config("n144_d6_chi256")
    m = g.MPS.from_cov(ctx, np.ascontiguousarray(w.gamma), d=w.d, chi_max=w.chi, eps_trunc=w.eps,
                       lambda2_freeze=w.freeze, precision=g.PREC_MIXED)
    try:
        S = 100_000
        a = torch.empty((S, w.N), dtype=torch.uint8, device="cuda:0")
        b = torch.empty_like(a)
        m.sample(S, seed=5, counter0=0, out=a)
        m.offload()
        m.sample(S, seed=5, counter0=0, out=b)
        torch.cuda.synchronize()
        assert torch.equal(a, b)
    finally:
        m.release()


def test_offload_rejects_fp64(ctx):
    w = wl.small(6, 2, d=4, chi=16)
    m = g.MPS.from_cov(ctx, np.ascontiguousarray(w.gamma), d=4, chi_max=16)
    try:
        with pytest.raises(g.GbsmpsError) as e:
            m.offload()
        assert e.value.code == g.ERR_ARG
        m.tensor(0)                                   # still resident
    finally:
        m.release()


@pytest.mark.parametrize("offload", [False, True])
def test_chunked_sampling_equals_one_chunk(ctx, monkeypatch, offload):
    """Samples are processed in chunks (GBSMPS_SAMPLE_CHUNK caps their size);
    every sample's arithmetic is its own and its Philox counter is its global
    index, so the patterns do not depend on the chunking, resident or
    offloaded (an offloaded MPS streams its planes once per chunk)."""
    w = wl.small(24, 8, d=6, chi=64, depth=5, rlo=0.1, rhi=0.45)
    m = g.MPS.from_cov(ctx, np.ascontiguousarray(w.gamma), d=6, chi_max=64, eps_trunc=1e-12,
                       lambda2_freeze=1e-9, precision=g.PREC_MIXED)
    try:
        if offload:
            m.offload()
        S = 3000
        u = wl.uniforms(S, 24, seed=81)
        monkeypatch.delenv("GBSMPS_SAMPLE_CHUNK", raising=False)
        f1 = np.zeros(S, dtype=np.uint8)
        a = m.sample(S, uniforms=u, flags=f1)
        p = m.sample(S, seed=3, counter0=11)
        monkeypatch.setenv("GBSMPS_SAMPLE_CHUNK", "700")
        f2 = np.zeros(S, dtype=np.uint8)
        b = m.sample(S, uniforms=u, flags=f2)
        q = m.sample(S, seed=3, counter0=11)
        assert np.array_equal(a, b) and np.array_equal(f1, f2) and np.array_equal(p, q)
    finally:
        m.release()
