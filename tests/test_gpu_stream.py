"""Streamed build + sampling (gbsmps_build_sample_stream): the chain of state
k+1 runs beside the sampling of state k, and the rest of build k+1 waits for
that sampling.  The patterns must be byte-for-byte those of separate
gbsmps_build_from_cov + gbsmps_sample calls with the same Philox keys and
counters (the build is deterministic; the sampler's tiles do not depend on
how many SMs its persistent grid spans)."""
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
    rs = np.random.default_rng(5)
    out = []
    for i in range(4):
        N = int(rs.integers(10, 41))
        d = int(rs.choice([4, 6]))
        chi = int(rs.choice([16, 32, 64]))
        w = wl.small(N, 900 + i, d=d, chi=chi, depth=max(1, N // 6), rlo=0.1, rhi=0.5)
        prec = g.PREC_MIXED if i != 2 else g.PREC_FP64
        out.append((w, dict(d=d, chi_max=chi, eps_trunc=1e-12, lambda2_freeze=1e-8, precision=prec)))
    return out


def _separate(ctx, states, S, seeds, c0s):
    res = []
    for (w, o), sd, c0 in zip(states, seeds, c0s):
        m = g.MPS.from_cov(ctx, np.ascontiguousarray(w.gamma), **o)
        try:
            out = np.zeros((S, w.N), dtype=np.uint8)
            m.sample(S, seed=sd, counter0=c0, out=out)
        finally:
            m.release()
        res.append(out)
    return res


def test_stream_matches_separate_calls_host_and_device(ctx):
    import torch
    states = _states()
    S = 3000
    seeds = [11, 12, 13, 14]
    c0s = [0, 5000, 77, 123456]
    want = _separate(ctx, states, S, seeds, c0s)
    opts = [g.opts_default(**o) for _, o in states]
    # host memory (page-locked outputs: the copies stay asynchronous)
    gam_h = [np.ascontiguousarray(w.gamma) for w, _ in states]
    outs_h = [torch.zeros((S, w.N), dtype=torch.uint8).pin_memory() for w, _ in states]
    g.gbsmps_build_sample_stream(ctx.h, gam_h, opts, S, seeds, c0s, [o.numpy() for o in outs_h])
    for k in range(len(states)):
        assert np.array_equal(outs_h[k].numpy(), want[k]), f"state {k} (host memory)"
    # device memory, twice in a row (the call leaves nothing behind)
    gam_d = [torch.from_numpy(x).cuda() for x in gam_h]
    for rep in range(2):
        outs_d = [torch.zeros((S, w.N), dtype=torch.uint8, device="cuda") for w, _ in states]
        g.gbsmps_build_sample_stream(ctx.h, gam_d, opts, S, seeds, c0s, outs_d)
        for k in range(len(states)):
            assert np.array_equal(outs_d[k].cpu().numpy(), want[k]), f"state {k} (device, call {rep})"


def test_stream_bench_workload_matches_separate(ctx):
    """Two states of the 144-mode d=6 chi=256 workload: here the next chain
    really overlaps a long sampling (the sampler leaves one SM free)."""
    import torch
    w = wl.config("n144_d6_chi256")
    o = dict(d=w.d, chi_max=w.chi, eps_trunc=w.eps, lambda2_freeze=w.freeze, precision=g.PREC_MIXED)
    S = 20000
    gam = torch.from_numpy(np.ascontiguousarray(w.gamma)).cuda()
    want = []
    for sd in (3, 4):
        m = g.MPS.from_cov(ctx, gam, **o)
        try:
            out = torch.zeros((S, w.N), dtype=torch.uint8, device="cuda")
            m.sample(S, seed=sd, counter0=0, out=out)
            want.append(out.cpu().numpy())
        finally:
            m.release()
    outs = [torch.zeros((S, w.N), dtype=torch.uint8, device="cuda") for _ in range(2)]
    g.gbsmps_build_sample_stream(ctx.h, [gam, gam], [g.opts_default(**o)] * 2, S, [3, 4], [0, 0], outs)
    for k in range(2):
        assert np.array_equal(outs[k].cpu().numpy(), want[k]), f"state {k}"


def test_stream_empty_and_bad_arguments(ctx):
    g.gbsmps_build_sample_stream(ctx.h, [], [], 10, [], [], [])
    w = wl.small(8, 1, d=4, chi=8, depth=2)
    bad = g.opts_default(d=0)
    with pytest.raises(g.GbsmpsError):
        g.gbsmps_build_sample_stream(ctx.h, [np.ascontiguousarray(w.gamma)], [bad], 4, [1], [0],
                                     [np.zeros((4, 8), dtype=np.uint8)])


@pytest.mark.parametrize("knobs", [
    {"GBSMPS_STREAM_AHEAD": "1", "GBSMPS_STREAM_RESERVE": "0"},
    {"GBSMPS_STREAM_AHEAD": "5", "GBSMPS_STREAM_RESERVE": "76", "GBSMPS_STREAM_BUILD_PRIO": "1"},
])
def test_stream_knobs_keep_the_patterns(ctx, monkeypatch, knobs):
    """The stream's look-ahead, the SMs the sampler leaves free and the
    streams' priorities are scheduling choices: the patterns stay
    byte-for-byte those of separate calls."""
    states = _states()
    S = 2000
    seeds = [21, 22, 23, 24]
    c0s = [0, 1, 2, 3]
    want = _separate(ctx, states, S, seeds, c0s)
    for k, v in knobs.items():
        monkeypatch.setenv(k, v)
    opts = [g.opts_default(**o) for _, o in states]
    gam_h = [np.ascontiguousarray(w.gamma) for w, _ in states]
    outs = [np.zeros((S, w.N), dtype=np.uint8) for w, _ in states]
    g.gbsmps_build_sample_stream(ctx.h, gam_h, opts, S, seeds, c0s, outs)
    for k in range(len(states)):
        assert np.array_equal(outs[k], want[k]), f"state {k}"
