"""Serving on the GPU: requests of different N, chi, d and precision run
concurrently on the server's slots; every result must equal the same request
run alone through the direct entry points (the kernels are deterministic, so
equality is bitwise), and the memory accounting must return to zero."""
import numpy as np
import pytest

import paper_2512_10643_gb300 as g
import workloads as wl

pytestmark = pytest.mark.gpu


def _requests():
    rs = np.random.default_rng(7)
    out = []
    for i in range(8):
        N = int(rs.integers(12, 41))
        d = int(rs.choice([4, 6]))
        chi = int(rs.choice([16, 32, 64]))
        prec = g.PREC_MIXED if i % 2 else g.PREC_FP64
        S = int(rs.integers(300, 2500))
        w = wl.small(N, 900 + i, d=d, chi=chi, depth=max(1, N // 8), rlo=0.1, rhi=0.4)
        opts = dict(d=d, chi_max=chi, eps_trunc=1e-12, lambda2_freeze=1e-9, precision=prec)
        out.append((w, S, opts, 1000 + i))
    return out


def test_served_results_equal_alone():
    reqs = _requests()
    alone = []
    with g.Context(0) as ctx:
        for w, S, opts, seed in reqs:
            m = g.MPS.from_cov(ctx, np.ascontiguousarray(w.gamma), **opts)
            try:
                alone.append(m.sample(S, seed=seed, counter0=5))
            finally:
                m.release()
    with g.Server(0, slots=4) as srv:
        ids = [srv.submit(w.gamma, S, seed=seed, counter0=5, **opts) for w, S, opts, seed in reqs[:3]]
        # later arrivals join while the first ones are on the device
        ids += [srv.submit(w.gamma, S, seed=seed, counter0=5, **opts) for w, S, opts, seed in reqs[3:]]
        res = [srv.wait(i, timeout_s=300) for i in ids]
        st = srv.stats()
    for (out, info), ref in zip(res, alone):
        assert info["state"] == 2
        assert np.array_equal(out, ref)
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["hbm_in_use"] == 0 and st["hbm_peak"] <= st["hbm_budget"]
    infos = [i for _, i in res]
    overlap = max(sum(1 for y in infos if y["t_admit"] <= x["t_admit"] < y["t_done"]) for x in infos)
    assert overlap >= 2                      # jobs shared the GPU
    assert len({i["slot"] for i in infos}) >= 2


def test_failed_request_reports_and_server_continues():
    w = wl.small(10, 3, d=4, chi=16)
    bad = np.array(w.gamma)
    bad[0, 1] += 1e-3                         # not symmetric
    with g.Server(0, slots=2) as srv:
        a = srv.submit(bad, 100, d=4, chi_max=16, validate=1)
        b = srv.submit(w.gamma, 100, d=4, chi_max=16)
        with pytest.raises(g.GbsmpsError) as e:
            srv.wait(a, 120)
        assert e.value.code == g.ERR_NOT_SYMMETRIC
        out, info = srv.wait(b, 120)
        assert info["state"] == 2 and out.shape == (100, 10)
        assert srv.stats()["failed"] == 1


def test_batched_serving_within_tolerance():
    """batch_max > 1: queued requests are built together in one batched call.
    The batch sums the environment products in another order, so a result
    equals the request run alone up to rounding: samples bit-exact except
    draws that either side flags at a CDF boundary."""
    reqs = _requests()
    alone = []
    with g.Context(0) as ctx:
        for w, S, opts, seed in reqs:
            m = g.MPS.from_cov(ctx, np.ascontiguousarray(w.gamma), **opts)
            try:
                f = np.zeros(S, dtype=np.uint8)
                alone.append((m.sample(S, seed=seed, counter0=5, flags=f), f))
            finally:
                m.release()
    with g.Server(0, slots=1, batch_max=8) as srv:
        ids = [srv.submit(w.gamma, S, seed=seed, counter0=5, **opts) for w, S, opts, seed in reqs]
        res = [srv.wait(i, timeout_s=300) for i in ids]
        st = srv.stats()
    assert st["completed"] == len(reqs) and st["hbm_in_use"] == 0
    assert max(info["batch"] for _, info in res) >= 2           # batches formed
    for (out, info), (ref, rf) in zip(res, alone):
        ok = (info["flags"] == 0) & (rf == 0)
        assert ok.mean() > 0.97
        assert np.array_equal(out[ok], ref[ok])
        assert np.all(out.astype(int).sum(1) % 2 == 0)
