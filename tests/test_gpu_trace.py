"""Kernel tracing (gbsmps_trace, gbsmps_trace_read_kernel): CUDA-event timing
of the sampler GEMM and of the environment GEMM with their algorithmic work,
as bench.py reads them for its roofline objects."""
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


def test_trace_both_kernels(ctx):
    w = wl.small(24, 3, d=4, chi=32, depth=4, rlo=0.1, rhi=0.4)
    g.gbsmps_trace(ctx.h, True)
    try:
        m = g.MPS.from_cov(ctx, np.ascontiguousarray(w.gamma), d=4, chi_max=32, eps_trunc=1e-12,
                           lambda2_freeze=1e-8, precision=g.PREC_MIXED)
        try:
            m.sample(500, seed=1)
        finally:
            m.release()
        s = g.gbsmps_trace_read_kernel(ctx.h, 0)
        e = g.gbsmps_trace_read_kernel(ctx.h, 1)
        p = g.gbsmps_trace_read_kernel(ctx.h, 2)
        assert s["launches"] == g.gbsmps_trace_read(ctx.h)["launches"]
        # two sampler launches per site (pre-pass and rest), two environment
        # launches per site, one PCO launch for the whole state (24 sites:
        # one wave of CTAs)
        assert s["launches"] == 2 * w.N and e["launches"] == 2 * w.N
        assert p["launches"] == 1 and p["ms"] > 0
        for t in (s, e):
            assert t["ms"] > 0 and t["flops"] > 0 and t["bytes"] > 0
    finally:
        g.gbsmps_trace(ctx.h, False)
    with pytest.raises(g.GbsmpsError):
        g.gbsmps_trace_read_kernel(ctx.h, 3)
