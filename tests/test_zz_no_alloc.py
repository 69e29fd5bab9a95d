"""The allocation-free single-site build gives the same tensor as the
allocating entry point, on consecutive calls that reuse its static working
memory.  (For callers that must not allocate device memory while they run:
pre-reserved serving processes, latency-critical loops, foreign allocators.)
Kept in the last-collected file so that a run that stops at the first failure
has already run every other test."""
import numpy as np
import pytest

from oracle import basis as B
from oracle import mps as M

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


def _case(seed, nl, nr, chil, chir):
    r = np.random.default_rng(seed)
    n = nl + 1 + nr
    Q = (r.standard_normal((n, n)) + 1j * r.standard_normal((n, n))) * 0.35
    Q = 0.5 * (Q + Q.T)
    bl = B.kept_basis(np.sort(r.uniform(0.05, 0.4, nl))[::-1], chil) if nl else M.vacuum_basis()
    br = B.kept_basis(np.sort(r.uniform(0.05, 0.4, nr))[::-1], chir) if nr else M.vacuum_basis()
    return (Q, bl.occ.astype(np.uint8).reshape(bl.D, nl),
            br.occ.astype(np.uint8).reshape(br.D, nr))


def test_no_alloc_matches_allocating_entry_twice(ctx):
    import torch
    dev = torch.device("cuda:0")
    # two different problems in a row: the second call reuses (and must fully
    # rewrite) the working memory left by the first
    for seed, nl, nr, d, chil, chir, c in ((0, 3, 4, 5, 90, 120, 0.8), (1, 2, 3, 6, 40, 64, 1.3)):
        Q, ol, orr = _case(seed, nl, nr, chil, chir)
        ref = g.gbsmps_build_site(ctx.h, Q, c, ol, orr, d)
        Qd = torch.from_numpy(np.ascontiguousarray(Q).view(np.float64).reshape(Q.shape + (2,))).to(dev)
        out = torch.full((ol.shape[0], d, orr.shape[0], 2), float("nan"), dtype=torch.float64, device=dev)
        g.gbsmps_build_site_noalloc(ctx.h, Qd, c, torch.from_numpy(ol).to(dev),
                                    torch.from_numpy(orr).to(dev), d, out)
        got = out.cpu().numpy().view(np.complex128)[..., 0]
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("precision", [0, 1])
def test_no_alloc_boundary_sites_and_precisions(ctx, precision):
    """A first site (no left modes: its occupation block is cleared in the
    static array instead of repacked), a last site (no right modes) and a
    middle site, in FP64 and in mixed precision (FP32 passes), each against
    the allocating entry in the same precision, two calls in a row."""
    import torch
    dev = torch.device("cuda:0")
    for seed, nl, nr, d, chil, chir, c in ((3, 0, 3, 6, 1, 70, 1.1), (4, 2, 0, 5, 50, 1, 0.9),
                                           (5, 2, 2, 4, 30, 30, 1.0)):
        Q, ol, orr = _case(seed, nl, nr, chil, chir)
        ref = g.gbsmps_build_site(ctx.h, Q, c, ol, orr, d, precision=precision)
        Qd = torch.from_numpy(np.ascontiguousarray(Q).view(np.float64).reshape(Q.shape + (2,))).to(dev)
        out = torch.full((ol.shape[0], d, orr.shape[0], 2), float("nan"), dtype=torch.float64, device=dev)
        g.gbsmps_build_site_noalloc(ctx.h, Qd, c, torch.from_numpy(ol).to(dev),
                                    torch.from_numpy(orr).to(dev), d, out, precision=precision)
        got = out.cpu().numpy().view(np.complex128)[..., 0]
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_no_alloc_rejects_sizes_beyond_its_limit(ctx):
    import torch
    dev = torch.device("cuda:0")
    Q, ol, orr = _case(2, 1, 1, 200, 10)
    assert ol.shape[0] > 128
    Qd = torch.from_numpy(np.ascontiguousarray(Q).view(np.float64).reshape(Q.shape + (2,))).to(dev)
    out = torch.zeros((ol.shape[0], 3, orr.shape[0], 2), dtype=torch.float64, device=dev)
    with pytest.raises(g.GbsmpsError) as e:
        g.gbsmps_build_site_noalloc(ctx.h, Qd, 1.0, torch.from_numpy(ol).to(dev),
                                    torch.from_numpy(orr).to(dev), 3, out)
    assert e.value.code == g.ERR_BOUNDS
