"""The C-ABI library loads without a GPU and exports every entry point that
include/gbsmps.h declares; host-side argument checks return codes, not aborts."""
import ctypes as C
import os

import pytest

import paper_2512_10643_gb300 as g


def _built():
    return os.path.exists(g.LIB_PATH)


@pytest.mark.skipif(not _built(), reason="libgbsmps.so not built")
def test_header_symbols_exported():
    L = g.lib()
    syms = g.header_symbols()
    assert "gbsmps_build_from_cov" in syms and "gbsmps_sample" in syms
    missing = [s for s in syms if not hasattr(L, s)]
    assert missing == []


@pytest.mark.skipif(not _built(), reason="libgbsmps.so not built")
def test_host_side_errors_without_gpu():
    L = g.lib()
    o = g.opts_default()
    assert o.d == 4 and o.chi_max == 64 and o.precision == g.PREC_FP64
    assert L.gbsmps_opts_default(None) == g.ERR_ARG
    assert L.gbsmps_info(None, None, None, None, None, None) == g.ERR_ARG
    assert L.gbsmps_release(None) == g.ERR_ARG
    assert L.gbsmps_strerror(g.ERR_NOT_PURE).decode().startswith("covariance")
    h = C.c_void_p()
    assert L.gbsmps_create(0, None, None) == g.ERR_ARG
    # NULL context is rejected before any CUDA call
    assert L.gbsmps_build_from_cov(None, 4, None, 0, C.byref(o), C.byref(h)) == g.ERR_ARG


def test_product_path_has_no_oracle_dependency():
    """The product package never imports the oracle."""
    root = os.path.dirname(g.HERE)
    for dirpath, _, files in os.walk(g.HERE):
        for f in files:
            if f.endswith((".py", ".cu", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt
    assert os.path.isdir(os.path.join(root, "oracle"))
