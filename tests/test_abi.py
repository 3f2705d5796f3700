"""CPU-side checks of the C interface: the library builds, loads and exports every
function include/lddmm.h declares, and argument validation needs no GPU."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lddmm.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lddmm_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def so():
    from paper_1807_11560_gb300 import build, lddmm
    if not os.path.exists(lddmm.LIB_PATH):
        build.build()
    return ctypes.CDLL(lddmm.LIB_PATH)


def test_header_declares_the_method_calls():
    names = _declared()
    for n in ("lddmm_create", "lddmm_set_images", "lddmm_energy", "lddmm_gradient",
              "lddmm_hessvec", "lddmm_gn_solve", "lddmm_destroy", "lddmm_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(so):
    missing = [n for n in _declared() if not hasattr(so, n)]
    assert not missing, missing


def test_create_rejects_bad_sizes_without_touching_the_gpu(so):
    from paper_1807_11560_gb300 import lddmm
    L = lddmm.lib()
    h = ctypes.c_void_p()
    arr = ctypes.c_int * 3
    # odd band, band larger than grid, bad ndim, bad sigma: all EINVAL before any CUDA call
    assert L.lddmm_create(ctypes.byref(h), 3, arr(16, 16, 16), arr(7, 8, 8), 0.01, 2, 0.1, 4, None) == 1
    assert L.lddmm_create(ctypes.byref(h), 3, arr(16, 16, 16), arr(32, 8, 8), 0.01, 2, 0.1, 4, None) == 1
    assert L.lddmm_create(ctypes.byref(h), 4, arr(16, 16, 16), arr(8, 8, 8), 0.01, 2, 0.1, 4, None) == 1
    assert L.lddmm_create(ctypes.byref(h), 3, arr(16, 16, 16), arr(8, 8, 8), 0.01, 2, -1.0, 4, None) == 1
    assert L.lddmm_create(ctypes.byref(h), 3, arr(16, 16, 16), arr(8, 8, 8), 0.01, 2, 0.1, 0, None) == 1
    assert h.value is None
    assert L.lddmm_hessvec(None, None, None) == 1
    assert L.lddmm_last_error(None) == b"null context"


def test_binding_refuses_to_run_without_the_library(monkeypatch, tmp_path):
    from paper_1807_11560_gb300 import lddmm
    monkeypatch.setattr(lddmm, "_lib", None)
    monkeypatch.setattr(lddmm, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        lddmm.lib()


def test_default_opts_fill_the_whole_struct_and_bad_options_are_refused(so):
    """The binding's struct has the header's layout (the library's defaults land
    in the right fields, up to the last one), and an out-of-range option is
    refused before any CUDA call."""
    import ctypes as ct
    from paper_1807_11560_gb300 import lddmm
    L = lddmm.lib()
    o = lddmm.Opts()
    ct.memset(ct.byref(o), 0x7f, ct.sizeof(o))
    L.lddmm_default_opts(ct.byref(o))
    assert (o.precision, o.use_graphs, o.persistent, o.tensor_cores) == (1, 1, 1, 1)
    assert (o.recompute, o.autotune, o.newton, o.state_eq) == (0, 1, 0, 0)
    assert o.debug_stall == 0
    assert o.pcg_tol == 1e-12 and o.max_halvings == 10
    h = ct.c_void_p()
    arr = ct.c_int * 3
    o.debug_stall = -1
    assert L.lddmm_create(ct.byref(h), 3, arr(16, 16, 16), arr(8, 8, 8), 0.01, 2, 0.1, 4, ct.byref(o)) == 1
    assert h.value is None
