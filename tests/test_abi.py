"""The C-ABI library builds, loads and exports every symbol include/gs.h declares.

Runs without a GPU: only argument checks that return before any CUDA call are
exercised here.
"""
import ctypes

import pytest

from paper_2309_10292_gb300 import gs


@pytest.fixture(scope="module")
def lib():
    from paper_2309_10292_gb300 import build
    build.build()
    return gs.lib()


def test_exports_every_declared_symbol(lib):
    names = gs.header_symbols()
    assert "gs_create" in names and "gs_step" in names
    for n in names:
        assert hasattr(lib, n), f"libgs.so does not export {n}"
    assert set(gs._SIGS) == set(names), "binding and header disagree"


def test_argument_checks_without_gpu(lib):
    out = ctypes.c_void_p(1)
    rc = lib.gs_create(0, 0.2, 0.1, 0.02, 0.048, 1.0, 0.0, 0, gs.GS_F32, ctypes.byref(out))
    assert rc == gs.GS_EINVAL and out.value is None
    assert "L=0" in gs.gs_last_error()
    rc = lib.gs_create(8, 0.2, 0.1, 0.02, 0.048, 1.0, 0.0, 0, 7, ctypes.byref(out))
    assert rc == gs.GS_EINVAL and "dtype" in gs.gs_last_error()
    rc = lib.gs_create(8, float("nan"), 0.1, 0.02, 0.048, 1.0, 0.0, 0, 0, ctypes.byref(out))
    assert rc == gs.GS_EINVAL
    rc = lib.gs_create(gs_max_l() + 1, 0.2, 0.1, 0.02, 0.048, 1.0, 0.0, 0, 0, ctypes.byref(out))
    assert rc == gs.GS_EINVAL
    assert lib.gs_step(None, 1) == gs.GS_EINVAL
    assert lib.gs_noise_field(0, 0, 10, 9, None, None) == gs.GS_EINVAL
    assert lib.gs_noise_field(0, 0, -1, 0, None, None) == gs.GS_EINVAL
    assert lib.gs_destroy(None) == gs.GS_OK
    with pytest.raises(gs.GsError) as e:
        gs.gs_create(-3, 0.2, 0.1, 0.02, 0.048, 1.0, 0.0, 0, "f32")
    assert e.value.status == gs.GS_EINVAL


def gs_max_l():
    import re
    return int(re.search(r"#define GS_MAX_L (\d+)", open(gs.HEADER).read()).group(1))
