"""Failures made on the host, no GPU involved: with no usable CUDA device, the compressors and the
column assembly return ZBC_ECUDA with a message instead of crashing; a null handle is refused
with ZBC_EINVAL by both products.  The calls pass placeholder device pointers that nothing
dereferences on this path, so the test refuses to run where a GPU is present."""
import ctypes as C

import numpy as np
import pytest

from paper_2103_06393_gb300 import build, inputs

torch = pytest.importorskip("torch")
if torch.cuda.is_available():
    pytest.skip("needs a machine without a usable GPU", allow_module_level=True)


@pytest.fixture(scope="module")
def zbc():
    build.build()
    from paper_2103_06393_gb300 import zbc as z
    return z


def _setup(z):
    g = z.grid_struct(inputs.Grid(16, 12, 10, 0.002))
    segs = z.zbc_segments(2, C.c_void_p(0x1000), C.c_void_p(0x2000), C.c_void_p(0x3000))
    return g, segs, C.c_void_p(0x10000)


def test_without_a_device_calls_fail_with_a_status(zbc):
    L = zbc.lib()
    g, segs, fake = _setup(zbc)
    nv = 16 * 12 * 10
    h = C.c_void_p()
    st = zbc.zbc_compress_stats()
    xs = zbc.zbc_cross_stats()
    cols = np.array([0, 1], np.int32)
    calls = {
        "tucker_compress": lambda: L.tucker_compress(fake, 3 * nv, 2, C.byref(g), 3, zbc.C64, 1e-5, zbc.HOSVD,
                                                     None, zbc.C64, C.byref(h), C.byref(st), None),
        "cross_tucker_assemble": lambda: L.cross_tucker_assemble(C.byref(g), C.byref(segs), 298.2e6,
                                                                 cols.ctypes.data_as(C.c_void_p), 2, 3, 0, 1, 1e-5,
                                                                 None, None, 0, C.byref(h), C.byref(st), C.byref(xs),
                                                                 None),
        "cross_tucker_compress": lambda: L.cross_tucker_compress(fake, 3 * nv, 2, C.byref(g), 3, zbc.C64, 1e-5, None,
                                                                 None, 0, C.byref(h), C.byref(st), C.byref(xs), None),
        "vsie_assemble_columns": lambda: L.vsie_assemble_columns(C.byref(g), C.byref(segs), 298.2e6, fake, 2, 3, fake,
                                                                 3 * nv, zbc.C64, None),
    }
    for name, call in calls.items():
        status = call()
        assert status == zbc.ZBC_ECUDA, (name, status)
        assert L.zbc_last_error().decode(), name
        assert not h.value, name     # no handle was created


def test_products_refuse_a_null_handle(zbc):
    L = zbc.lib()
    fake = C.c_void_p(0x10000)
    assert L.zbc_matvec(None, fake, 8, 1, fake, 8, zbc.FP32_SIMT, None) == zbc.ZBC_EINVAL
    assert "null" in L.zbc_last_error().decode()
    assert L.zbc_rmatvec(None, fake, 8, 1, fake, 8, zbc.FP32_SIMT, None) == zbc.ZBC_EINVAL
    assert "null" in L.zbc_last_error().decode()
