"""Host-side argument checks of the fibre-cross compressors (cross_tucker_assemble,
cross_tucker_compress): every case below is refused with ZBC_EINVAL and a message before any
device pointer is touched or any CUDA call is made, so these run without a GPU.  Also the
binding's structures against the header's."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2103_06393_gb300 import build, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def zbc():
    build.build()
    from paper_2103_06393_gb300 import zbc as z
    return z


def _segs(z, m=2):
    # non-null pointers that the refused calls never dereference
    return z.zbc_segments(m, C.c_void_p(0x1000), C.c_void_p(0x2000), C.c_void_p(0x3000))


def _assemble(z, grid=(16, 12, 10), cols=(0,), q=3, op=0, nq=1, tol=1e-5, params=None, checks=None, m=2):
    g = z.grid_struct(inputs.Grid(*grid, 0.002))
    s = _segs(z, m)
    c = np.asarray(cols, dtype=np.int32)
    prm, chk = z._cross_args(params, checks)
    h = C.c_void_p()
    st = z.lib().cross_tucker_assemble(C.byref(g), C.byref(s), 298.2e6, c.ctypes.data_as(C.c_void_p), c.size, q, op,
                                       nq, tol, C.byref(prm) if prm is not None else None,
                                       chk.ctypes.data_as(C.c_void_p), chk.shape[0], C.byref(h), None, None, None)
    return st, z.lib().zbc_last_error().decode()


@pytest.mark.parametrize("kw,needle", [
    (dict(params={"rmax": 65}), "rmax"),
    (dict(params={"over": 17}), "over"),
    (dict(params={"sweeps": 17}), "sweeps"),
    (dict(params={"s0": 65}), "s0"),
    (dict(checks=[[3, 0, 0]]), "mode"),
    (dict(checks=[[0, 12, 0]]), "out of range"),
    (dict(checks=[[1, 0, 10]]), "out of range"),
    (dict(cols=(2,)), "cols_host"),
    (dict(cols=(-1,)), "cols_host"),
    (dict(grid=(15, 12, 10)), "even"),
    (dict(grid=(16, 12, 2048)), "grid sizes"),
    (dict(q=4), "q must be"),
    (dict(op=2), "operator"),
    (dict(nq=17), "nq"),
    (dict(tol=0.0), "tol"),
])
def test_assemble_refuses(zbc, kw, needle):
    st, msg = _assemble(zbc, **kw)
    assert st == zbc.ZBC_EINVAL
    assert needle in msg, msg


def test_compress_refuses(zbc):
    g = zbc.grid_struct(inputs.Grid(16, 12, 10, 0.002))
    h = C.c_void_p()
    L = zbc.lib()
    fake = C.c_void_p(0x1000)
    nv = 16 * 12 * 10

    def call(ld=3 * nv, q=3, dt=zbc.C64, params=None, checks=None, tol=1e-5):
        prm, chk = zbc._cross_args(params, checks)
        return L.cross_tucker_compress(fake, ld, 2, C.byref(g), q, dt, tol,
                                       C.byref(prm) if prm is not None else None, chk.ctypes.data_as(C.c_void_p),
                                       chk.shape[0], C.byref(h), None, None, None)

    assert call(ld=3 * nv - 1) == zbc.ZBC_EINVAL
    assert call(q=13) == zbc.ZBC_EINVAL
    assert call(params={"rmax": 64, "over": -1}) == zbc.ZBC_EINVAL
    assert call(checks=[[2, 16, 0]]) == zbc.ZBC_EINVAL
    assert call(tol=1.0) == zbc.ZBC_EINVAL


def test_binding_structures_match_the_header(zbc):
    text = open(os.path.join(ROOT, "include", "zbc.h")).read()
    for cname, pyt in (("zbc_cross_params", zbc.zbc_cross_params), ("zbc_cross_stats", zbc.zbc_cross_stats)):
        body = re.search(r"typedef struct \{([^{}]*)\}\s*" + cname + ";", text).group(1)
        body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
        fields = re.findall(r"(int32_t|int64_t|double)\s+(\w+);", body)
        ctype = {"int32_t": C.c_int32, "int64_t": C.c_int64, "double": C.c_double}
        assert [(n, ctype[t]) for t, n in fields] == list(pyt._fields_), cname
