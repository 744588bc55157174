"""zbc_rmatvec_noalloc: the adjoint product for callers that cannot allocate device memory at
call time (a fixed memory budget, allocator hooks that must not re-enter the allocator).  On two
calls in a row (the shared scratch array keeps the previous call's contents) it must agree with
zbc_rmatvec and with the FP64 oracle's Algorithm 2 on the handle's own tensors, on plain and on
ACA storage, and it must refuse, with a clear status, work that does not fit its fixed scratch
or a handle whose decompression cache was never built.  Collected last so a failure here stops
nothing else."""
import numpy as np
import pytest

from oracle import greens, products, tucker
from paper_2103_06393_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import __graft_entry__  # noqa: E402

__graft_entry__.build()
from paper_2103_06393_gb300 import zbc  # noqa: E402

RTOL = 1e-5


def _handle(V=None, n=(16, 14, 12), m=12):
    w = inputs.scaled_workload("precision", n, m=m)
    g, s = w.grid, w.segments
    Z = greens.assemble_columns(g.shape, g.h, s.centre, s.tangent, s.length, w.freq_hz, np.arange(s.m))
    tens = tucker.compress_columns(Z, g.shape, 3, 1e-6)
    return zbc.zbc_create_from_host(g, 3, tens, V), g


def _rel(a, b):
    return float(np.max(np.linalg.norm(a - b, axis=0) / np.linalg.norm(b, axis=0)))


@pytest.mark.parametrize("aca", [False, True])
def test_noalloc_matches_rmatvec_twice(aca):
    rng = np.random.default_rng(1)
    V = (rng.normal(size=(9, 12)) + 1j * rng.normal(size=(9, 12))) if aca else None
    h, g = _handle(V)
    m = h.info().m
    Phi = zbc.to_colmajor(inputs.cn01((3 * g.nv, 5), seed=2).astype(np.complex64))
    ref = zbc.colmajor(m, 5, torch.complex64)
    zbc.zbc_rmatvec(h, Phi, ref, zbc.FP32_SIMT)        # also builds the decompression cache
    torch.cuda.synchronize()
    r = zbc.from_colmajor(ref)
    tens, Vh = h.tensors()
    Phih = zbc.from_colmajor(Phi).astype(np.complex128)
    if aca:
        ref_o = products.rmatvec_aca(tens, Vh.astype(np.complex128), g.shape, Phih)
    else:
        ref_o = products.rmatvec(tens, g.shape, Phih)
    for _ in range(2):
        out = zbc.colmajor(m, 5, torch.complex64)
        out.fill_(float("nan"))
        zbc.zbc_rmatvec_noalloc(h, Phi, out)
        zbc.zbc_product_status(h)             # synchronises; raises if a device wait gave up
        got = zbc.from_colmajor(out)
        assert _rel(got, r) < RTOL            # the allocating entry point
        assert _rel(got, ref_o) < RTOL        # the FP64 oracle (relative error per right-hand side)


def test_noalloc_requires_built_cache():
    h, g = _handle()
    Phi = zbc.to_colmajor(inputs.cn01((3 * g.nv, 2), seed=3).astype(np.complex64))
    out = zbc.colmajor(h.info().m, 2, torch.complex64)
    with pytest.raises(zbc.ZbcError) as e:
        zbc.zbc_rmatvec_noalloc(h, Phi, out)
    assert e.value.status == zbc.ZBC_EINVAL and "cache" in str(e.value)


def test_noalloc_rejects_work_beyond_scratch():
    # 2048 rank-1 columns on a 2x2x2 grid: q*M*p complex64 with p = 1024 is 48 MiB > 16 MiB
    grid = inputs.Grid(2, 2, 2, 0.01)
    one = (np.ones((1, 1, 1), complex), [np.ones((2, 1), complex) / np.sqrt(2)] * 3)
    tens = [[one] * 3 for _ in range(2048)]
    h = zbc.zbc_create_from_host(grid, 3, tens)
    Phi = zbc.colmajor(3 * 8, 1024, torch.complex64)
    out = zbc.colmajor(2048, 1024, torch.complex64)
    with pytest.raises(zbc.ZbcError) as e:
        zbc.zbc_rmatvec_noalloc(h, Phi, out)
    assert e.value.status == zbc.ZBC_EINVAL and "scratch" in str(e.value)
