"""Device-side failure detection without a GPU fault: a bounded wait made to run out (its poll
limit set to zero for one launch through the test hook zbc_test_wait_limit) must abort the
kernel cleanly and be reported by zbc_product_status as ZBC_ETIMEOUT, after which the next call
is correct against the FP64 oracle; a NaN or Inf in X or Phi must be reported as ZBC_ENAN by
every product form that reads it."""
import time

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


def _rel(a, b):
    return float(np.max(np.linalg.norm(a - b, axis=0) / np.linalg.norm(b, axis=0)))


def _handle(n=(34, 12, 10), m=10):
    w = inputs.scaled_workload("precision", n, m=m)
    g, s = w.grid, w.segments
    Z = greens.assemble_columns(g.shape, g.h, s.centre, s.tangent, s.length, w.freq_hz, np.arange(s.m))
    tens = tucker.compress_columns(Z, g.shape, 3, 1e-6)
    return zbc.zbc_create_from_host(g, 3, tens), g, tens


def _status(h):
    try:
        zbc.zbc_product_status(h)
        return zbc.ZBC_OK
    except zbc.ZbcError as e:
        return e.status


@pytest.mark.parametrize("noalloc", [False, True])
def test_bounded_wait_gives_up_and_the_next_call_is_correct(noalloc):
    h, g, tens = _handle()
    p = 3
    Phi = inputs.cn01((3 * g.nv, p), seed=4).astype(np.complex64)
    Phid = zbc.to_colmajor(Phi)
    Po = products.rmatvec(tens, g.shape, Phi)
    Psi = zbc.colmajor(len(tens), p, torch.complex64)

    def call():
        if noalloc:
            zbc.zbc_rmatvec_noalloc(h, Phid, Psi)
        else:
            zbc.zbc_rmatvec(h, Phid, Psi, zbc.FP32_SIMT)

    zbc.zbc_rmatvec(h, Phid, Psi, zbc.FP32_SIMT)      # builds the cache (noalloc needs it)
    assert _status(h) == zbc.ZBC_OK
    t0 = time.time()
    zbc.zbc_test_wait_limit(h, 0)                     # the next launch's first stage wait: 0 polls
    call()
    assert _status(h) == zbc.ZBC_ETIMEOUT
    assert time.time() - t0 < 60.0                    # the abort path ends within its bounds
    assert _status(h) == zbc.ZBC_OK                   # the word was cleared
    Psi.fill_(float("nan"))
    call()                                            # the limit applied to one launch only
    assert _status(h) == zbc.ZBC_OK
    assert _rel(zbc.from_colmajor(Psi), Po) < 1e-5


def test_nonfinite_inputs_are_reported():
    h, g, tens = _handle()
    p = 4
    X = inputs.cn01((len(tens), p), seed=5).astype(np.complex64)
    Phi = inputs.cn01((3 * g.nv, p), seed=6).astype(np.complex64)
    Xbad, Phibad = X.copy(), Phi.copy()
    Xbad[3, 1] = np.inf
    Phibad[2 * g.nv + 17, 2] = complex(0.0, np.nan)
    Y = zbc.colmajor(3 * g.nv, p, torch.complex64)
    Psi = zbc.colmajor(len(tens), p, torch.complex64)
    for prec in (zbc.FP32_SIMT, zbc.TF32X3, zbc.BF16X3, zbc.TC_MODE1):
        zbc.zbc_matvec(h, zbc.to_colmajor(Xbad), Y, prec)
        assert _status(h) == zbc.ZBC_ENAN, prec
        zbc.zbc_matvec(h, zbc.to_colmajor(X), Y, prec)
        assert _status(h) == zbc.ZBC_OK, prec
    for prec in (zbc.FP32_SIMT, zbc.TC_MODE1):
        zbc.zbc_rmatvec(h, zbc.to_colmajor(Phibad), Psi, prec)
        assert _status(h) == zbc.ZBC_ENAN, prec
        zbc.zbc_rmatvec(h, zbc.to_colmajor(Phi), Psi, prec)
        assert _status(h) == zbc.ZBC_OK, prec
    assert _rel(zbc.from_colmajor(Psi), products.rmatvec(tens, g.shape, Phi)) < 1e-5
