"""Tensor-core products (tcgen05: TF32X3 and BF16X3 contractions, and TC2 with the mode product
on the tensor cores too) against the FP64 oracle on the same
compressed data: several RHS counts (padding of the RHS chunk), ragged tiles, ACA storage."""
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
TC = [zbc.TF32X3, zbc.BF16X3, zbc.TC2]


def rel_cols(a, b):
    return np.linalg.norm(a - b, axis=0) / np.linalg.norm(b, axis=0)


def _handle(w, tol, V=None):
    g, s = w.grid, w.segments
    Z = greens.assemble_columns(g.shape, g.h, s.centre, s.tangent, s.length, w.freq_hz, np.arange(s.m),
                                mask_radius=g.mask_radius)
    tens = tucker.compress_columns(Z, g.shape, 3, tol)
    tens = [[(t[0].astype(np.complex64).astype(np.complex128),
              [U.astype(np.complex64).astype(np.complex128) for U in t[1]]) for t in tj] for tj in tens]
    return zbc.zbc_create_from_host(g, 3, tens, V), tens


def _fwd(h, w, tens, p, prec, V=None, seed=0):
    g = w.grid
    m = len(tens) if V is None else V.shape[0]
    X = inputs.cn01((m, p), seed=seed).astype(np.complex64)
    Y = zbc.colmajor(3 * g.nv, p, torch.complex64)
    zbc.zbc_matvec(h, zbc.to_colmajor(X), Y, prec)
    torch.cuda.synchronize()
    if V is None:
        Yo = products.matvec(tens, g.shape, X)
    else:
        Yo = products.matvec_aca(tens, V.astype(np.complex64).astype(np.complex128), g.shape, X)
    return zbc.from_colmajor(Y), Yo


@pytest.mark.parametrize("prec", TC)
@pytest.mark.parametrize("p", [1, 5, 16, 20, 40])
def test_tc_matvec_tiny(prec, p):
    w = inputs.workload("tiny")
    h, tens = _handle(w, 1e-8)
    Y, Yo = _fwd(h, w, tens, p, prec)
    assert rel_cols(Y, Yo).max() < RTOL


@pytest.mark.parametrize("prec", TC)
@pytest.mark.parametrize("n", [(13, 11, 7), (40, 17, 5), (130, 9, 3)])
def test_tc_matvec_ragged(prec, n):
    w = inputs.scaled_workload("precision", n, m=11)
    h, tens = _handle(w, 1e-5)
    Y, Yo = _fwd(h, w, tens, 9, prec, seed=4)
    assert rel_cols(Y, Yo).max() < RTOL


@pytest.mark.parametrize("prec", TC)
def test_tc_matvec_precision_scaled(prec):
    w = inputs.scaled_workload("precision", (48, 48, 48), m=24)
    h, tens = _handle(w, 1e-6)
    Y, Yo = _fwd(h, w, tens, 16, prec, seed=5)
    e = rel_cols(Y, Yo).max()
    print("rel err", prec, e)
    assert e < RTOL


@pytest.mark.parametrize("prec", TC)
def test_tc_matvec_aca_storage(prec):
    w = inputs.scaled_workload("precision", (16, 16, 16), m=5)
    rng = np.random.default_rng(0)
    V = rng.normal(size=(9, 5)) + 1j * rng.normal(size=(9, 5))
    h, tens = _handle(w, 1e-6, V=V)
    Y, Yo = _fwd(h, w, tens, 3, prec, V=V)
    assert rel_cols(Y, Yo).max() < RTOL
