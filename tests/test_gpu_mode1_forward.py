"""The forward product Y = Z X in its mode-1 tensor-core form (ZBC_TC_MODE1: per block of 128
(i23, s) rows one fp16 hi/lo tcgen05 GEMM over the (column, rank) rows, A = W X generated on the
CUDA cores into tensor memory, B = U1, the accumulator folded into FP32 registers every 6 chunks)
against the FP64 oracle on the same compressed data: 4, 8 and 16 right-hand sides per pass,
several passes, ragged grids (n1 not a multiple of 16, i23 blocks cut by the end of n2 n3), i1
tiles (n1 > 96), chunks that hold one column or 32, ranks up to 64, ACA storage, extreme and mixed
scales of X, and bit-for-bit repeatability."""
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


def rel_cols(a, b):
    return np.linalg.norm(a - b, axis=0) / np.linalg.norm(b, axis=0)


def _c64(tens):
    return [[(t[0].astype(np.complex64).astype(np.complex128),
              [U.astype(np.complex64).astype(np.complex128) for U in t[1]]) for t in tj] for tj in tens]


def _handle(w, tol, V=None):
    g, s = w.grid, w.segments
    Z = greens.assemble_columns(g.shape, g.h, s.centre, s.tangent, s.length, w.freq_hz, np.arange(s.m),
                                mask_radius=g.mask_radius, mask_box=g.mask_box)
    tens = _c64(tucker.compress_columns(Z, g.shape, 3, tol))
    return zbc.zbc_create_from_host(g, 3, tens, V), tens


def _random_tensors(n, M, seed, rmax):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(M):
        tj = []
        for _k in range(3):
            r = [int(rng.integers(1, min(rmax, ni) + 1)) for ni in n]
            G = rng.normal(size=r) + 1j * rng.normal(size=r)
            Us = [np.linalg.qr(rng.normal(size=(ni, ri)) + 1j * rng.normal(size=(ni, ri)))[0]
                  for ni, ri in zip(n, r)]
            tj.append((G, Us))
        out.append(tj)
    return _c64(out)


def _fwd(h, shape, tens, p, seed=0, X=None, V=None, prec=None):
    nv = int(np.prod(shape))
    m = len(tens) if V is None else V.shape[0]
    if X is None:
        X = inputs.cn01((m, p), seed=seed).astype(np.complex64)
    Y = zbc.colmajor(3 * nv, p, torch.complex64)
    zbc.zbc_matvec(h, zbc.to_colmajor(X), Y, zbc.TC_MODE1 if prec is None else prec)
    zbc.zbc_product_status(h)
    if V is None:
        Yo = products.matvec(tens, shape, X.astype(np.complex128))
    else:
        Yo = products.matvec_aca(tens, V.astype(np.complex64).astype(np.complex128), shape, X.astype(np.complex128))
    return zbc.from_colmajor(Y), Yo


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 8, 9, 16, 17, 40])
def test_mode1_fwd_tiny(p):
    w = inputs.workload("tiny")
    h, tens = _handle(w, 1e-8)
    Y, Yo = _fwd(h, w.grid.shape, tens, p)
    assert rel_cols(Y, Yo).max() < RTOL


@pytest.mark.parametrize("n,p", [((13, 11, 7), 5), ((20, 13, 7), 16), ((37, 9, 5), 6), ((96, 10, 8), 16),
                                 ((8, 8, 8), 8), ((90, 3, 2), 12)])
def test_mode1_fwd_ragged(n, p):
    # n1 = 13, 20, 37, 90: D columns padded to a multiple of 32; n2 n3 = 77, 117, 45, 80, 64, 6:
    # the last i23 block partly past the end
    w = inputs.scaled_workload("precision", n, m=7)
    h, tens = _handle(w, 1e-5)
    Y, Yo = _fwd(h, n, tens, p, seed=3)
    assert rel_cols(Y, Yo).max() < RTOL


def test_mode1_fwd_agrees_with_tf32x3():
    w = inputs.scaled_workload("precision", (32, 24, 16), m=12)
    h, tens = _handle(w, 1e-6)
    Y1, Yo = _fwd(h, w.grid.shape, tens, 16, seed=5)
    Y0, _ = _fwd(h, w.grid.shape, tens, 16, seed=5, prec=zbc.TF32X3)
    assert rel_cols(Y1, Yo).max() < RTOL and rel_cols(Y0, Yo).max() < RTOL


@pytest.mark.parametrize("rmax,n", [(64, (64, 8, 4)), (33, (40, 7, 6))])
def test_mode1_fwd_high_ranks(rmax, n):
    # r1 up to 64: a chunk of 32 rows holds part of one column
    tens = _random_tensors(n, 20, seed=rmax, rmax=rmax)
    h = zbc.zbc_create_from_host(inputs.Grid(*n, 0.002), 3, tens)
    Y, Yo = _fwd(h, n, tens, 8, seed=9)
    assert rel_cols(Y, Yo).max() < RTOL


def test_mode1_fwd_many_columns():
    # 2500 columns of small tensors (r1 = 1 .. 3): chunks of up to 32 columns, ~200 chunks per
    # component, so hundreds of folds per block
    n = (8, 6, 5)
    tens = _random_tensors(n, 2500, seed=11, rmax=3)
    h = zbc.zbc_create_from_host(inputs.Grid(*n, 0.002), 3, tens)
    Y, Yo = _fwd(h, n, tens, 7, seed=12)
    assert rel_cols(Y, Yo).max() < RTOL


def test_mode1_fwd_aca_storage():
    w = inputs.scaled_workload("precision", (16, 16, 16), m=5)
    rng = np.random.default_rng(0)
    V = rng.normal(size=(9, 5)) + 1j * rng.normal(size=(9, 5))
    h, tens = _handle(w, 1e-6, V=V)
    Y, Yo = _fwd(h, w.grid.shape, tens, 6, V=V)
    assert rel_cols(Y, Yo).max() < RTOL


@pytest.mark.parametrize("scale", [1e-20, 1e-6, 1e6, 1e25])
def test_mode1_fwd_extreme_scales(scale):
    w = inputs.scaled_workload("precision", (24, 12, 10), m=6)
    h, tens = _handle(w, 1e-6)
    X = (inputs.cn01((len(tens), 8), seed=13) * scale).astype(np.complex64)
    Y, Yo = _fwd(h, w.grid.shape, tens, 8, X=X)
    assert np.all(np.isfinite(Y))
    assert rel_cols(Y, Yo).max() < RTOL


def test_mode1_fwd_mixed_column_scales():
    # right-hand sides 1e40 apart in one pass: each has its own exponent
    w = inputs.scaled_workload("precision", (24, 12, 10), m=5)
    h, tens = _handle(w, 1e-6)
    X = inputs.cn01((len(tens), 16), seed=22).astype(np.complex128)
    X *= np.array([1e-20, 1e20, 1.0, 3e-5] * 4)[None, :]
    Y, Yo = _fwd(h, w.grid.shape, tens, 16, X=X.astype(np.complex64))
    assert rel_cols(Y, Yo).max() < RTOL


@pytest.mark.parametrize("n,p", [((100, 4, 3), 8), ((160, 6, 5), 16), ((200, 3, 2), 3), ((97, 5, 4), 16)])
def test_mode1_fwd_i1_tiles(n, p):
    # n1 > 96: i1 tiles of at most 96 rows (100 -> 2 x 64, 160 -> 2 x 80, 200 -> 3 x 80, 97 -> 2 x 64),
    # the last tile partly past n1
    w = inputs.scaled_workload("precision", n, m=4)
    h, tens = _handle(w, 1e-5)
    Y, Yo = _fwd(h, n, tens, p, seed=23)
    assert rel_cols(Y, Yo).max() < RTOL


def test_mode1_fwd_repeatable():
    w = inputs.scaled_workload("precision", (24, 16, 12), m=8)
    h, tens = _handle(w, 1e-6)
    X = zbc.to_colmajor(inputs.cn01((len(tens), 16), seed=4).astype(np.complex64))
    outs = []
    for _ in range(2):
        Y = zbc.colmajor(3 * w.grid.nv, 16, torch.complex64)
        zbc.zbc_matvec(h, X, Y, zbc.TC_MODE1)
        zbc.zbc_product_status(h)
        outs.append(zbc.from_colmajor(Y))
    assert np.array_equal(outs[0], outs[1])
