"""The forward product Y = Z X in its decompress-and-contract tensor-core form (ZBC_TC_DC: per
block of 32 i1 x 4T i23 voxels and chunk of at most 8 stored columns, Z generated from U1 and the
cached W on the CUDA cores as fp16 hi/lo A operand in shared memory, the contraction with X' as
a tcgen05 GEMM with N = 2P, the accumulator folded into an FP32 sum in tensor memory every 8
chunks) against the FP64 oracle on the same compressed data: passes of 16, 32, 64 and 128
right-hand sides and several passes, ragged grids (n1 not a multiple of 32, i23 blocks cut by the
end of n2 n3), chunks cut by the rank budget (ranks up to 64), ACA storage, q = 12 handles,
extreme and mixed scales of X, agreement with the FP32 form and bit-for-bit repeatability."""
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


def _random_tensors(n, M, seed, rmax, q=3):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(M):
        tj = []
        for _k in range(q):
            r = [int(rng.integers(1, min(rmax, ni) + 1)) for ni in n]
            G = rng.normal(size=r) + 1j * rng.normal(size=r)
            Us = [np.linalg.qr(rng.normal(size=(ni, ri)) + 1j * rng.normal(size=(ni, ri)))[0]
                  for ni, ri in zip(n, r)]
            tj.append((G, Us))
        out.append(tj)
    return _c64(out)


def _fwd(h, shape, tens, p, seed=0, X=None, V=None, q=3):
    nv = int(np.prod(shape))
    m = len(tens) if V is None else V.shape[0]
    if X is None:
        X = inputs.cn01((m, p), seed=seed).astype(np.complex64)
    Y = zbc.colmajor(q * nv, p, torch.complex64)
    zbc.zbc_matvec(h, zbc.to_colmajor(X), Y, zbc.TC_DC)
    zbc.zbc_product_status(h)
    if V is None:
        Yo = products.matvec(tens, shape, X.astype(np.complex128))
    else:
        Yo = products.matvec_aca(tens, V.astype(np.complex64).astype(np.complex128), shape, X.astype(np.complex128))
    return zbc.from_colmajor(Y), Yo


@pytest.mark.parametrize("p", [1, 5, 16, 17, 32, 33, 64, 65, 128, 200])
def test_dc_fwd_tiny(p):
    w = inputs.workload("tiny")
    h, tens = _handle(w, 1e-8)
    Y, Yo = _fwd(h, w.grid.shape, tens, p)
    assert rel_cols(Y, Yo).max() < RTOL


@pytest.mark.parametrize("n", [(37, 9, 5), (70, 11, 3), (12, 13, 7), (96, 8, 6)])
@pytest.mark.parametrize("p", [16, 40])
def test_dc_fwd_ragged_grids(n, p):
    w = inputs.scaled_workload("precision", n, m=21)
    h, tens = _handle(w, 1e-6)
    Y, Yo = _fwd(h, n, tens, p, seed=3)
    assert rel_cols(Y, Yo).max() < RTOL


@pytest.mark.parametrize("rmax", [7, 33, 64])
def test_dc_fwd_random_ranks_and_chunking(rmax):
    n = (66, 64, 5)
    tens = _random_tensors(n, 45, seed=rmax, rmax=rmax)
    h = zbc.zbc_create_from_host(inputs.Grid(*n, 0.002), 3, tens)
    for p in (3, 32, 100):
        Y, Yo = _fwd(h, n, tens, p, seed=p)
        assert rel_cols(Y, Yo).max() < RTOL, p


def test_dc_fwd_many_columns_folds():
    """2500 columns: many folds of the tensor-core sum into the FP32 sum."""
    n = (8, 6, 5)
    tens = _random_tensors(n, 2500, seed=9, rmax=4)
    h = zbc.zbc_create_from_host(inputs.Grid(*n, 0.002), 3, tens)
    for p in (16, 64):
        Y, Yo = _fwd(h, n, tens, p, seed=p)
        assert rel_cols(Y, Yo).max() < RTOL, p


def test_dc_fwd_aca_storage():
    w = inputs.scaled_workload("precision", (26, 20, 18), m=14)
    rng = np.random.default_rng(4)
    V = rng.normal(size=(9, 14)) + 1j * rng.normal(size=(9, 14))
    h, tens = _handle(w, 1e-6, V)
    for p in (1, 32, 64):
        Y, Yo = _fwd(h, w.grid.shape, tens, p, seed=p, V=V)
        assert rel_cols(Y, Yo).max() < RTOL, p


def test_dc_fwd_q12():
    n = (34, 10, 4)
    tens = _random_tensors(n, 6, seed=12, rmax=6, q=12)
    h = zbc.zbc_create_from_host(inputs.Grid(*n, 0.002), 12, tens)
    Y, Yo = _fwd(h, n, tens, 20, seed=1, q=12)
    assert rel_cols(Y, Yo).max() < RTOL


@pytest.mark.parametrize("scale", [1e-20, 1e25])
def test_dc_fwd_extreme_and_mixed_scales(scale):
    w = inputs.scaled_workload("precision", (24, 20, 16), m=10)
    h, tens = _handle(w, 1e-6)
    X = inputs.cn01((10, 24), seed=5).astype(np.complex64) * np.float32(scale)
    # right-hand sides 1e15 apart in one pass (toward the middle of the float range, so that Y's
    # entries of the odd one out stay representable in complex64)
    X[:, 3] *= np.float32(1e-15 if scale > 1 else 1e15)
    Y, Yo = _fwd(h, w.grid.shape, tens, 24, X=X)
    assert rel_cols(Y, Yo).max() < RTOL


def test_dc_fwd_matches_fp32_and_repeats_bitwise():
    w = inputs.scaled_workload("precision", (40, 24, 16), m=33)
    h, tens = _handle(w, 1e-6)
    p = 48
    X = zbc.to_colmajor(inputs.cn01((33, p), seed=8).astype(np.complex64))
    nv = w.grid.nv
    Y1, Y2, Yf = (zbc.colmajor(3 * nv, p, torch.complex64) for _ in range(3))
    zbc.zbc_matvec(h, X, Y1, zbc.TC_DC)
    zbc.zbc_matvec(h, X, Y2, zbc.TC_DC)
    zbc.zbc_matvec(h, X, Yf, zbc.FP32_SIMT)
    zbc.zbc_product_status(h)
    assert torch.equal(Y1, Y2)
    a, b = zbc.from_colmajor(Y1), zbc.from_colmajor(Yf)
    assert rel_cols(a, b).max() < 2 * RTOL
