"""The adjoint product Psi = Z^H Phi in its mode-1 tensor-core form (ZBC_TC_MODE1: T = U1^H Phi^k as
one fp16 hi/lo tcgen05 GEMM per group of 128 (column, rank) rows, then sum conj(W) T) against the
FP64 oracle on the same compressed data: right-hand-side counts that pad the pass or need several
passes, ragged grids (n1 not a multiple of 8, N blocks cut by the end of i23), groups that split a
column's ranks, ranks up to 64, many columns, ACA storage, extreme scales of Phi, wide n1 (i1
tiles), and bit-for-bit repeatability."""
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
    """M columns x 3 components of random Tucker tensors, ranks 1..rmax per mode, orthonormal
    factors, complex64-exact."""
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


def _adj(h, shape, tens, p, seed=1, scale=1.0, V=None, prec=None):
    nv = int(np.prod(shape))
    m = len(tens) if V is None else V.shape[0]
    Phi = (inputs.cn01((3 * nv, p), seed=seed) * scale).astype(np.complex64)
    Psi = zbc.colmajor(m, p, torch.complex64)
    zbc.zbc_rmatvec(h, zbc.to_colmajor(Phi), Psi, zbc.TC_MODE1 if prec is None else prec)
    zbc.zbc_product_status(h)
    if V is None:
        Po = products.rmatvec(tens, shape, Phi.astype(np.complex128))
    else:
        Po = products.rmatvec_aca(tens, V.astype(np.complex64).astype(np.complex128), shape,
                                  Phi.astype(np.complex128))
    return zbc.from_colmajor(Psi), Po


@pytest.mark.parametrize("p", [1, 2, 3, 5, 8, 16, 17, 40])
def test_mode1_tiny(p):
    w = inputs.workload("tiny")
    h, tens = _handle(w, 1e-8)
    P, Po = _adj(h, w.grid.shape, tens, p)
    assert rel_cols(P, Po).max() < RTOL


@pytest.mark.parametrize("n,p", [((13, 11, 7), 5), ((20, 13, 7), 16), ((37, 9, 5), 3), ((96, 10, 8), 16),
                                 ((8, 8, 8), 1)])
def test_mode1_ragged(n, p):
    # n1 = 13, 20, 37: K padded to a multiple of 8 (and 37 -> two K chunks of 24 and 16);
    # n2 n3 = 77, 117, 45, 80, 64: the last N block partly past the end of i23
    w = inputs.scaled_workload("precision", n, m=7)
    h, tens = _handle(w, 1e-5)
    P, Po = _adj(h, n, tens, p, seed=3)
    assert rel_cols(P, Po).max() < RTOL


def test_mode1_agrees_with_simt():
    w = inputs.scaled_workload("precision", (32, 24, 16), m=12)
    h, tens = _handle(w, 1e-6)
    P1, Po = _adj(h, w.grid.shape, tens, 16, seed=5)
    P0, _ = _adj(h, w.grid.shape, tens, 16, seed=5, prec=zbc.FP32_SIMT)
    assert rel_cols(P1, Po).max() < RTOL and rel_cols(P0, Po).max() < RTOL
    assert rel_cols(P1, P0).max() < 2 * RTOL


@pytest.mark.parametrize("rmax,n", [(64, (64, 8, 4)), (33, (40, 7, 6))])
def test_mode1_high_ranks(rmax, n):
    # r1 up to 64 (the product kernels' limit): a column's ranks straddle groups of 128 rows
    tens = _random_tensors(n, 20, seed=rmax, rmax=rmax)
    h = zbc.zbc_create_from_host(inputs.Grid(*n, 0.002), 3, tens)
    P, Po = _adj(h, n, tens, 5, seed=9)
    assert rel_cols(P, Po).max() < RTOL


def test_mode1_many_columns():
    # 2500 columns of small tensors: ~100 groups per component, many items per CTA
    n = (8, 6, 5)
    tens = _random_tensors(n, 2500, seed=11, rmax=7)
    h = zbc.zbc_create_from_host(inputs.Grid(*n, 0.002), 3, tens)
    P, Po = _adj(h, n, tens, 3, seed=12)
    assert rel_cols(P, Po).max() < RTOL


def test_mode1_aca_storage():
    w = inputs.scaled_workload("precision", (16, 16, 16), m=5)
    rng = np.random.default_rng(0)
    V = rng.normal(size=(9, 5)) + 1j * rng.normal(size=(9, 5))
    h, tens = _handle(w, 1e-6, V=V)
    P, Po = _adj(h, w.grid.shape, tens, 3, V=V)
    assert rel_cols(P, Po).max() < RTOL


@pytest.mark.parametrize("scale", [1e-20, 1e-6, 1e6, 1e30])
def test_mode1_extreme_scales(scale):
    # each N block of Phi is brought into fp16's range by its own powers of two; the scales keep
    # Psi (~1e-8 scale at this voxel size) inside FP32's normal range, as any FP32 form needs
    w = inputs.scaled_workload("precision", (24, 12, 10), m=6)
    h, tens = _handle(w, 1e-6)
    P, Po = _adj(h, w.grid.shape, tens, 4, seed=13, scale=scale)
    assert np.all(np.isfinite(P))
    assert rel_cols(P, Po).max() < RTOL


def test_mode1_mixed_block_scales():
    # one region of Phi 1e12 times larger than the rest: per-block exponents keep both accurate
    n = (16, 12, 10)
    w = inputs.scaled_workload("precision", n, m=4)
    h, tens = _handle(w, 1e-6)
    nv = int(np.prod(n))
    Phi = inputs.cn01((3 * nv, 2), seed=21).astype(np.complex128)
    Phi[: nv // 3] *= 1e12
    Phi = Phi.astype(np.complex64)
    Psi = zbc.colmajor(len(tens), 2, torch.complex64)
    zbc.zbc_rmatvec(h, zbc.to_colmajor(Phi), Psi, zbc.TC_MODE1)
    zbc.zbc_product_status(h)
    Po = products.rmatvec(tens, n, Phi.astype(np.complex128))
    assert rel_cols(zbc.from_colmajor(Psi), Po).max() < RTOL


def test_mode1_mixed_column_scales():
    # right-hand sides 1e40 apart in one pass: each gets its own exponent per N block
    n = (24, 12, 10)
    w = inputs.scaled_workload("precision", n, m=5)
    h, tens = _handle(w, 1e-6)
    nv = int(np.prod(n))
    Phi = inputs.cn01((3 * nv, 16), seed=22).astype(np.complex128)
    Phi *= np.array([1e-20, 1e20, 1.0, 3e-5] * 4)[None, :]
    Phi = Phi.astype(np.complex64)
    Psi = zbc.colmajor(len(tens), 16, torch.complex64)
    zbc.zbc_rmatvec(h, zbc.to_colmajor(Phi), Psi, zbc.TC_MODE1)
    zbc.zbc_product_status(h)
    Po = products.rmatvec(tens, n, Phi.astype(np.complex128))
    assert rel_cols(zbc.from_colmajor(Psi), Po).max() < RTOL


@pytest.mark.parametrize("p", [8, 16])
def test_mode1_n1_160_single_buffer(p):
    # n1 = 160: A takes 320 TMEM columns, so N blocks of 192 rows with one D buffer
    n = (160, 6, 5)
    w = inputs.scaled_workload("precision", n, m=4)
    h, tens = _handle(w, 1e-5)
    P, Po = _adj(h, n, tens, p, seed=19)
    assert rel_cols(P, Po).max() < RTOL


@pytest.mark.parametrize("n,p", [((200, 5, 3), 16), ((232, 3, 2), 16), ((330, 3, 2), 5), ((257, 4, 3), 2)])
def test_mode1_wide_n1(n, p):
    # n1 = 200: A takes 2 x 224 TMEM columns, N blocks of 32 rows; n1 = 232, 330, 257: i1 tiles of
    # 160 (two or three of them, the last partly past n1), each with its own partial sums
    w = inputs.scaled_workload("precision", n, m=3)
    h, tens = _handle(w, 1e-5)
    P, Po = _adj(h, n, tens, p, seed=17)
    assert rel_cols(P, Po).max() < RTOL


def test_mode1_repeatable():
    w = inputs.scaled_workload("precision", (24, 16, 12), m=8)
    h, tens = _handle(w, 1e-6)
    Phi = zbc.to_colmajor(inputs.cn01((3 * w.grid.nv, 16), seed=4).astype(np.complex64))
    outs = []
    for _ in range(2):
        Psi = zbc.colmajor(len(tens), 16, torch.complex64)
        zbc.zbc_rmatvec(h, Phi, Psi, zbc.TC_MODE1)
        zbc.zbc_product_status(h)
        outs.append(zbc.from_colmajor(Psi))
    assert np.array_equal(outs[0], outs[1])
