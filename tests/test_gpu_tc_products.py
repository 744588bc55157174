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
                                mask_radius=g.mask_radius, mask_box=g.mask_box)
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


@pytest.mark.parametrize("prec", [zbc.FP32_SIMT] + TC)
def test_high_ranks_up_to_64(prec):
    # ACA's U columns reach Tucker ranks far above the Green's-function columns' (r1 up to 64):
    # random tensors with r1 in [33, 64] on a 70 x 20 x 6 grid, both products
    rng = np.random.default_rng(21)
    n = (70, 20, 6)
    tens = []
    for _ in range(10):
        tj = []
        for _k in range(3):
            r = (int(rng.integers(33, 65)), int(rng.integers(1, 9)), int(rng.integers(1, 7)))
            G = rng.normal(size=r) + 1j * rng.normal(size=r)
            Us = [np.linalg.qr(rng.normal(size=(ni, ri)) + 1j * rng.normal(size=(ni, ri)))[0] for ni, ri in zip(n, r)]
            tj.append((G.astype(np.complex64).astype(np.complex128),
                       [U.astype(np.complex64).astype(np.complex128) for U in Us]))
        tens.append(tj)
    grid = inputs.Grid(*n, 0.002)
    h = zbc.zbc_create_from_host(grid, 3, tens)
    p = 12
    X = inputs.cn01((10, p), seed=5).astype(np.complex64)
    Y = zbc.colmajor(3 * grid.nv, p, torch.complex64)
    try:
        zbc.zbc_matvec(h, zbc.to_colmajor(X), Y, prec)
    except zbc.ZbcError as e:
        # TC2's shared-memory layout holds mode-product operands up to r1 ~ 40 only; beyond
        # that it must refuse cleanly (the autotuner then skips it)
        assert prec == zbc.TC2 and e.status == zbc.ZBC_EINVAL and "does not fit" in str(e)
        return
    zbc.zbc_product_status(h)
    assert rel_cols(zbc.from_colmajor(Y), products.matvec(tens, n, X)).max() < RTOL
    if prec == zbc.FP32_SIMT:
        Phi = inputs.cn01((3 * grid.nv, p), seed=6).astype(np.complex64)
        Psi = zbc.colmajor(10, p, torch.complex64)
        zbc.zbc_rmatvec(h, zbc.to_colmajor(Phi), Psi, prec)
        zbc.zbc_product_status(h)
        assert rel_cols(zbc.from_colmajor(Psi), products.rmatvec(tens, n, Phi)).max() < RTOL


@pytest.mark.parametrize("prec", TC)
def test_tc_long_i1_many_columns(prec):
    # n1 = 96 as in the 96^3 workload (U1 entries ~ 0.1, whose fp16 lo terms would fall below
    # fp16's normal range without scaling) and 256 columns (32 chunks: eight folds of D)
    w = inputs.scaled_workload("precision", (96, 10, 8), m=256)
    h, tens = _handle(w, 1e-6)
    Y, Yo = _fwd(h, w, tens, 16, prec, seed=9)
    assert rel_cols(Y, Yo).max() < RTOL


@pytest.mark.parametrize("prec", [zbc.FP32_SIMT, zbc.TF32X3, zbc.TC2, zbc.TC_MODE1])
def test_twelve_components_per_column(prec):
    # q = 12 (a piecewise-linear basis: 4 functions x 3 components per voxel): the product
    # kernels take q from the handle, four times the work of q = 3
    rng = np.random.default_rng(31)
    n = (24, 12, 10)
    tens = []
    for _ in range(9):
        tj = []
        for _k in range(12):
            r = tuple(int(rng.integers(1, 9)) for _ in range(3))
            G = rng.normal(size=r) + 1j * rng.normal(size=r)
            Us = [np.linalg.qr(rng.normal(size=(ni, ri)) + 1j * rng.normal(size=(ni, ri)))[0] for ni, ri in zip(n, r)]
            tj.append((G.astype(np.complex64).astype(np.complex128),
                       [U.astype(np.complex64).astype(np.complex128) for U in Us]))
        tens.append(tj)
    grid = inputs.Grid(*n, 0.002)
    h = zbc.zbc_create_from_host(grid, 12, tens)
    assert h.info().q == 12
    p = 5
    X = inputs.cn01((9, p), seed=7).astype(np.complex64)
    Y = zbc.colmajor(12 * grid.nv, p, torch.complex64)
    zbc.zbc_matvec(h, zbc.to_colmajor(X), Y, prec)
    zbc.zbc_product_status(h)
    assert rel_cols(zbc.from_colmajor(Y), products.matvec(tens, n, X)).max() < RTOL
    if prec in (zbc.FP32_SIMT, zbc.TC_MODE1):
        Phi = inputs.cn01((12 * grid.nv, p), seed=8).astype(np.complex64)
        Psi = zbc.colmajor(9, p, torch.complex64)
        zbc.zbc_rmatvec(h, zbc.to_colmajor(Phi), Psi, prec)
        zbc.zbc_product_status(h)
        assert rel_cols(zbc.from_colmajor(Psi), products.rmatvec(tens, n, Phi)).max() < RTOL


def test_hosvd_twelve_components():
    # tucker_compress with q = 12 on planted-rank columns: ranks recovered, error within tol
    from oracle import tucker as otucker
    rng = np.random.default_rng(33)
    n = (16, 12, 10)
    nv = n[0] * n[1] * n[2]
    cols, planted = [], []
    for _ in range(3):
        col = []
        for _k in range(12):
            r = tuple(int(rng.integers(1, 5)) for _ in range(3))
            G = rng.normal(size=r) + 1j * rng.normal(size=r)
            Us = [np.linalg.qr(rng.normal(size=(ni, ri)) + 1j * rng.normal(size=(ni, ri)))[0] for ni, ri in zip(n, r)]
            col.append(otucker.reconstruct(G, Us).reshape(-1, order="F"))
            # the mode-g rank of a generic core is min(r_g, product of the other two ranks)
            planted.append(tuple(min(r[gm], r[(gm + 1) % 3] * r[(gm + 2) % 3]) for gm in range(3)))
        cols.append(np.concatenate(col))
    Z = np.stack(cols, axis=1)
    grid = inputs.Grid(*n, 0.002)
    h, st = zbc.tucker_compress(zbc.to_colmajor(Z.astype(np.complex128)), grid, 1e-10, q=12)
    ranks, _, _ = h.export()
    assert [tuple(x) for x in ranks.reshape(-1, 3)] == planted
    assert st.max_rel_err <= 1e-10 * (1 + 1e-6) + 1e-12


@pytest.mark.parametrize("prec", TC)
def test_tc_many_rhs_on_three_group_tiles(prec):
    # p = 72 on n1 = 96 (three 32-row groups per i1 tile): 64 right-hand sides per CTA do not fit
    # TMEM with three M tiles, so the forms fall back to 32 per CTA (or fewer u values)
    w = inputs.scaled_workload("precision", (96, 6, 4), m=12)
    h, tens = _handle(w, 1e-6)
    Y, Yo = _fwd(h, w, tens, 72, prec, seed=12)
    assert rel_cols(Y, Yo).max() < RTOL


@pytest.mark.parametrize("prec", [zbc.FP32_SIMT] + TC)
@pytest.mark.parametrize("M", [1, 3, 9])
def test_few_columns(prec, M):
    # fewer columns than a chunk, a stage ring, or one producer half's share
    w = inputs.scaled_workload("precision", (20, 14, 6), m=M)
    h, tens = _handle(w, 1e-6)
    for p in (1, 3):
        Y, Yo = _fwd(h, w, tens, p, prec, seed=M + p)
        assert rel_cols(Y, Yo).max() < RTOL
    if prec == zbc.FP32_SIMT:
        g = w.grid
        Phi = inputs.cn01((3 * g.nv, 2), seed=M).astype(np.complex64)
        Psi = zbc.colmajor(M, 2, torch.complex64)
        zbc.zbc_rmatvec(h, zbc.to_colmajor(Phi), Psi, prec)
        zbc.zbc_product_status(h)
        assert rel_cols(zbc.from_colmajor(Psi), products.rmatvec(tens, g.shape, Phi)).max() < RTOL
