"""The K operator (Eq. nKt: the magnetic-field coupling grad g x t) and the Gauss-Legendre
quadrature along segments in the GPU column assembly (vsie_assemble_columns_op) against the FP64
oracle, then through compression and both products (FP32 and the mode-1 tensor-core forms)."""
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

OPS = {"N": zbc.OP_N, "K": zbc.OP_K}


def rel_cols(a, b):
    return np.linalg.norm(a - b, axis=0) / np.linalg.norm(b, axis=0)


def _assemble(w, op, nq, dtype=torch.complex128, cols=None):
    g, s = w.grid, w.segments
    cols = np.arange(s.m) if cols is None else np.asarray(cols)
    cd = torch.from_numpy(cols.astype(np.int32)).cuda()
    Z = zbc.colmajor(3 * g.nv, cols.size, dtype)
    zbc.vsie_assemble_columns_op(g, zbc.DeviceSegments(s), w.freq_hz, cd, Z, op=OPS[op], nq=nq)
    torch.cuda.synchronize()
    return zbc.from_colmajor(Z)


def _oracle(w, op, nq):
    g, s = w.grid, w.segments
    return greens.assemble_columns(g.shape, g.h, s.centre, s.tangent, s.length, w.freq_hz, np.arange(s.m),
                                   mask_radius=g.mask_radius, mask_box=g.mask_box, operator=op, nq=nq)


@pytest.mark.parametrize("op,nq", [("K", 1), ("K", 3), ("K", 8), ("N", 4), ("N", 1), ("K", 16)])
def test_assembly_matches_oracle(op, nq):
    w = inputs.scaled_workload("tiny", (20, 18, 16), m=10)
    Zg = _assemble(w, op, nq)
    Zo = _oracle(w, op, nq)
    assert rel_cols(Zg, Zo).max() < 1e-12
    Z32 = _assemble(w, op, nq, torch.complex64)
    assert rel_cols(Z32, Zo).max() < 1e-7


def test_n_point_matched_is_the_plain_entry_point():
    w = inputs.scaled_workload("tiny", (12, 10, 8), m=5)
    a = _assemble(w, "N", 1)
    g, s = w.grid, w.segments
    cd = torch.arange(s.m, dtype=torch.int32, device="cuda")
    Z = zbc.colmajor(3 * g.nv, s.m, torch.complex128)
    zbc.vsie_assemble_columns(g, zbc.DeviceSegments(s), w.freq_hz, cd, Z)
    torch.cuda.synchronize()
    assert np.array_equal(a, zbc.from_colmajor(Z))


def test_bad_operator_and_quadrature_rejected():
    w = inputs.scaled_workload("tiny", (6, 6, 6), m=2)
    g, s = w.grid, w.segments
    cd = torch.arange(2, dtype=torch.int32, device="cuda")
    Z = zbc.colmajor(3 * g.nv, 2, torch.complex128)
    for op, nq in ((2, 1), (zbc.OP_K, 0), (zbc.OP_K, 17)):
        with pytest.raises(zbc.ZbcError) as e:
            zbc.vsie_assemble_columns_op(g, zbc.DeviceSegments(s), w.freq_hz, cd, Z, op=op, nq=nq)
        assert e.value.status == zbc.ZBC_EINVAL


@pytest.mark.parametrize("prec", [zbc.FP32_SIMT, zbc.TC_MODE1])
def test_k_columns_compress_and_multiply(prec):
    # the magnetic coupling: assembled with 3-point quadrature, HOSVD-compressed on the GPU, then
    # Y = Z X and Psi = Z^H Phi against the oracle on the handle's tensors
    w = inputs.scaled_workload("precision", (24, 20, 16), m=12)
    g = w.grid
    Zd = zbc.to_colmajor(_assemble(w, "K", 3))
    h, st = zbc.tucker_compress(Zd, g, 1e-6)
    tens, _ = h.tensors()
    Zo = _oracle(w, "K", 3)
    Zt = np.stack([tucker.decompress_column(tj, g.shape) for tj in tens], axis=1)
    assert np.linalg.norm(Zt - Zo) / np.linalg.norm(Zo) < 2e-6
    p = 8
    X = inputs.cn01((w.segments.m, p), seed=31).astype(np.complex64)
    Phi = inputs.cn01((3 * g.nv, p), seed=32).astype(np.complex64)
    Y = zbc.colmajor(3 * g.nv, p, torch.complex64)
    Psi = zbc.colmajor(w.segments.m, p, torch.complex64)
    zbc.zbc_matvec(h, zbc.to_colmajor(X), Y, prec)
    zbc.zbc_rmatvec(h, zbc.to_colmajor(Phi), Psi, prec)
    zbc.zbc_product_status(h)
    assert rel_cols(zbc.from_colmajor(Y), products.matvec(tens, g.shape, X.astype(np.complex128))).max() < 1e-5
    assert rel_cols(zbc.from_colmajor(Psi), products.rmatvec(tens, g.shape, Phi.astype(np.complex128))).max() < 1e-5


@pytest.mark.parametrize("d,oracle_rank", [(0.55, 16), (1.0, 11)])
def test_gpu_compressor_reproduces_the_distance_study(d, oracle_rank):
    # the rank-vs-distance study (tests/test_oracle_rank_trends.py) through the GPU path: K columns
    # with 4-point quadrature assembled and HOSVD-compressed on the GPU give the oracle's max rank
    g = inputs.Grid(16, 16, 16, 1.0 / 16)
    s = inputs.loop_coil_y(0.5, d, 24)
    w = inputs.Workload("rank-distance", g, s, 298.06e6, 1e-8, 1)
    Zd = zbc.to_colmajor(_assemble(w, "K", 4))
    h, st = zbc.tucker_compress(Zd, g, 1e-8)
    assert abs(st.max_rank - oracle_rank) <= 1
    assert st.max_rel_err <= 1e-8 * (1 + 1e-9)


def _assemble_q(w, op, nq, q, dtype=torch.complex128):
    g, s = w.grid, w.segments
    cd = torch.arange(s.m, dtype=torch.int32, device="cuda")
    Z = zbc.colmajor(q * g.nv, s.m, dtype)
    zbc.vsie_assemble_columns_op(g, zbc.DeviceSegments(s), w.freq_hz, cd, Z, op=OPS[op], nq=nq, q=q)
    torch.cuda.synchronize()
    return zbc.from_colmajor(Z)


@pytest.mark.parametrize("op,nq", [("K", 2), ("N", 1), ("N", 3)])
def test_pwl_assembly_matches_oracle(op, nq):
    # the piecewise-linear basis (q = 12): 2 x 2 x 2 Gauss points per voxel, row block 3 l + k
    w = inputs.scaled_workload("tiny", (14, 12, 10), m=6)
    g, s = w.grid, w.segments
    Zg = _assemble_q(w, op, nq, 12)
    Zo = greens.assemble_columns(g.shape, g.h, s.centre, s.tangent, s.length, w.freq_hz, np.arange(s.m), q=12,
                                 mask_radius=g.mask_radius, mask_box=g.mask_box, operator=op, nq=nq)
    assert Zg.shape == Zo.shape == (12 * g.nv, s.m)
    for b in range(12):   # each block against its own scale (the linear blocks are ~100x smaller;
        blk = slice(b * g.nv, (b + 1) * g.nv)   # some columns of a block are exactly zero)
        assert np.linalg.norm(Zg[blk] - Zo[blk]) <= 1e-12 * np.linalg.norm(Zo[blk]), b
    Z32 = _assemble_q(w, op, nq, 12, torch.complex64)
    assert rel_cols(Z32, Zo).max() < 1e-7


@pytest.mark.parametrize("prec", [zbc.FP32_SIMT, zbc.TC_MODE1])
def test_pwl_k_columns_compress_and_multiply(prec):
    # q = 12 magnetic coupling columns through the GPU HOSVD and both products
    w = inputs.scaled_workload("precision", (20, 16, 12), m=6)
    g = w.grid
    Zd = zbc.to_colmajor(_assemble_q(w, "K", 2, 12))
    h, st = zbc.tucker_compress(Zd, g, 1e-6, q=12)
    assert h.info().q == 12
    tens, _ = h.tensors()
    p = 6
    X = inputs.cn01((w.segments.m, p), seed=41).astype(np.complex64)
    Phi = inputs.cn01((12 * g.nv, p), seed=42).astype(np.complex64)
    Y = zbc.colmajor(12 * g.nv, p, torch.complex64)
    Psi = zbc.colmajor(w.segments.m, p, torch.complex64)
    zbc.zbc_matvec(h, zbc.to_colmajor(X), Y, prec)
    zbc.zbc_rmatvec(h, zbc.to_colmajor(Phi), Psi, prec)
    zbc.zbc_product_status(h)
    assert rel_cols(zbc.from_colmajor(Y), products.matvec(tens, g.shape, X.astype(np.complex128))).max() < 1e-5
    assert rel_cols(zbc.from_colmajor(Psi), products.rmatvec(tens, g.shape, Phi.astype(np.complex128))).max() < 1e-5
