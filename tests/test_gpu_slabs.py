"""Voxel-slab sharding through the real product kernels, on one GPU: every rank's slab handle is
built in turn (paper_2103_06393_gb300/shard.py), its zbc_matvec must give the unsharded product's
rows of its slab and the sum of the ranks' zbc_rmatvec partials the unsharded adjoint, both within
1e-5 per right-hand side of the FP64 oracle on the original tensors."""
import numpy as np
import pytest

from oracle import products
from paper_2103_06393_gb300 import inputs, shard

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import __graft_entry__  # noqa: E402

__graft_entry__.build()
from paper_2103_06393_gb300 import zbc  # noqa: E402

RTOL = 1e-5


def _rel(a, b):
    return float(np.max(np.linalg.norm(a - b, axis=0) / np.linalg.norm(b, axis=0)))


def _handle(shape, m, aca):
    w = inputs.scaled_workload("precision", shape, m=m)
    g, s = w.grid, w.segments
    Z = zbc.colmajor(3 * g.nv, s.m, torch.complex128)
    zbc.vsie_assemble_columns(g, zbc.DeviceSegments(s), w.freq_hz, torch.arange(s.m, dtype=torch.int32,
                                                                                 device="cuda"), Z)
    h, _ = zbc.tucker_compress(Z, g, 1e-6)
    if aca:            # the same tensors behind a dense V (m' x M): Z' = U V^H
        tens, _ = h.tensors()
        rng = np.random.default_rng(3)
        V = rng.normal(size=(5, s.m)) + 1j * rng.normal(size=(5, s.m))
        h = zbc.zbc_create_from_host(g, 3, tens, V)
    return h, g


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("aca", [False, True])
@pytest.mark.parametrize("prec", ["fp32", "mode1", "dc"])
def test_slab_handles_reproduce_both_products(world, aca, prec):
    shape = (40, 18, 10)                     # slabs of 5 + 5 and of 3 + 3 + 4 planes
    h, g = _handle(shape, 12, aca)
    inf = h.info()
    p = 5
    fw, aj = {"fp32": (zbc.FP32_SIMT, zbc.FP32_SIMT), "mode1": (zbc.TC_MODE1, zbc.TC_MODE1),
              "dc": (zbc.TC_DC, zbc.TC_MODE1)}[prec]
    X = inputs.cn01((inf.m, p), seed=1).astype(np.complex64)
    Phi = inputs.cn01((3 * g.nv, p), seed=2).astype(np.complex64)
    tens, V = h.tensors()
    if aca:
        Yo = products.matvec_aca(tens, V.astype(np.complex128), g.shape, X)
        Po = products.rmatvec_aca(tens, V.astype(np.complex128), g.shape, Phi)
    else:
        Yo = products.matvec(tens, g.shape, X)
        Po = products.rmatvec(tens, g.shape, Phi)
    Y = zbc.colmajor(3 * g.nv, p, torch.complex64)
    Psi = zbc.colmajor(inf.m, p, torch.complex64)
    zbc.zbc_matvec(h, zbc.to_colmajor(X), Y, fw)
    zbc.zbc_rmatvec(h, zbc.to_colmajor(Phi), Psi, aj)
    zbc.zbc_product_status(h)
    Yfull, Pfull = zbc.from_colmajor(Y), zbc.from_colmajor(Psi)
    Psum = np.zeros((inf.m, p), dtype=np.complex128)
    for r in range(world):
        hr = shard.slab_handle(h, g, r, world)
        rows = shard.slab_rows(g.shape, 3, r, world)
        Yr = zbc.colmajor(rows.size, p, torch.complex64)
        Pr = zbc.colmajor(inf.m, p, torch.complex64)
        zbc.zbc_matvec(hr, zbc.to_colmajor(X), Yr, fw)
        zbc.zbc_rmatvec(hr, zbc.to_colmajor(Phi[rows]), Pr, aj)
        zbc.zbc_product_status(hr)
        yr = zbc.from_colmajor(Yr)
        assert _rel(yr, Yo[rows]) < RTOL, r          # the oracle on the original tensors
        assert _rel(yr, Yfull[rows]) < RTOL, r       # the unsharded call's rows
        Psum += zbc.from_colmajor(Pr)
    assert _rel(Psum, Po) < RTOL
    assert _rel(Psum, Pfull) < RTOL


def test_thin_slabs_are_refused():
    h, g = _handle((16, 12, 6), 4, False)
    with pytest.raises(ValueError):
        shard.slab_handle(h, g, 0, 4)               # 6 planes over 4 ranks: slabs of 1 and 2 planes
