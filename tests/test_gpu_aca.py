"""GPU ACA (plain, dense U then Tucker) and Algorithm 3 (Tucker-compressed U) against the
oracle's FP64 ACA on the same geometry: pivots, rank, norm estimate, approximation error and
the products on the resulting U V^H storage."""
import numpy as np
import pytest

from oracle import aca, greens, products
from paper_2103_06393_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import __graft_entry__  # noqa: E402

__graft_entry__.build()
from paper_2103_06393_gb300 import zbc  # noqa: E402


def _case(mask_radius=None, n=(12, 12, 10), m=64):
    w = inputs.scaled_workload("batching", n, m=m)
    g = w.grid
    if mask_radius is not None:
        g = inputs.Grid(g.n1, g.n2, g.n3, g.h, mask_radius)
    s = w.segments
    Z = greens.assemble_columns(g.shape, g.h, s.centre, s.tangent, s.length, w.freq_hz, np.arange(s.m),
                                mask_radius=g.mask_radius)
    return w, g, s, Z


def _uvh(h, g):
    tens, V = h.tensors()
    Zt = products.matvec(tens, g.shape, V.astype(np.complex128).conj().T)
    return Zt, tens, V


@pytest.mark.parametrize("tol", [1e-4, 1e-6])
def test_aca_dense_matches_oracle(tol):
    w, g, s, Z = _case()
    Uo, Vo, info = aca.aca_dense(lambda i: Z[i, :], lambda j: Z[:, j], Z.shape[0], Z.shape[1], tol, 64)
    h, st, piv = zbc.aca_compress(g, zbc.DeviceSegments(s), w.freq_hz, tol, 64, zbc.ACA_DENSE_U, tucker_tol=1e-10)
    assert st.rank == info["rank"]
    assert [tuple(p) for p in piv] == [tuple(p) for p in info["pivots"]]
    assert abs(st.s2 - info["s2"]) <= 1e-9 * info["s2"]
    Zt, _, _ = _uvh(h, g)
    ref = np.linalg.norm(Z - Uo @ Vo.conj().T) / np.linalg.norm(Z)
    err = np.linalg.norm(Z - Zt) / np.linalg.norm(Z)
    assert err <= ref + 1e-6 and err < 30 * tol


def test_aca_dense_masked_rows_and_products():
    w, g, s, Z = _case(mask_radius=0.008)
    assert np.all(Z[0, :] == 0)
    tol = 1e-5
    Uo, Vo, info = aca.aca_dense(lambda i: Z[i, :], lambda j: Z[:, j], Z.shape[0], Z.shape[1], tol, 64)
    h, st, piv = zbc.aca_compress(g, zbc.DeviceSegments(s), w.freq_hz, tol, 64, zbc.ACA_DENSE_U)
    assert st.row_restarts >= 1
    assert [tuple(p) for p in piv] == [tuple(p) for p in info["pivots"]]
    inf = h.info()
    assert inf.has_v == 1 and inf.m == s.m and inf.M == st.rank
    tens, V = h.tensors()
    X = inputs.cn01((s.m, 4), seed=1).astype(np.complex64)
    Y = zbc.colmajor(3 * g.nv, 4, torch.complex64)
    for prec in (zbc.FP32_SIMT, zbc.TF32X3, zbc.BF16X3):
        zbc.zbc_matvec(h, zbc.to_colmajor(X), Y, prec)
        torch.cuda.synchronize()
        Yo = products.matvec_aca(tens, V.astype(np.complex128), g.shape, X)
        e = np.linalg.norm(zbc.from_colmajor(Y) - Yo, axis=0) / np.linalg.norm(Yo, axis=0)
        assert e.max() < 1e-5
    Phi = inputs.cn01((3 * g.nv, 4), seed=2).astype(np.complex64)
    Psi = zbc.colmajor(s.m, 4, torch.complex64)
    zbc.zbc_rmatvec(h, zbc.to_colmajor(Phi), Psi, zbc.FP32_SIMT)
    torch.cuda.synchronize()
    Po = products.rmatvec_aca(tens, V.astype(np.complex128), g.shape, Phi)
    e = np.linalg.norm(zbc.from_colmajor(Psi) - Po, axis=0) / np.linalg.norm(Po, axis=0)
    assert e.max() < 1e-5


def test_algorithm3_against_oracle():
    w, g, s, Z = _case()
    tol = 1e-5
    Ut, Vt, info = aca.aca_tucker(lambda i: Z[i, :], lambda j: Z[:, j], g.shape, 3, Z.shape[1], tol, 64)
    h, st, piv = zbc.aca_compress(g, zbc.DeviceSegments(s), w.freq_hz, tol, 64, zbc.ACA_ALG3)
    assert abs(st.rank - info["rank"]) <= 2
    assert [tuple(p) for p in piv[:3]] == [tuple(p) for p in info["pivots"][:3]]
    Zt, _, _ = _uvh(h, g)
    err = np.linalg.norm(Z - Zt) / np.linalg.norm(Z)
    assert err < 30 * tol
    assert st.max_tucker_err <= 3 * tol * (1 + 1e-9)
