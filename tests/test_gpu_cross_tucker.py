"""Tucker compression from fibres on the GPU (cross_tucker_compress / cross_tucker_assemble; end of
Sec. II.B.1 and Sec. V) against the FP64 oracle (oracle/cross_tucker.py): exact planted ranks, the
ranks and the error on Green's function columns, the Green's-function source against the same
entries read from an assembled column, the reported check-fibre error, the products on the
resulting handle, and argument errors."""
import numpy as np
import pytest

from oracle import cross_tucker as xt
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


def _planted(n, r, seed):
    rng = np.random.default_rng(seed)
    G = rng.normal(size=r) + 1j * rng.normal(size=r)
    Us = [np.linalg.qr(rng.normal(size=(ni, ri)) + 1j * rng.normal(size=(ni, ri)))[0] for ni, ri in zip(n, r)]
    return tucker.reconstruct(G, Us)


def _gpu_assemble(w, op="N", nq=1, q=3, cols=None):
    g, s = w.grid, w.segments
    cols = np.arange(s.m) if cols is None else np.asarray(cols)
    cd = torch.from_numpy(cols.astype(np.int32)).cuda()
    Z = zbc.colmajor(q * g.nv, cols.size, torch.complex128)
    zbc.vsie_assemble_columns_op(g, zbc.DeviceSegments(s), w.freq_hz, cd, Z, op=OPS[op], nq=nq, q=q)
    torch.cuda.synchronize()
    return Z


def _recon_err(A, tj):
    G, Us = tj[0], tj[1]
    return np.linalg.norm(A - tucker.reconstruct(G, Us)) / np.linalg.norm(A)


def _checks(n, count, seed):
    return inputs.cross_check_fibres(n, count, seed)


def _ranks(h):
    return h.export()[0]     # [column][component] -> (r1, r2, r3)


@pytest.mark.parametrize("n,r", [((20, 18, 12), (5, 3, 4)), ((16, 16, 16), (7, 7, 2)), ((10, 30, 12), (2, 6, 3))])
def test_planted_ranks(n, r):
    tens_in = [_planted(n, r, seed=sum(r) + k) for k in range(3)]
    cols = np.stack([A.reshape(-1, order="F") for A in tens_in]).T          # 3 columns, q = 1
    Zd = zbc.to_colmajor(cols.astype(np.complex128))
    h, st, xs = zbc.cross_tucker_compress(Zd, inputs.Grid(*n, 0.002), 1e-9, q=1)
    tens, _ = h.tensors()
    ranks = _ranks(h)
    for j, A in enumerate(tens_in):
        _, _, info = xt.cross_tucker(xt.dense_source(A), n, 1e-9)
        assert info["ranks"] == r
        assert tuple(ranks[j][0]) == r
        assert _recon_err(A, tens[j][0]) < 1e-6      # complex64 storage
    assert st.n_tensors == 3 and st.max_rank == max(r)


@pytest.mark.parametrize("tol", [1e-4, 1e-6])
def test_green_columns_match_the_oracle(tol):
    w = inputs.scaled_workload("precision", (24, 20, 16), m=6)
    g = w.grid
    Z = _gpu_assemble(w)
    h, st, xs = zbc.cross_tucker_compress(Z, g, tol, checks=_checks(g.shape, 24, 3))
    tens, _ = h.tensors()
    ranks = _ranks(h)
    Zh = zbc.from_colmajor(Z)
    for j in range(w.segments.m):
        for k in range(3):
            A = tucker.fold(Zh[k * g.nv:(k + 1) * g.nv, j], g.shape)
            _, _, info = xt.cross_tucker(xt.dense_source(A), g.shape, tol)
            assert all(abs(a - b) <= 1 for a, b in zip(ranks[j][k], info["ranks"])), (ranks[j][k], info["ranks"])
            assert _recon_err(A, tens[j][k]) <= 2 * tol + 1e-6
    assert 0 <= xs.max_check_err <= 2 * tol + 1e-6
    assert st.max_rel_err == xs.max_check_err


def test_check_error_is_the_models_error_on_the_fibres():
    w = inputs.scaled_workload("precision", (20, 16, 12), m=3)
    g = w.grid
    Z = _gpu_assemble(w)
    chk = _checks(g.shape, 16, 5)
    h, st, xs = zbc.cross_tucker_compress(Z, g, 1e-3, checks=chk)
    tens, _ = h.tensors()
    Zh = zbc.from_colmajor(Z)
    worst = 0.0
    for j in range(3):
        for k in range(3):
            A = tucker.fold(Zh[k * g.nv:(k + 1) * g.nv, j], g.shape)
            G, Us = tens[j][k][0], tens[j][k][1]
            worst = max(worst, xt.check_error(xt.dense_source(A), G, Us, g.shape, chk))
    # the GPU measures its FP64 model; the stored complex64 model differs by ~1e-7 relative
    assert xs.max_check_err == pytest.approx(worst, rel=0.05, abs=1e-6)


@pytest.mark.parametrize("op,nq,q", [("N", 1, 3), ("K", 3, 3), ("N", 2, 12)])
def test_green_source_equals_assembled_entries(op, nq, q):
    # the entries evaluated fibre by fibre are the assembly's (the same device function), so both
    # sources give the same handle: bit for bit for the point-matched kernel, to rounding where the
    # quadrature's sums may be contracted differently in the two kernels
    w = inputs.scaled_workload("precision", (16, 14, 12), m=4)
    g = w.grid
    Z = _gpu_assemble(w, op, nq, q)
    chk = _checks(g.shape, 8, 7)
    h1, st1, xs1 = zbc.cross_tucker_compress(Z, g, 1e-5, q=q, checks=chk)
    h2, st2, xs2 = zbc.cross_tucker_assemble(g, zbc.DeviceSegments(w.segments), w.freq_hz, np.arange(4), 1e-5, q=q,
                                             op=OPS[op], nq=nq, checks=chk)
    t1, _ = h1.tensors()
    t2, _ = h2.tensors()
    if (op, nq, q) == ("N", 1, 3):
        assert np.array_equal(_ranks(h1), _ranks(h2))
        for j in range(4):
            for k in range(q):
                for a, b in zip([t1[j][k][0], *t1[j][k][1]], [t2[j][k][0], *t2[j][k][1]]):
                    assert np.array_equal(a, b)
        assert xs1.entries == xs2.entries and xs1.max_check_err == xs2.max_check_err
    else:
        # a last-bit difference may move an oversampling pivot: compare the models, not factors
        assert np.abs(_ranks(h1) - _ranks(h2)).max() <= 1
        for j in range(4):
            for k in range(q):
                m1 = tucker.reconstruct(t1[j][k][0], t1[j][k][1])
                m2 = tucker.reconstruct(t2[j][k][0], t2[j][k][1])
                assert np.linalg.norm(m1 - m2) <= 4e-5 * np.linalg.norm(m2)


def test_entries_grow_linearly():
    # a 64^3 grid: the fibres, the cross and the checks take far fewer entries than the column
    w = inputs.scaled_workload("precision", (64, 64, 64), m=2)
    g = w.grid
    h, st, xs = zbc.cross_tucker_assemble(g, zbc.DeviceSegments(w.segments), w.freq_hz, [0, 1], 1e-6,
                                          checks=_checks(g.shape, 12, 9))
    assert xs.entries < 6 * g.nv / 2       # 6 tensors
    assert xs.max_check_err <= 3e-6       # an estimate of the error (about +-30 %)
    Zo = greens.assemble_columns(g.shape, g.h, w.segments.centre, w.segments.tangent, w.segments.length,
                                 w.freq_hz, [1], mask_radius=g.mask_radius, mask_box=g.mask_box)
    tens, _ = h.tensors()
    for k in range(3):
        A = tucker.fold(Zo[k * g.nv:(k + 1) * g.nv, 0], g.shape)
        assert _recon_err(A, tens[1][k]) <= 2e-6


@pytest.mark.parametrize("prec", [zbc.FP32_SIMT, zbc.TC_MODE1])
def test_products_on_a_cross_handle(prec):
    w = inputs.scaled_workload("precision", (24, 20, 16), m=8)
    g = w.grid
    h, _, _ = zbc.cross_tucker_assemble(g, zbc.DeviceSegments(w.segments), w.freq_hz, np.arange(8), 1e-6, op=zbc.OP_K,
                                        nq=3)
    tens, _ = h.tensors()
    p = 6
    X = inputs.cn01((8, p), seed=51).astype(np.complex64)
    Phi = inputs.cn01((3 * g.nv, p), seed=52).astype(np.complex64)
    Y = zbc.colmajor(3 * g.nv, p, torch.complex64)
    Psi = zbc.colmajor(8, p, torch.complex64)
    zbc.zbc_matvec(h, zbc.to_colmajor(X), Y, prec)
    zbc.zbc_rmatvec(h, zbc.to_colmajor(Phi), Psi, prec)
    zbc.zbc_product_status(h)
    rel = lambda a, b: (np.linalg.norm(a - b, axis=0) / np.linalg.norm(b, axis=0)).max()
    assert rel(zbc.from_colmajor(Y), products.matvec(tens, g.shape, X.astype(np.complex128))) < 1e-5
    assert rel(zbc.from_colmajor(Psi), products.rmatvec(tens, g.shape, Phi.astype(np.complex128))) < 1e-5


def test_append_and_parameters():
    w = inputs.scaled_workload("precision", (16, 12, 10), m=4)
    g, ds = w.grid, zbc.DeviceSegments(w.segments)
    h, _, _ = zbc.cross_tucker_assemble(g, ds, w.freq_hz, [0, 1], 1e-5)
    h, _, _ = zbc.cross_tucker_assemble(g, ds, w.freq_hz, [2, 3], 1e-5, append_to=h)
    hall, _, _ = zbc.cross_tucker_assemble(g, ds, w.freq_hz, [0, 1, 2, 3], 1e-5)
    assert h.info().M == 4
    assert np.array_equal(_ranks(h), _ranks(hall))
    # a rank cap of 2 and one sweep: every rank <= 2
    hc, st, _ = zbc.cross_tucker_assemble(g, ds, w.freq_hz, [0], 1e-8, params={"sweeps": 1, "rmax": 2, "over": 1, "s0": 4})
    assert st.max_rank == 2


def test_bad_arguments_rejected():
    w = inputs.scaled_workload("precision", (16, 12, 10), m=2)
    g, ds = w.grid, zbc.DeviceSegments(w.segments)
    cases = [dict(params={"rmax": 65}), dict(params={"over": 17}), dict(params={"sweeps": 17}),
             dict(checks=np.array([[3, 0, 0]])), dict(checks=np.array([[0, 12, 0]])), dict(checks=np.array([[2, 0, 12]]))]
    for kw in cases:
        with pytest.raises(zbc.ZbcError) as e:
            zbc.cross_tucker_assemble(g, ds, w.freq_hz, [0], 1e-5, **kw)
        assert e.value.status == zbc.ZBC_EINVAL, kw
    with pytest.raises(zbc.ZbcError):
        zbc.cross_tucker_assemble(g, ds, w.freq_hz, [2], 1e-5)        # segment out of range
    odd = inputs.Grid(15, 12, 10, g.h)
    with pytest.raises(zbc.ZbcError):
        zbc.cross_tucker_assemble(odd, ds, w.freq_hz, [0], 1e-5)


def test_complex64_columns():
    # the same columns stored complex64: ranks within 1 of the complex128 run, the same error level
    w = inputs.scaled_workload("precision", (20, 16, 12), m=3)
    g = w.grid
    Z = _gpu_assemble(w)
    Z64 = Z.to(torch.complex64)
    h1, _, _ = zbc.cross_tucker_compress(Z, g, 1e-4)
    h2, _, _ = zbc.cross_tucker_compress(Z64, g, 1e-4)
    assert np.abs(_ranks(h1) - _ranks(h2)).max() <= 1
    tens, _ = h2.tensors()
    Zh = zbc.from_colmajor(Z)
    for j in range(3):
        for k in range(3):
            A = tucker.fold(Zh[k * g.nv:(k + 1) * g.nv, j], g.shape)
            assert _recon_err(A, tens[j][k]) <= 2e-4 + 1e-6
