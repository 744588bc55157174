"""GPU parity of the C-ABI path against the FP64 oracle: assembly, HOSVD compression and the
FP32 SIMT products (Algorithms 1 and 2), with ragged grids, several right-hand-side counts,
ACA storage, checkpoints and error statuses."""

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

RTOL_FP32 = 1e-5   # relative L2 per right-hand side for the FP32 paths


def rel_cols(a, b):
    return np.linalg.norm(a - b, axis=0) / np.linalg.norm(b, axis=0)


def dense(w, cols=None):
    g, s = w.grid, w.segments
    cols = np.arange(s.m) if cols is None else cols
    return greens.assemble_columns(g.shape, g.h, s.centre, s.tangent, s.length, w.freq_hz, cols,
                                   mask_radius=g.mask_radius, mask_box=g.mask_box)


def gpu_assemble(w, dtype=torch.complex128, cols=None):
    g, s = w.grid, w.segments
    cols = np.arange(s.m) if cols is None else np.asarray(cols)
    ds = zbc.DeviceSegments(s)
    cd = torch.from_numpy(cols.astype(np.int32)).cuda()
    Z = zbc.colmajor(3 * g.nv, cols.size, dtype)
    zbc.vsie_assemble_columns(g, ds, w.freq_hz, cd, Z)
    torch.cuda.synchronize()
    return Z


def c64(tens):
    """Round an oracle Tucker list to complex64 storage and back (what the GPU holds)."""
    return [[(t[0].astype(np.complex64).astype(np.complex128),
              [U.astype(np.complex64).astype(np.complex128) for U in t[1]]) for t in tj] for tj in tens]


# ------------------------------------------------------------------------------------------
# assembly
# ------------------------------------------------------------------------------------------

def test_assembly_fp64_matches_oracle():
    w = inputs.workload("tiny")
    Zg = zbc.from_colmajor(gpu_assemble(w))
    Zo = dense(w)
    assert rel_cols(Zg, Zo).max() < 1e-13


def test_assembly_complex64_and_mask_exact():
    w = inputs.scaled_workload("batching", (20, 18, 16), m=12)
    g = inputs.Grid(20, 18, 16, w.grid.h, mask_radius=0.012)
    w = inputs.Workload(w.name, g, w.segments, w.freq_hz, w.tol, w.p)
    Zo = dense(w)
    Z64 = zbc.from_colmajor(gpu_assemble(w))
    assert np.array_equal(Z64 == 0, Zo == 0)       # the mask is decided identically
    assert (Zo == 0).any()
    Z32 = zbc.from_colmajor(gpu_assemble(w, torch.complex64))
    assert rel_cols(Z32, Zo).max() < 1e-7


def test_assembly_box_mask_exact():
    w = inputs.scaled_workload("batching", (20, 18, 16), m=12)
    g = inputs.Grid(20, 18, 16, w.grid.h, mask_box=0.0105)
    w = inputs.Workload(w.name, g, w.segments, w.freq_hz, w.tol, w.p)
    Zo = dense(w)
    Z64 = zbc.from_colmajor(gpu_assemble(w))
    assert np.array_equal(Z64 == 0, Zo == 0)
    assert (Zo == 0).any() and (Zo != 0).any()
    assert rel_cols(Z64, Zo).max() < 1e-13


def test_assembly_out_of_range_column_is_zero():
    w = inputs.scaled_workload("tiny", (6, 6, 6), m=4)
    Z = zbc.from_colmajor(gpu_assemble(w, cols=[0, 7, -1, 3]))
    assert np.all(Z[:, 1] == 0) and np.all(Z[:, 2] == 0) and np.all(Z[:, 0] != 0)


# ------------------------------------------------------------------------------------------
# HOSVD compression
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("name,n,m,tol", [("tiny", (24, 24, 24), 16, 1e-8),
                                          ("tiny", (24, 24, 24), 16, 1e-6),
                                          ("precision", (32, 32, 32), 6, 1e-6),
                                          ("precision", (40, 24, 18), 4, 1e-4)])
def test_hosvd_ranks_and_error_bound(name, n, m, tol):
    w = inputs.scaled_workload(name, n, m=m)
    g = w.grid
    Zd = gpu_assemble(w)
    h, st = zbc.tucker_compress(Zd, g, tol)
    tens, _ = h.tensors()
    Z = zbc.from_colmajor(Zd)
    ties = 0
    for j in range(m):
        for k in range(3):
            A = tucker.fold(Z[k * g.nv:(k + 1) * g.nv, j], g.shape)
            _, _, info = tucker.hosvd(A, tol)
            gr = tuple(U.shape[1] for U in tens[j][k][1])
            for mode in range(3):
                if info["margin"][mode] < 1e-5:
                    ties += 1
                    assert abs(gr[mode] - info["ranks"][mode]) <= 1
                else:
                    assert gr[mode] == info["ranks"][mode], (j, k, mode, gr, info["ranks"], info["margin"])
            Ar = tucker.reconstruct(tens[j][k][0], tens[j][k][1])
            err = np.linalg.norm(Ar - A) / np.linalg.norm(A)
            # the FP64 bound is tol; complex64 storage adds ~1e-7
            assert err <= tol * (1 + 1e-6) + 3e-7, (j, k, err)
            for U in tens[j][k][1]:
                assert np.abs(U.conj().T @ U - np.eye(U.shape[1])).max() < 1e-6
    assert ties <= 2
    assert st.max_rel_err <= tol * (1 + 1e-9)


def test_hosvd_append_and_info():
    w = inputs.scaled_workload("tiny", (16, 16, 16), m=6)
    Zd = gpu_assemble(w)
    h, _ = zbc.tucker_compress(Zd[:4], w.grid, 1e-6)
    h, _ = zbc.tucker_compress(Zd[4:], w.grid, 1e-6, append_to=h)
    inf = h.info()
    assert inf.M == 6 and inf.m == 6 and inf.q == 3
    h2, _ = zbc.tucker_compress(Zd, w.grid, 1e-6)
    r1, p1, _ = h.export()
    r2, p2, _ = h2.export()
    assert np.array_equal(r1, r2)
    tucker_b, v_b, full_b = h.memory_bytes()
    ranks = [tuple(r) for r in r1.reshape(-1, 3)]
    from oracle import memory
    assert tucker_b == 8 * memory.tucker_entries(ranks, w.grid.shape)
    assert full_b == 8 * memory.full_entries(3, w.grid.nv, 6) and v_b == 0


# ------------------------------------------------------------------------------------------
# products (FP32 SIMT)
# ------------------------------------------------------------------------------------------

def _oracle_handle(w, tol, V=None):
    Z = dense(w)
    tens = c64(tucker.compress_columns(Z, w.grid.shape, 3, tol))
    h = zbc.zbc_create_from_host(w.grid, 3, tens, V)
    return h, tens


def _run(h, w, tens, p, prec, V=None, seed=0):
    g = w.grid
    m = len(tens) if V is None else V.shape[0]
    X = inputs.cn01((m, p), seed=seed).astype(np.complex64)
    Phi = inputs.cn01((3 * g.nv, p), seed=seed + 1).astype(np.complex64)
    Y = zbc.colmajor(3 * g.nv, p, torch.complex64)
    Psi = zbc.colmajor(m, p, torch.complex64)
    zbc.zbc_matvec(h, zbc.to_colmajor(X), Y, prec)
    zbc.zbc_rmatvec(h, zbc.to_colmajor(Phi), Psi, prec)
    zbc.zbc_product_status(h)   # synchronises; raises if a kernel gave up a bounded wait
    if V is None:
        Yo = products.matvec(tens, g.shape, X)
        Po = products.rmatvec(tens, g.shape, Phi)
    else:
        Vc = V.astype(np.complex64).astype(np.complex128)
        Yo = products.matvec_aca(tens, Vc, g.shape, X)
        Po = products.rmatvec_aca(tens, Vc, g.shape, Phi)
    return zbc.from_colmajor(Y), Yo, zbc.from_colmajor(Psi), Po, X, Phi


@pytest.mark.parametrize("p", [1, 2, 3, 16, 20])
def test_simt_products_tiny(p):
    w = inputs.workload("tiny")
    h, tens = _oracle_handle(w, 1e-8)
    Y, Yo, P, Po, _, _ = _run(h, w, tens, p, zbc.FP32_SIMT)
    assert rel_cols(Y, Yo).max() < RTOL_FP32
    assert rel_cols(P, Po).max() < RTOL_FP32


@pytest.mark.parametrize("n", [(13, 11, 7), (33, 9, 3), (40, 17, 5)])
def test_simt_products_ragged_tiles(n):
    w = inputs.scaled_workload("precision", n, m=5)
    h, tens = _oracle_handle(w, 1e-5)
    Y, Yo, P, Po, _, _ = _run(h, w, tens, 5, zbc.FP32_SIMT, seed=3)
    assert rel_cols(Y, Yo).max() < RTOL_FP32
    assert rel_cols(P, Po).max() < RTOL_FP32


@pytest.mark.parametrize("n", [(160, 7, 3), (257, 5, 2)])
def test_simt_products_several_i1_tiles(n):
    # n1 > 128: more than one i1 tile, the last one partly padding
    w = inputs.scaled_workload("precision", n, m=6)
    h, tens = _oracle_handle(w, 1e-5)
    Y, Yo, P, Po, _, _ = _run(h, w, tens, 5, zbc.FP32_SIMT, seed=4)
    assert rel_cols(Y, Yo).max() < RTOL_FP32
    assert rel_cols(P, Po).max() < RTOL_FP32


def _random_tensors(n, M, seed, rmax=7):
    """M columns x 3 components of random Tucker tensors with ranks 1..rmax (odd and even),
    orthonormal factors, complex64-exact."""
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
    return c64(out)


def test_simt_products_many_columns():
    # 2500 stored columns: many turns of the copy pipeline's stages, and more columns than one
    # adjoint CTA keeps sums for (the j range is split into blocks)
    n = (8, 6, 5)
    tens = _random_tensors(n, 2500, seed=11)
    grid = inputs.Grid(*n, 0.002)
    h = zbc.zbc_create_from_host(grid, 3, tens)
    w = inputs.Workload("random", grid, None, 0.0, 0.0, 16)
    Y, Yo, P, Po, _, _ = _run(h, w, tens, 16, zbc.FP32_SIMT, seed=5)
    assert rel_cols(Y, Yo).max() < RTOL_FP32
    assert rel_cols(P, Po).max() < RTOL_FP32


def test_simt_adjoint_identity():
    w = inputs.scaled_workload("precision", (32, 32, 32), m=12)
    h, tens = _oracle_handle(w, 1e-6)
    Y, Yo, P, Po, X, Phi = _run(h, w, tens, 4, zbc.FP32_SIMT, seed=7)
    lhs = np.vdot(Phi, Y)          # Phi^H (Z X)
    rhs = np.vdot(P, X)            # (Z^H Phi)^H X
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


def test_simt_aca_storage():
    w = inputs.scaled_workload("precision", (16, 16, 16), m=5)
    rng = np.random.default_rng(0)
    V = (rng.normal(size=(9, 5)) + 1j * rng.normal(size=(9, 5)))
    h, tens = _oracle_handle(w, 1e-6, V=V)
    assert h.info().has_v == 1 and h.info().m == 9
    Y, Yo, P, Po, _, _ = _run(h, w, tens, 3, zbc.FP32_SIMT, V=V)
    assert rel_cols(Y, Yo).max() < RTOL_FP32
    assert rel_cols(P, Po).max() < RTOL_FP32


def test_save_load_roundtrip(tmp_path):
    w = inputs.scaled_workload("tiny", (12, 12, 12), m=3)
    h, tens = _oracle_handle(w, 1e-6)
    path = str(tmp_path / "z.zbc")
    h.save(path)
    h2 = zbc.zbc_load(path)
    r1, p1, _ = h.export()
    r2, p2, _ = h2.export()
    assert np.array_equal(r1, r2) and np.array_equal(p1, p2)
    with open(path, "r+b") as f:
        f.write(b"XXXX")
    with pytest.raises(zbc.ZbcError) as e:
        zbc.zbc_load(path)
    assert e.value.status == zbc.ZBC_EIO


def test_error_statuses():
    w = inputs.scaled_workload("tiny", (8, 8, 8), m=2)
    h, tens = _oracle_handle(w, 1e-6)
    X = zbc.colmajor(2, 1, torch.complex64)
    Ysmall = torch.zeros((1, 10), dtype=torch.complex64, device="cuda")
    with pytest.raises(zbc.ZbcError) as e:
        zbc.zbc_matvec(h, X, Ysmall)
    assert e.value.status == zbc.ZBC_EINVAL
    assert "ldy" in str(e.value)
