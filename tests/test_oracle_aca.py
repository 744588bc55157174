"""Pins of the oracle's ACA and Algorithm 3 (Sec. II.B.2, Sec. III.C)."""
import numpy as np

from oracle import aca, greens, products, tucker
from paper_2103_06393_gb300 import inputs


def test_exact_rank_matrix_stops():
    rng = np.random.default_rng(0)
    r = 5
    A = (rng.normal(size=(60, r)) + 1j * rng.normal(size=(60, r))) @ (rng.normal(size=(r, 40)) + 1j * rng.normal(size=(r, 40)))
    U, V, info = aca.aca_dense(lambda i: A[i, :], lambda j: A[:, j], 60, 40, 1e-10, 40)
    assert info["rank"] in (r, r + 1)
    assert np.linalg.norm(A - U @ V.conj().T) <= 1e-12 * np.linalg.norm(A)


def test_norm_estimate_is_frobenius_identity():
    """s_k must equal ||U V^H||_F^2 exactly (reading of the norm update with the conjugate)."""
    rng = np.random.default_rng(1)
    A = rng.normal(size=(50, 30)) + 1j * rng.normal(size=(50, 30))
    A = A * np.exp(-0.3 * np.arange(30))[None, :]
    U, V, info = aca.aca_dense(lambda i: A[i, :], lambda j: A[:, j], 50, 30, 1e-30, 12)
    assert info["rank"] == 12
    assert np.isclose(info["s2"], np.linalg.norm(U @ V.conj().T) ** 2, rtol=1e-12)


def test_aca_interpolates_pivots():
    rng = np.random.default_rng(2)
    A = rng.normal(size=(20, 15)) + 1j * rng.normal(size=(20, 15))
    U, V, info = aca.aca_dense(lambda i: A[i, :], lambda j: A[:, j], 20, 15, 1e-30, 6)
    R = U @ V.conj().T
    for (i, j) in info["pivots"]:
        assert np.allclose(R[i, :], A[i, :], atol=1e-12) and np.allclose(R[:, j], A[:, j], atol=1e-12)


def _green_case(mask_radius=None):
    w = inputs.scaled_workload("batching", (8, 8, 6), m=48)
    g, s = w.grid, w.segments
    if mask_radius is not None:
        g = inputs.Grid(g.n1, g.n2, g.n3, g.h, mask_radius)
    Z = greens.assemble_columns(g.shape, g.h, s.centre, s.tangent, s.length, w.freq_hz, np.arange(s.m),
                                mask_radius=g.mask_radius, mask_box=g.mask_box)
    return g, Z


def test_aca_error_tracks_tolerance_on_green_matrix():
    g, Z = _green_case()
    for tol in (1e-3, 1e-6):
        U, V, info = aca.aca_dense(lambda i: Z[i, :], lambda j: Z[:, j], Z.shape[0], Z.shape[1], tol, 48)
        err = np.linalg.norm(Z - U @ V.conj().T) / np.linalg.norm(Z)
        assert err < 30 * tol
        assert info["rank"] < 48


def test_algorithm3_matches_dense_aca():
    g, Z = _green_case()
    tol = 1e-5
    Ud, Vd, infod = aca.aca_dense(lambda i: Z[i, :], lambda j: Z[:, j], Z.shape[0], Z.shape[1], tol, 48)
    Ut, Vt, infot = aca.aca_tucker(lambda i: Z[i, :], lambda j: Z[:, j], g.shape, 3, Z.shape[1], tol, 48,
                                   tucker_tol=1e-12)
    # with a near-exact Tucker tolerance, Algorithm 3 reproduces plain ACA
    assert infot["pivots"] == infod["pivots"]
    Zt = products.matvec(Ut, g.shape, Vt.conj().T)       # U V^H assembled through Algorithm 1
    assert np.linalg.norm(Zt - Ud @ Vd.conj().T) <= 1e-9 * np.linalg.norm(Z)
    # at the paper's 3*eps Tucker tolerance the approximation error stays of the order of tol
    Ut3, Vt3, info3 = aca.aca_tucker(lambda i: Z[i, :], lambda j: Z[:, j], g.shape, 3, Z.shape[1], tol, 48)
    Z3 = products.matvec(Ut3, g.shape, Vt3.conj().T)
    assert np.linalg.norm(Z3 - Z) / np.linalg.norm(Z) < 30 * tol


def test_masked_start_row_is_skipped():
    g, Z = _green_case(mask_radius=0.006)
    assert np.all(Z[0, :] == 0)            # corner voxel is masked
    U, V, info = aca.aca_dense(lambda i: Z[i, :], lambda j: Z[:, j], Z.shape[0], Z.shape[1], 1e-4, 48)
    assert info["pivots"][0][0] != 0


def test_algorithm3_complex64_storage_and_trace():
    """store=complex64 keeps tensors that are exactly complex64 values, still tracks
    the tolerance, and the trace's residuals are Algorithm 3's: x_k = Z[:, j_k] - U_{<k} V[j_k, <k]^H
    on the stored tensors, and r_k = Z[i_k, :] - U_{<k}[i_k, :] V_{<k}^H by element-wise evaluation."""
    g, Z = _green_case()
    tol = 1e-5
    Ut, Vt, info = aca.aca_tucker(lambda i: Z[i, :], lambda j: Z[:, j], g.shape, 3, Z.shape[1], tol, 48,
                                  store=np.complex64, trace=True)
    for col in Ut:
        for G, Us, _ in col:
            for a in [G] + list(Us):
                assert np.array_equal(a, a.astype(np.complex64).astype(np.complex128))
    Zt = products.matvec([[(G, Us) for G, Us, _ in col] for col in Ut], g.shape, Vt.conj().T)
    assert np.linalg.norm(Z - Zt) / np.linalg.norm(Z) < 30 * tol
    assert len(info["trace"]) == info["rank"]
    tens = [[(G, Us) for G, Us, _ in col] for col in Ut]
    for k, (i, j) in enumerate(info["pivots"]):
        st = info["trace"][k]
        x = Z[:, j].copy()
        if k:
            x -= products.matvec(tens[:k], g.shape, Vt[j, :k].conj()[:, None])[:, 0]
        assert np.allclose(st["x"], x, rtol=0, atol=1e-12 * np.abs(Z).max())
        r = Z[i, :].copy()
        if k:
            r -= np.array([tucker.reconstruct(*tens[l][i // g.nv]).reshape(-1, order="F")[i % g.nv]
                           for l in range(k)]) @ Vt[:, :k].conj().T
        assert np.allclose(st["r"], r, rtol=0, atol=1e-12 * np.abs(Z).max())
