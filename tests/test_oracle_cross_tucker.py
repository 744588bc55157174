"""Pins of the fibre-cross Tucker oracle (oracle/cross_tucker.py; end of Sec. II.B.1 and Sec. V)
against facts that do not come from the oracle itself: LAPACK's partial pivoting, exact Tucker
ranks planted in random tensors, the interpolation property of the cross, the HOSVD of the
assembled column, and the direct evaluation of every fibre."""
import numpy as np
import pytest
import scipy.linalg

from oracle import cross_tucker as xt
from oracle import greens, tucker
from paper_2103_06393_gb300 import inputs


def _planted(n, r, seed):
    rng = np.random.default_rng(seed)
    G = rng.normal(size=r) + 1j * rng.normal(size=r)
    Us = [np.linalg.qr(rng.normal(size=(ni, ri)) + 1j * rng.normal(size=(ni, ri)))[0] for ni, ri in zip(n, r)]
    return tucker.reconstruct(G, Us)


def _green_tensor(w, e, k):
    g, s = w.grid, w.segments
    Z = greens.assemble_columns(g.shape, g.h, s.centre, s.tangent, s.length, w.freq_hz, [e],
                                mask_radius=g.mask_radius, mask_box=g.mask_box)[:, 0]
    return tucker.fold(Z[k * g.nv:(k + 1) * g.nv], g.shape)


@pytest.mark.parametrize("n,w,seed", [(30, 7, 0), (12, 12, 1), (50, 3, 2)])
def test_greedy_pivots_are_lapack_partial_pivoting(n, w, seed):
    # on a real matrix, choosing the row of largest modulus in the eliminated column is exactly
    # the row order of LAPACK's getrf with partial pivoting (scipy.linalg.lu: P = p l u)
    P = np.random.default_rng(seed).normal(size=(n, w))
    p, _, _ = scipy.linalg.lu(P)
    lapack = np.argmax(p, axis=0)[:w]   # P[lapack[c]] is row c of p^T P
    assert np.array_equal(xt.greedy_pivots(P, w), lapack)


def test_greedy_pivots_of_a_scaled_permutation():
    perm = np.array([4, 0, 3, 1, 2])
    P = np.zeros((5, 5), dtype=complex)
    P[perm, np.arange(5)] = [2.0, -1j, 0.5, 3.0 + 1j, -0.1]
    assert np.array_equal(xt.greedy_pivots(P, 5), perm)
    # an exhausted column takes the lowest free row and eliminates nothing
    Z = np.zeros((4, 2))
    Z[2, 0] = 1.0
    assert np.array_equal(xt.greedy_pivots(Z, 2), [2, 0])


def test_spread_indices():
    assert list(xt.spread_indices(16, 4)) == [2, 6, 10, 14]
    assert list(xt.spread_indices(3, 8)) == [0, 1, 2]
    assert list(xt.spread_indices(96, 1)) == [48]


@pytest.mark.parametrize("n,r", [((20, 17, 12), (5, 3, 4)), ((16, 16, 16), (7, 7, 2)), ((9, 30, 11), (2, 6, 3))])
def test_planted_ranks_recovered_exactly(n, r):
    A = _planted(n, r, seed=sum(r))
    G, Us, info = xt.cross_tucker(xt.dense_source(A), n, 1e-10)
    assert info["ranks"] == r
    assert xt.error_vs_dense(A, G, Us) < 1e-12
    for U in Us:
        assert np.allclose(U.conj().T @ U, np.eye(U.shape[1]), atol=1e-13)


def test_separable_tensor_is_rank_one():
    rng = np.random.default_rng(5)
    a, b, c = (rng.normal(size=m) + 1j * rng.normal(size=m) for m in (14, 10, 8))
    A = np.einsum("i,j,k->ijk", a, b, c)
    G, Us, info = xt.cross_tucker(xt.dense_source(A), A.shape, 1e-8)
    assert info["ranks"] == (1, 1, 1)
    assert xt.error_vs_dense(A, G, Us) < 1e-14


def test_zero_tensor():
    A = np.zeros((8, 6, 4), dtype=complex)
    G, Us, info = xt.cross_tucker(xt.dense_source(A), A.shape, 1e-6)
    assert info["ranks"] == (1, 1, 1)
    assert np.all(G == 0) and np.all(np.isfinite(Us[0]))


def test_model_interpolates_the_cross():
    # G x1 U1 x2 U2 x3 U3 equals the tensor on every entry of J1 x J2 x J3, whatever the ranks
    w = inputs.scaled_workload("precision", (24, 20, 16), m=3)
    A = _green_tensor(w, 1, 2)
    G, Us, info = xt.cross_tucker(xt.dense_source(A), A.shape, 1e-3)
    J = info["cross"]
    At = tucker.reconstruct(G, Us)
    sub = np.ix_(J[0], J[1], J[2])
    assert np.max(np.abs(At[sub] - A[sub])) <= 1e-12 * np.max(np.abs(A))
    # and not elsewhere (the tolerance leaves a visible error off the cross)
    assert np.max(np.abs(At - A)) > 1e3 * 1e-12 * np.max(np.abs(A))


@pytest.mark.parametrize("tol", [1e-4, 1e-6, 1e-8])
def test_green_columns_against_hosvd(tol):
    # the fibre ranks track the HOSVD ranks of the assembled column, and the error stays at the
    # level of tol (the cross certifies no bound; 2 tol covers the measured cases)
    w = inputs.scaled_workload("precision", (32, 24, 20), m=4)
    for e in range(4):
        for k in range(3):
            A = _green_tensor(w, e, k)
            _, _, ih = tucker.hosvd(A, tol)
            G, Us, info = xt.cross_tucker(xt.dense_source(A), A.shape, tol)
            assert all(abs(a - b) <= 2 for a, b in zip(info["ranks"], ih["ranks"])), (info["ranks"], ih["ranks"])
            assert xt.error_vs_dense(A, G, Us) <= 2 * tol


def test_green_source_indexes_the_column():
    # entries evaluated voxel by voxel (v = i1 + n1 (i2 + n2 i3)) are the assembled column's
    w = inputs.scaled_workload("precision", (12, 10, 8), m=2)
    g, s = w.grid, w.segments
    for k in range(3):
        A = _green_tensor(w, 1, k)
        src = xt.green_source(g.shape, g.h, s.centre, s.tangent, s.length, w.freq_hz, 1, k, mask_radius=g.mask_radius, mask_box=g.mask_box)
        i1, i2, i3 = np.meshgrid(np.arange(12), np.arange(10), np.arange(8), indexing="ij")
        assert np.array_equal(src(i1, i2, i3), A)


def test_check_error_over_all_fibres_is_the_true_error():
    # the check-fibre estimate taken over every fibre of one mode is ||A - model||_F / ||model||_F
    w = inputs.scaled_workload("precision", (16, 12, 10), m=2)
    A = _green_tensor(w, 0, 1)
    G, Us, _ = xt.cross_tucker(xt.dense_source(A), A.shape, 1e-4)
    M = tucker.reconstruct(G, Us)
    true = np.linalg.norm(A - M) / np.linalg.norm(M)
    for checks in ([(0, i2, i3) for i3 in range(10) for i2 in range(12)],
                   [(2, i1, i2) for i2 in range(12) for i1 in range(16)]):
        est = xt.check_error(xt.dense_source(A), G, Us, A.shape, checks)
        assert est == pytest.approx(true, rel=1e-9)
    # random fibres estimate it within a small factor
    rnd = inputs.cross_check_fibres(A.shape, 64, seed=1)
    assert 0.3 * true < xt.check_error(xt.dense_source(A), G, Us, A.shape, rnd) < 3 * true
    # and a mode-2 and a mode-3 fibre agree with slicing the model
    assert np.allclose(xt.tucker_fibre(G, Us, 1, 3, 7), M[3, :, 7], rtol=0, atol=1e-15 * np.abs(M).max())
    assert np.allclose(xt.tucker_fibre(G, Us, 2, 5, 2), M[5, 2, :], rtol=0, atol=1e-15 * np.abs(M).max())


def test_entries_grow_linearly():
    # entries evaluated = sweeps x sum_g n_g |I_a||I_b| + r1 r2 r3: far fewer than n_v once the
    # side is large (the memory the method saves, Sec. V)
    w = inputs.scaled_workload("precision", (64, 64, 64), m=2)
    A = _green_tensor(w, 0, 0)
    G, Us, info = xt.cross_tucker(xt.dense_source(A), A.shape, 1e-6)
    assert info["entries"] < A.size / 2
    assert xt.error_vs_dense(A, G, Us) <= 2e-6
