"""Pins of the oracle's Tucker model and truncated HOSVD (Eq. Tucker, Sec. II.B.1)."""
import itertools

import numpy as np
import pytest

from oracle import greens, tucker
from paper_2103_06393_gb300 import inputs


def _orth(n, r, rng):
    a = rng.normal(size=(n, r)) + 1j * rng.normal(size=(n, r))
    q, _ = np.linalg.qr(a)
    return q


def _planted(n, r, rng, decay=None):
    G = rng.normal(size=r) + 1j * rng.normal(size=r)
    if decay is not None:
        G = G * decay
    Us = [_orth(n[g], r[g], rng) for g in range(3)]
    return G, Us


def test_mode_product_against_loops():
    rng = np.random.default_rng(0)
    G = rng.normal(size=(2, 3, 2)) + 1j * rng.normal(size=(2, 3, 2))
    Us = [rng.normal(size=(4, 2)) + 1j * rng.normal(size=(4, 2)),
          rng.normal(size=(3, 3)) + 0j, rng.normal(size=(5, 2)) * 1j]
    A = tucker.reconstruct(G, Us)
    B = np.zeros((4, 3, 5), dtype=complex)
    for i, j, k in itertools.product(range(4), range(3), range(5)):
        for a, b, c in itertools.product(range(2), range(3), range(2)):
            B[i, j, k] += G[a, b, c] * Us[0][i, a] * Us[1][j, b] * Us[2][k, c]
    assert np.allclose(A, B, rtol=1e-13, atol=1e-13)
    assert np.isclose(tucker.element(G, Us, 3, 1, 4), B[3, 1, 4], rtol=1e-13)
    # P = G x1 U1: P[i,b,c] = sum_a G[a,b,c] U1[i,a]
    P = tucker.mode_product(G, Us[0], 0)
    assert np.isclose(P[1, 2, 0], sum(G[a, 2, 0] * Us[0][1, a] for a in range(2)), rtol=1e-13)


def test_fold_is_column_major():
    n = (3, 4, 2)
    col = np.arange(24)
    A = tucker.fold(col, n)
    for i1, i2, i3 in itertools.product(range(3), range(4), range(2)):
        assert A[i1, i2, i3] == i1 + 3 * (i2 + 4 * i3)


@pytest.mark.parametrize("r", [(1, 1, 1), (3, 2, 4), (5, 5, 5)])
def test_planted_rank_recovered(r):
    rng = np.random.default_rng(1)
    n = (9, 10, 11)
    G, Us = _planted(n, r, rng)
    A = tucker.reconstruct(G, Us)
    G2, U2, info = tucker.hosvd(A, 1e-12)
    assert info["ranks"] == r
    assert np.linalg.norm(tucker.reconstruct(G2, U2) - A) <= 1e-12 * np.linalg.norm(A)
    for U in U2:
        assert np.allclose(U.conj().T @ U, np.eye(U.shape[1]), atol=1e-13)


def test_separable_tensor_rank_one():
    rng = np.random.default_rng(2)
    a, b, c = (rng.normal(size=n) + 1j * rng.normal(size=n) for n in (6, 7, 8))
    A = np.einsum("i,j,k->ijk", a, b, c)
    _, _, info = tucker.hosvd(A, 1e-10)
    assert info["ranks"] == (1, 1, 1)


def test_truncation_rule_known_sequence():
    s = np.array([1.0, 0.1, 0.01, 0.001, 0.0001])
    norm2 = float(np.sum(s ** 2))
    # thr = tol^2/3 * norm2; tol chosen so that thr sits between tails
    tail = lambda r: float(np.sum(s[r:] ** 2))
    for r_expect in (1, 2, 3, 4):
        thr = 0.5 * (tail(r_expect) + tail(r_expect - 1)) if r_expect > 1 else 2 * tail(1)
        tol = np.sqrt(3 * thr / norm2)
        r, _ = tucker.truncation_rank(s, norm2, tol)
        assert r == r_expect
    r, _ = tucker.truncation_rank(s, norm2, 1e-30)
    assert r == 5


def test_hosvd_error_bound_on_green_tensor():
    w = inputs.scaled_workload("tiny", (12, 12, 12), m=4)
    g, s = w.grid, w.segments
    Z = greens.assemble_columns(g.shape, g.h, s.centre, s.tangent, s.length, w.freq_hz, [0, 2])
    for tol in (1e-3, 1e-6, 1e-9):
        for j in range(2):
            for k in range(3):
                A = tucker.fold(Z[k * g.nv:(k + 1) * g.nv, j], g.shape)
                G, Us, info = tucker.hosvd(A, tol)
                err2 = np.linalg.norm(tucker.reconstruct(G, Us) - A) ** 2
                tails = sum(float(np.sum(info["sigma"][m][info["ranks"][m]:] ** 2)) for m in range(3))
                assert err2 <= tails * (1 + 1e-8) + 1e-30
                assert tails <= tol ** 2 * info["norm2"] * (1 + 1e-12)
                assert max(info["ranks"]) < 12 or tol < 1e-8


def test_zero_tensor():
    G, Us, info = tucker.hosvd(np.zeros((4, 5, 6), dtype=complex), 1e-6)
    assert info["ranks"] == (1, 1, 1)
    assert np.all(tucker.reconstruct(G, Us) == 0)
