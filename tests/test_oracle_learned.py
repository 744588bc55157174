"""Pins of the randomized Tucker and the rank-predictor MLP oracles (no counterpart in
the paper): planted ranks, the error bound, agreement with HOSVD, finite differences."""
import numpy as np
import pytest

from oracle import mlp, randomized, tucker
from paper_2103_06393_gb300 import inputs


def _orth(n, r, rng):
    q, _ = np.linalg.qr(rng.normal(size=(n, r)) + 1j * rng.normal(size=(n, r)))
    return q


def _sketches(shape, width, seed):
    n1, n2, n3 = shape
    return [inputs.gaussian_sketch(n2 * n3, width, seed),
            inputs.gaussian_sketch(n1 * n3, width, seed + 1),
            inputs.gaussian_sketch(n1 * n2, width, seed + 2)]


def test_unfold_f_column_order():
    A = np.arange(2 * 3 * 4).reshape((2, 3, 4), order="F")
    U1 = randomized.unfold_f(A, 0)
    assert U1[1, 2 + 3 * 1] == A[1, 2, 1]
    U2 = randomized.unfold_f(A, 1)
    assert U2[2, 1 + 2 * 3] == A[1, 2, 3]
    U3 = randomized.unfold_f(A, 2)
    assert U3[3, 1 + 2 * 2] == A[1, 2, 3]


def test_randomized_recovers_planted_rank():
    rng = np.random.default_rng(0)
    n, r = (12, 13, 14), (3, 4, 2)
    G = rng.normal(size=r) + 1j * rng.normal(size=r)
    A = tucker.reconstruct(G, [_orth(n[g], r[g], rng) for g in range(3)])
    Gr, Ur, info = randomized.randomized_tucker(A, (7, 8, 6), _sketches(n, 8, 10), 1e-10)
    assert not info["fallback"]
    assert info["ranks"] == r
    assert np.linalg.norm(tucker.reconstruct(Gr, Ur) - A) <= 1e-10 * np.linalg.norm(A)


def test_randomized_falls_back_when_width_too_small():
    rng = np.random.default_rng(1)
    n, r = (10, 10, 10), (6, 6, 6)
    G = rng.normal(size=r) + 1j * rng.normal(size=r)
    A = tucker.reconstruct(G, [_orth(n[g], r[g], rng) for g in range(3)])
    Gr, Ur, info = randomized.randomized_tucker(A, (3, 3, 3), _sketches(n, 3, 4), 1e-6)
    assert info["fallback"]
    Gh, Uh, infoh = tucker.hosvd(A, 1e-6)
    assert info["ranks"] == infoh["ranks"]


def test_randomized_error_bound_on_smooth_tensor():
    x = np.linspace(0.3, 1.0, 16)
    A = 1.0 / (x[:, None, None] + 2 * x[None, :, None] + 3 * x[None, None, :]) + 0j
    tol = 1e-6
    _, _, infoh = tucker.hosvd(A, tol)
    widths = [r + 4 for r in infoh["ranks"]]
    Gr, Ur, info = randomized.randomized_tucker(A, widths, _sketches(A.shape, max(widths), 7), tol)
    assert not info["fallback"]
    err = np.linalg.norm(tucker.reconstruct(Gr, Ur) - A) / np.linalg.norm(A)
    assert err <= tol


def test_mlp_gradients_finite_differences():
    params = mlp.init_params(0)
    rng = np.random.default_rng(1)
    X = rng.normal(size=(5, 7))
    T = rng.normal(size=(5, 9))
    out, cache = mlp.forward(params, X)
    grads = mlp.backward(params, cache, out, T)
    eps = 1e-6
    for li in range(4):
        W, b = params[li]
        for (a, c) in [(0, 0), (3, 2), (W.shape[0] - 1, W.shape[1] - 1)]:
            Wp, Wm = W.copy(), W.copy()
            Wp[a, c] += eps
            Wm[a, c] -= eps
            pp = list(params); pp[li] = (Wp, b)
            pm = list(params); pm[li] = (Wm, b)
            fd = (mlp.loss(mlp.forward(pp, X)[0], T) - mlp.loss(mlp.forward(pm, X)[0], T)) / (2 * eps)
            assert abs(fd - grads[li][0][a, c]) <= 1e-6 * max(1.0, abs(fd))
        bp, bm = b.copy(), b.copy()
        bp[1] += eps
        bm[1] -= eps
        pp = list(params); pp[li] = (W, bp)
        pm = list(params); pm[li] = (W, bm)
        fd = (mlp.loss(mlp.forward(pp, X)[0], T) - mlp.loss(mlp.forward(pm, X)[0], T)) / (2 * eps)
        assert abs(fd - grads[li][1][1]) <= 1e-6 * max(1.0, abs(fd))


def test_adam_reduces_loss():
    params = mlp.init_params(3)
    rng = np.random.default_rng(4)
    X = rng.normal(size=(64, 7))
    T = np.tanh(X @ rng.normal(size=(7, 9)))
    state = {}
    l0 = mlp.loss(mlp.forward(params, X)[0], T)
    for _ in range(200):
        out, cache = mlp.forward(params, X)
        params = mlp.adam_step(params, mlp.backward(params, cache, out, T), state, lr=3e-3)
    assert mlp.loss(mlp.forward(params, X)[0], T) < 0.2 * l0
