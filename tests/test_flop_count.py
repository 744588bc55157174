"""Pin of the algorithmic flop count (Table III, Sec. III.B) that sets every TFLOP/s figure of
the bench and of the reference arm: Algorithm 1 run as explicit loops on tiny Tucker tensors,
counting one complex multiply-add per innermost iteration, in the paper's decompression order
(x1, x2, x3 mode products, then Y^k += Z^{kj}(:) X_{j:}).  The loops' result is checked against
the dense product, so the count belongs to a correct computation; both counters (the oracle's
and the bench's) must equal 8 x the counted MACs."""
import numpy as np
import pytest

import bench
from oracle import products, tucker


def _tensors(n, ranks, seed):
    rng = np.random.default_rng(seed)
    out = []
    for rj in ranks:
        col = []
        for r in rj:
            G = rng.normal(size=r) + 1j * rng.normal(size=r)
            Us = [rng.normal(size=(n[g], r[g])) + 1j * rng.normal(size=(n[g], r[g])) for g in range(3)]
            col.append((G, Us))
        out.append(col)
    return out


def _counted_matvec(tens, n, X):
    """Algorithm 1 with every complex MAC counted; returns (Y, macs)."""
    n1, n2, n3 = n
    nv = n1 * n2 * n3
    q = len(tens[0])
    p = X.shape[1]
    Y = np.zeros((q * nv, p), dtype=complex)
    macs = 0
    for j, tj in enumerate(tens):
        for k, (G, (U1, U2, U3)) in enumerate(tj):
            r1, r2, r3 = G.shape
            A = np.zeros((n1, r2, r3), dtype=complex)           # G x1 U1
            for i1 in range(n1):
                for b in range(r2):
                    for c in range(r3):
                        for a in range(r1):
                            A[i1, b, c] += G[a, b, c] * U1[i1, a]
                            macs += 1
            B = np.zeros((n1, n2, r3), dtype=complex)           # x2 U2
            for i1 in range(n1):
                for i2 in range(n2):
                    for c in range(r3):
                        for b in range(r2):
                            B[i1, i2, c] += A[i1, b, c] * U2[i2, b]
                            macs += 1
            Z = np.zeros((n1, n2, n3), dtype=complex)           # x3 U3
            for i1 in range(n1):
                for i2 in range(n2):
                    for i3 in range(n3):
                        for c in range(r3):
                            Z[i1, i2, i3] += B[i1, i2, c] * U3[i3, c]
                            macs += 1
            z = Z.reshape(-1, order="F")
            for v in range(nv):                                  # Y^k += Z^{kj}(:) X_{j:}
                for s in range(p):
                    Y[k * nv + v, s] += z[v] * X[j, s]
                    macs += 1
    return Y, macs


@pytest.mark.parametrize("n,ranks,p", [
    ((3, 4, 2), [[(1, 2, 1), (2, 2, 2), (3, 1, 2)], [(2, 3, 1), (1, 1, 1), (3, 4, 2)]], 2),
    ((2, 3, 5), [[(2, 3, 4), (1, 1, 1), (2, 1, 3)]], 3),
    ((4, 2, 3), [[(4, 2, 3), (2, 2, 2), (1, 2, 3)], [(1, 1, 1), (3, 1, 2), (2, 2, 1)],
                 [(2, 1, 1), (1, 2, 2), (4, 1, 3)]], 1),
])
def test_table3_count_equals_counted_loops(n, ranks, p):
    tens = _tensors(n, [[r for r in rj] for rj in ranks], seed=len(ranks) + p)
    q, M = len(tens[0]), len(tens)
    X = np.random.default_rng(1).normal(size=(M, p)) + 0j
    Y, macs = _counted_matvec(tens, n, X)
    Zd = np.stack([np.concatenate([tucker.reconstruct(G, Us).reshape(-1, order="F") for G, Us in tj])
                   for tj in tens], axis=1)
    assert np.allclose(Y, Zd @ X, rtol=1e-12, atol=1e-12)
    rk = np.array([[G.shape for G, _ in tj] for tj in tens])
    assert products.flops(rk, n, q, M, p) == 8.0 * macs
    assert bench.table3_flops(rk, n, q, M, p) == 8.0 * macs


def test_aca_term_is_the_v_product():
    """With ACA storage the count adds X' = V^H X: r_c m p complex MACs (Table III, last row)."""
    n, rk, p, m = (2, 2, 2), np.ones((3, 3, 3), dtype=int), 4, 7
    base = bench.table3_flops(rk, n, 3, 3, p)
    V = np.ones((m, 3))
    X = np.ones((m, p))
    macs = 0
    Xp = np.zeros((3, p))
    for l in range(3):
        for s in range(p):
            for e in range(m):
                Xp[l, s] += V[e, l] * X[e, s]
                macs += 1
    assert bench.table3_flops(rk, n, 3, 3, p, m_aca=m) - base == 8.0 * macs
