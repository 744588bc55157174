"""Tucker model and truncated HOSVD (FP64).

Paper Eq. Tucker (Sec. II.B.1): A = G x1 U1 x2 U2 x3 U3, i.e.
    A[i, j, k] = sum_{a,b,c} G[a, b, c] U1[i, a] U2[j, b] U3[k, c],
with unitary factors U^g (n_g x r_g) and core G (r1 x r2 x r3).  The n-mode product
P = G x1 U1 is P[i, b, c] = sum_a G[a, b, c] U1[i, a].

Truncated HOSVD (Sec. II.B.1, De Lathauwer et al. 2000, used at tolerance 1e-8 in
Sec. IV.A and at 3*eps inside Algorithm 3): U^g = leading left singular vectors of
the mode-g unfolding; the core is A x1 U1^H x2 U2^H x3 U3^H.

Truncation rule (reading of "relative error similar to the tolerance", Sec. IV.A):
keep the smallest r_g with  sum_{i > r_g} sigma_i^(g)^2 <= (tol^2 / 3) ||A||_F^2,
so that De Lathauwer's bound gives ||A - A~||_F <= tol ||A||_F.  A mode keeps at
least rank 1 (an all-zero tensor gets a 1x1x1 zero core).
"""
import numpy as np


def fold(col: np.ndarray, n) -> np.ndarray:
    """Column segment of length n1*n2*n3 -> tensor, v = i1 + n1*(i2 + n2*i3) (Fig. 2 reshape)."""
    return np.reshape(np.asarray(col), tuple(n), order="F")


def unfold(A: np.ndarray, mode: int) -> np.ndarray:
    """Mode-g unfolding: n_g x (product of the other sizes)."""
    return np.moveaxis(A, mode, 0).reshape(A.shape[mode], -1)


def mode_product(T: np.ndarray, U: np.ndarray, mode: int) -> np.ndarray:
    """T x_mode U: contracts axis `mode` of T (size r) with the columns of U (n x r)."""
    Tm = np.moveaxis(T, mode, 0)
    out = np.tensordot(U, Tm, axes=([1], [0]))
    return np.moveaxis(out, 0, mode)


def reconstruct(G: np.ndarray, Us) -> np.ndarray:
    """Eq. Tucker: G x1 U1 x2 U2 x3 U3, in the paper's mode order."""
    A = mode_product(G, Us[0], 0)
    A = mode_product(A, Us[1], 1)
    return mode_product(A, Us[2], 2)


def element(G: np.ndarray, Us, i1: int, i2: int, i3: int) -> complex:
    """One entry G x1 U1[i1,:] x2 U2[i2,:] x3 U3[i3,:] (Algorithm 3, element-wise row fetch)."""
    t = np.tensordot(Us[0][i1, :], G, axes=([0], [0]))   # (r2, r3)
    t = np.tensordot(Us[1][i2, :], t, axes=([0], [0]))    # (r3,)
    return complex(np.dot(Us[2][i3, :], t))


def truncation_rank(sigma: np.ndarray, norm2: float, tol: float):
    """Smallest r >= 1 with sum_{i>r} sigma_i^2 <= (tol^2/3) norm2.

    Returns (r, margin): margin is the smallest relative distance
    |tail(r') - thr| / thr over r' in {r-1, r} (the decisions that fixed r), used
    to recognise near-ties where either neighbouring rank is a correct answer.
    """
    s2 = np.asarray(sigma, dtype=np.float64) ** 2
    thr = (tol * tol / 3.0) * norm2
    n = s2.size
    # tail[r] = sum_{i >= r} s2[i] (0-based), tail[n] = 0
    tail = np.zeros(n + 1)
    tail[:n] = np.cumsum(s2[::-1])[::-1]
    r = n
    for cand in range(1, n + 1):
        if tail[cand] <= thr:
            r = cand
            break
    if thr <= 0:
        return r, np.inf
    margins = [abs(tail[r] - thr) / thr]
    if r - 1 >= 1:
        margins.append(abs(tail[r - 1] - thr) / thr)
    return r, float(min(margins))


def hosvd(A: np.ndarray, tol: float):
    """Truncated HOSVD of a 3D complex tensor.

    Returns (G, [U1, U2, U3], info) with info = {'sigma': [s1, s2, s3], 'ranks': (r1, r2, r3),
    'margin': (m1, m2, m3), 'norm2': ||A||_F^2}.
    """
    A = np.asarray(A, dtype=np.complex128)
    norm2 = float(np.vdot(A, A).real)
    Us, sig, ranks, margins = [], [], [], []
    for g in range(3):
        U, s, _ = np.linalg.svd(unfold(A, g), full_matrices=False)
        r, mg = truncation_rank(s, norm2, tol)
        Us.append(np.ascontiguousarray(U[:, :r]))
        sig.append(s)
        ranks.append(r)
        margins.append(mg)
    G = mode_product(A, Us[0].conj().T, 0)
    G = mode_product(G, Us[1].conj().T, 1)
    G = mode_product(G, Us[2].conj().T, 2)
    return G, Us, {"sigma": sig, "ranks": tuple(ranks), "margin": tuple(margins), "norm2": norm2}


def compress_columns(Z: np.ndarray, n, q: int, tol: float):
    """Sec. III.A / Fig. 2: every column of Z (q*n_v x m) -> q Tucker tensors.

    Returns a list over columns j of a list over components k of (G, [U1, U2, U3], info).
    """
    n1, n2, n3 = n
    nv = n1 * n2 * n3
    out = []
    for j in range(Z.shape[1]):
        comps = []
        for k in range(q):
            comps.append(hosvd(fold(Z[k * nv:(k + 1) * nv, j], n), tol))
        out.append(comps)
    return out


def decompress_column(tensors_j, n) -> np.ndarray:
    """Concatenate the q decompressed tensors of one column (Algorithm 1, 'Decompress Z^{kj}')."""
    return np.concatenate([reconstruct(G, Us).reshape(-1, order="F") for (G, Us, *_rest) in tensors_j])
