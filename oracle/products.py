"""Algorithms 1 and 2 of the paper (Sec. III.B) by their plain definition, FP64.

The compressed matrix is a list over columns j of a list over components k of
Tucker tensors (G, [U1, U2, U3]).  Algorithm 1 decompresses Z^{kj} and accumulates
Y^k += Z^{kj}(:) X[j, :]; Algorithm 2 forms Y[j, :] = [Z^{1j}(:); ...; Z^{qj}(:)]^H X.
With ACA first (Z = U V^*), the same loops run over the r_c columns of U with
X <- V^* X before Algorithm 1 and Y <- V Y after Algorithm 2 (Sec. III.B).
"""
import numpy as np

from . import tucker


def matvec(tensors, n, X) -> np.ndarray:
    """Algorithm 1: Y = Z X, Z given column-wise as Tucker tensors; X is M x p."""
    X = np.asarray(X, dtype=np.complex128)
    if X.ndim == 1:
        X = X[:, None]
    n1, n2, n3 = n
    nv = n1 * n2 * n3
    q = len(tensors[0])
    Y = np.zeros((q * nv, X.shape[1]), dtype=np.complex128)
    for j, tj in enumerate(tensors):
        for k in range(q):
            G, Us = tj[k][0], tj[k][1]
            z = tucker.reconstruct(G, Us).reshape(-1, order="F")
            Y[k * nv:(k + 1) * nv, :] += np.outer(z, X[j, :])
    return Y


def rmatvec(tensors, n, Phi) -> np.ndarray:
    """Algorithm 2: Psi = Z^H Phi; Phi is (q n_v) x p, Psi is M x p."""
    Phi = np.asarray(Phi, dtype=np.complex128)
    if Phi.ndim == 1:
        Phi = Phi[:, None]
    Psi = np.zeros((len(tensors), Phi.shape[1]), dtype=np.complex128)
    for j, tj in enumerate(tensors):
        col = tucker.decompress_column(tj, n)
        Psi[j, :] = col.conj() @ Phi
    return Psi


def matvec_rows(tensors, n, X, rows) -> np.ndarray:
    """Selected rows of Algorithm 1's result (row = k*n_v + v), via element-wise
    Tucker evaluation (Algorithm 3's row fetch) -- for sampled parity at sizes
    where the full product is too slow on a CPU."""
    X = np.asarray(X, dtype=np.complex128)
    if X.ndim == 1:
        X = X[:, None]
    n1, n2, n3 = n
    nv = n1 * n2 * n3
    rows = np.asarray(rows)
    out = np.zeros((rows.size, X.shape[1]), dtype=np.complex128)
    ks = rows // nv
    vs = rows % nv
    i1 = vs % n1
    i2 = (vs // n1) % n2
    i3 = vs // (n1 * n2)
    for j, tj in enumerate(tensors):
        for k in range(len(tj)):
            sel = np.nonzero(ks == k)[0]
            if sel.size == 0:
                continue
            G, Us = tj[k][0], tj[k][1]
            # t[s] = sum_abc G[a,b,c] U1[i1_s,a] U2[i2_s,b] U3[i3_s,c]
            t = np.einsum("abc,sa,sb,sc->s", G, Us[0][i1[sel]], Us[1][i2[sel]], Us[2][i3[sel]],
                          optimize=True)
            out[sel, :] += np.outer(t, X[j, :])
    return out


def matvec_aca(tensors_u, V, n, X) -> np.ndarray:
    """Sec. III.B with ACA: Y = U (V^H X), U given as Tucker tensors (r_c columns), V is m x r_c."""
    Xp = np.asarray(V).conj().T @ np.asarray(X, dtype=np.complex128).reshape(V.shape[0], -1)
    return matvec(tensors_u, n, Xp)


def rmatvec_aca(tensors_u, V, n, Phi) -> np.ndarray:
    """Sec. III.B with ACA: Psi = V (U^H Phi)."""
    return np.asarray(V) @ rmatvec(tensors_u, n, Phi)


def flops(ranks, n, q, M, p) -> float:
    """Algorithmic real-flop count of one product (Table III terms, complex MAC = 8 flops):
    8*sum_{j,k} (n1 r1 r2 r3 + n1 n2 r2 r3 + n_v r3) + 8 q n_v M p.
    ranks: array (M, q, 3)."""
    n1, n2, n3 = n
    nv = n1 * n2 * n3
    r = np.asarray(ranks, dtype=np.float64)
    r1, r2, r3 = r[..., 0], r[..., 1], r[..., 2]
    dec = (n1 * r1 * r2 * r3 + n1 * n2 * r2 * r3 + nv * r3).sum()
    return 8.0 * dec + 8.0 * q * nv * M * p
