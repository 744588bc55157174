"""Tucker compression of a column from a few of its fibres (3D cross-Tucker), FP64.

Test infrastructure: only the tests, the smoke check and the benchmark's CPU legs import this
module; the library never calls it.

The paper offers this as the way around assembling a whole column when the tensor is too large
for the HOSVD of Sec. II.B.1 (end of Sec. II.B.1 and Sec. V, citing the linear-time Tucker
approximation of Oseledets, Savostyanov and Tyrtyshnikov, SIAM J. Matrix Anal. Appl. 30 (2008)):
the factors come from a few rows, columns and fibres of the tensor, so the work and the memory
grow linearly with its side.  The paper gives no algorithm of its own; this module is a plain
statement of the alternating fibre cross of that reference, in this reading:

  index sets I_g of each mode g (I_2, I_3 start as s0 evenly spread indices);
  a sweep visits g = 1, 2, 3 and, with a < b the other two modes,
    F_g   = the n_g x |I_a||I_b| matrix of mode-g fibres A(.., i_a, .., i_b, ..) through
            every pair of I_a x I_b (column c <-> (I_a[c mod |I_a|], I_b[c div |I_a|]));
    F_g   = P S Q^H (SVD);  r_g = the smallest r with sum_{i>r} s_i^2 <= ((tol/4)^2/3) ||F_g||_F^2
            (the HOSVD rule of Sec. II.B.1 on the sampled fibres, at a quarter of the tolerance:
            the fibres the pivots pick carry less of the tail than the whole unfolding), at most
            rmax;
    U_g   = P[:, :r_g];
    I_g   = the first w_g = min(r_g + over, n_g, |I_a||I_b|) rows chosen by greedy pivoting on
            P[:, :w_g] (Gaussian elimination with the row of largest modulus as pivot);
  a fixed number of sweeps (2 by default: a third changed no error in the measured cases);
  the core interpolates the tensor on the cross J_1 x J_2 x J_3 of the first r_g pivots:
    M_g = U_g[J_g, :] (square, nonsingular by the pivoting),
    G   = A[J_1, J_2, J_3] x1 M_1^-1 x2 M_2^-1 x3 M_3^-1,
  so that G x1 U_1 x2 U_2 x3 U_3 equals A on every entry of the cross.
The error is estimated on check fibres the caller draws (the tensor is never formed whole).
"""
import numpy as np

from . import greens
from .tucker import mode_product, reconstruct, truncation_rank

OTHER = {0: (1, 2), 1: (0, 2), 2: (0, 1)}
RANK_TOL_FACTOR = 0.25   # the rank rule on the fibres runs at tol / 4


def spread_indices(n: int, s: int) -> np.ndarray:
    """s indices spread evenly over [0, n): floor((2l + 1) n / (2 s)), l < s."""
    s = min(s, n)
    return np.array([((2 * l + 1) * n) // (2 * s) for l in range(s)], dtype=np.int64)


def greedy_pivots(P: np.ndarray, w: int) -> np.ndarray:
    """Rows chosen by Gaussian elimination with complete row search on the first w columns of P:
    step c takes the row of largest |R[i, c]| among rows not yet chosen (lowest index on ties),
    then removes that row's multiple from every row.  A column with no nonzero left takes the
    lowest unchosen row and eliminates nothing."""
    R = np.array(P[:, :w], dtype=np.complex128)
    n = R.shape[0]
    chosen = []
    free = np.ones(n, dtype=bool)
    for c in range(w):
        mag = np.where(free, np.abs(R[:, c]), -1.0)
        i = int(np.argmax(mag))          # first maximum: lowest index on ties
        chosen.append(i)
        free[i] = False
        piv = R[i, c]
        if mag[i] > 0.0:
            R -= np.outer(R[:, c] / piv, R[i, :])
    return np.array(chosen, dtype=np.int64)


def fibre_matrix(entry, n, g: int, Ia: np.ndarray, Ib: np.ndarray) -> np.ndarray:
    """n_g x (|Ia| |Ib|) mode-g fibres through Ia x Ib (a < b the other modes)."""
    a, b = OTHER[g]
    ca = np.tile(np.asarray(Ia, dtype=np.int64), len(Ib))      # column c -> Ia[c mod |Ia|]
    cb = np.repeat(np.asarray(Ib, dtype=np.int64), len(Ia))    #            Ib[c div |Ia|]
    idx = [None, None, None]
    idx[g] = np.broadcast_to(np.arange(n[g])[:, None], (n[g], ca.size))
    idx[a] = np.broadcast_to(ca[None, :], (n[g], ca.size))
    idx[b] = np.broadcast_to(cb[None, :], (n[g], ca.size))
    return np.asarray(entry(idx[0], idx[1], idx[2]), dtype=np.complex128)


def cross_tucker(entry, n, tol: float, rmax: int = 64, over: int = 4, s0: int = 8, sweeps: int = 2):
    """Tucker model of the tensor whose entries entry(i1, i2, i3) returns (index arrays in,
    complex values out), from fibres only.  Returns (G, [U1, U2, U3], info) with info =
    {'ranks', 'index_sets' (I_1..I_3 with the oversampling), 'cross' (J_1..J_3), 'entries'
    (tensor entries evaluated)}."""
    n = tuple(int(v) for v in n)
    I = [spread_indices(n[0], s0), spread_indices(n[1], s0), spread_indices(n[2], s0)]
    Us = [None, None, None]
    ranks = [0, 0, 0]
    entries = 0
    for _ in range(sweeps):
        for g in range(3):
            a, b = OTHER[g]
            F = fibre_matrix(entry, n, g, I[a], I[b])
            entries += F.size
            P, sv, _ = np.linalg.svd(F, full_matrices=False)
            norm2 = float(np.vdot(F, F).real)
            r, _ = truncation_rank(sv, norm2, RANK_TOL_FACTOR * tol)
            r = min(r, rmax, n[g], F.shape[1])
            w = min(r + over, n[g], F.shape[1])
            Us[g] = P[:, :r]
            ranks[g] = r
            I[g] = greedy_pivots(P, w)
    J = [I[g][:ranks[g]] for g in range(3)]
    C = entry(*np.meshgrid(J[0], J[1], J[2], indexing="ij"))
    entries += C.size
    G = np.asarray(C, dtype=np.complex128)
    for g in range(3):
        G = mode_product(G, np.linalg.inv(Us[g][J[g], :]), g)
    return G, [np.ascontiguousarray(U) for U in Us], {
        "ranks": tuple(ranks), "index_sets": I, "cross": J, "entries": entries}


def tucker_fibre(G, Us, g: int, ia: int, ib: int) -> np.ndarray:
    """The mode-g fibre of G x1 U1 x2 U2 x3 U3 through (ia, ib) (a < b the other modes)."""
    a, b = OTHER[g]
    T = mode_product(G, Us[a][ia:ia + 1, :], a)
    T = mode_product(T, Us[b][ib:ib + 1, :], b)
    return mode_product(T, Us[g], g).reshape(-1)


def check_error(entry, G, Us, n, checks) -> float:
    """Relative Frobenius error of the Tucker model estimated from the check fibres (g, ia, ib):
    a mode-g fibre drawn uniformly stands for all n_a n_b of them, so
        e^2 = (1 / #checks) sum_checks n_a n_b ||A_fibre - model_fibre||^2
    estimates ||A - model||_F^2, and the result is e / ||G||_F (= e / ||model||_F, the factors
    being orthonormal).  0 when both are zero."""
    num = 0.0
    for g, ia, ib in checks:
        a, b = OTHER[int(g)]
        idx = [None, None, None]
        idx[g] = np.arange(n[g])
        idx[a] = np.full(n[g], ia)
        idx[b] = np.full(n[g], ib)
        d = entry(idx[0], idx[1], idx[2]) - tucker_fibre(G, Us, int(g), int(ia), int(ib))
        num += float(n[a]) * n[b] * float(np.vdot(d, d).real)
    num /= len(checks)
    den = float(np.vdot(G, G).real)
    if den == 0.0:
        return 0.0 if num == 0.0 else np.inf
    return float(np.sqrt(num / den))


def dense_source(A: np.ndarray):
    """entry() of a tensor held whole (for tests against the HOSVD and planted ranks)."""
    A = np.asarray(A)
    return lambda i1, i2, i3: A[i1, i2, i3]


def green_source(n, h, centre, tangent, length, freq_hz, e: int, k: int, q: int = 3, mask_radius=0.0,
                 operator="N", nq=1, mask_box=0.0):
    """entry() of component k of column e of the coupling matrix (Eq. nNt / Eq. nKt), evaluated
    voxel by voxel from the Green's function (the column is never assembled)."""
    n1, n2, _ = n

    def entry(i1, i2, i3):
        i1, i2, i3 = (np.asarray(v, dtype=np.int64) for v in (i1, i2, i3))
        shape = i1.shape
        v = (i1 + n1 * (i2 + n2 * i3)).reshape(-1)
        z = greens.assemble_columns(n, h, centre, tangent, length, freq_hz, [e], q=q, mask_radius=mask_radius,
                                    rows=v, operator=operator, nq=nq, mask_box=mask_box)[:, 0]
        return z[k * v.size:(k + 1) * v.size].reshape(shape)

    return entry


def compress_columns(n, h, centre, tangent, length, freq_hz, cols, tol: float, q: int = 3, mask_radius=0.0,
                     operator="N", nq=1, checks=(), mask_box=0.0, **kw):
    """Every column e of cols -> q Tucker tensors from fibres of the Green's function; a list over
    columns of a list over components of (G, [U1, U2, U3], info), info['check_err'] on `checks`."""
    out = []
    for e in np.atleast_1d(cols):
        comps = []
        for k in range(q):
            src = green_source(n, h, centre, tangent, length, freq_hz, int(e), k, q, mask_radius, operator, nq,
                               mask_box)
            G, Us, info = cross_tucker(src, n, tol, **kw)
            info["check_err"] = check_error(src, G, Us, n, checks) if len(checks) else None
            comps.append((G, Us, info))
        out.append(comps)
    return out


def error_vs_dense(A: np.ndarray, G, Us) -> float:
    """||A - G x1 U1 x2 U2 x3 U3||_F / ||A||_F for a tensor held whole."""
    d = A - reconstruct(G, Us)
    nrm = np.linalg.norm(A)
    return float(np.linalg.norm(d) / nrm) if nrm > 0 else float(np.linalg.norm(d))
