"""Partially pivoted ACA and Algorithm 3 (Tucker-based ACA), FP64.

Paper Sec. II.B.2: A ~ U V^*, U (m1 x r_c), V (m2 x r_c), built from selected rows
and columns (ACA of Kurz / Bebendorf, in the variant of Zhao et al. 2005).
Paper Sec. III.C, Algorithm 3: the same loop with every new column of U reshaped
into q tensors and stored as truncated-HOSVD Tucker tensors at tolerance 3*eps;
rows of U come from element-wise Tucker evaluation, and the residual column and
the norm update use Algorithms 1 and 2 on the compressed U.

Readings where the paper is silent or garbled:
  * pivots are argmax |.| (magnitude of a complex entry), ties to the lowest index;
    rows and columns already used as pivots are excluded from later argmax;
  * the norm update uses the Frobenius identity
        ||sum_l u_l v_l^H||^2 = sum_l ||u_l||^2 ||v_l||^2 + 2 sum_{l<k} Re{(u_l^H u_k) conj(v_l^H v_k)},
    i.e. Re{(U^H x) . conj(V^H y)} (the algorithm's line prints the product without
    the conjugate);
  * the new column is appended before the stopping test (r_c counts it);
  * the start row is row 0; if a residual row is exactly zero (a masked voxel),
    that row is marked used and the next unused row in index order is tried.

Algorithm 3 takes two optional arguments used by the GPU parity tests:
  * store=np.complex64 rounds every new Tucker tensor (core and factors) to complex64 before
    it joins U, as a GPU handle stores them; the arithmetic stays complex128;
  * trace=True records, per iteration, the residual row r and column x the pivots were taken
    from, so that a test can tell pivots decided by a clear margin from near-ties.
"""
import numpy as np

from . import products, tucker


def _argmax_abs(v: np.ndarray, excluded) -> int:
    a = np.abs(v).astype(np.float64)
    if excluded:
        a[list(excluded)] = -1.0
    return int(np.argmax(a))   # first index among ties


def aca_dense(get_row, get_col, m1: int, m2: int, tol: float, max_rank: int):
    """Plain ACA with a dense U.  get_row(i) -> Z[i, :] (m2), get_col(j) -> Z[:, j] (m1).

    Returns (U (m1 x r), V (m2 x r), info) with Z ~ U V^H.
    """
    U = np.zeros((m1, 0), dtype=np.complex128)
    V = np.zeros((m2, 0), dtype=np.complex128)
    used_r, used_c = set(), set()
    s2 = 0.0
    i = 0
    pivots = []
    converged = False
    for k in range(min(m1, m2, max_rank)):
        while True:
            r = np.asarray(get_row(i), dtype=np.complex128).copy()
            if k > 0:
                r -= U[i, :] @ V.conj().T
            used_r.add(i)
            rr = np.abs(r).copy()
            if used_c:
                rr[list(used_c)] = 0.0
            if rr.max() > 0.0:
                break
            free = [t for t in range(m1) if t not in used_r]
            if not free:
                return U, V, {"rank": U.shape[1], "pivots": pivots, "s2": s2, "converged": True}
            i = free[0]
        j = _argmax_abs(r, used_c)
        y = (r / r[j]).conj()
        x = np.asarray(get_col(j), dtype=np.complex128).copy()
        if k > 0:
            x -= U @ V[j, :].conj()
        nx, ny = np.linalg.norm(x), np.linalg.norm(y)
        s2 += (nx * ny) ** 2
        if k > 0:
            s2 += 2.0 * np.sum(((U.conj().T @ x) * (V.conj().T @ y).conj()).real)
        U = np.concatenate([U, x[:, None]], axis=1)
        V = np.concatenate([V, y[:, None]], axis=1)
        used_c.add(j)
        pivots.append((i, j))
        if nx * ny <= tol * np.sqrt(s2):
            converged = True
            break
        a = np.abs(x)
        i = _argmax_abs(a, used_r)
    return U, V, {"rank": U.shape[1], "pivots": pivots, "s2": s2, "converged": converged}


def _stored(t, store):
    """A new tensor (G, Us, info) as U keeps it: rounded to `store` (complex64) when given."""
    if store is None:
        return t
    G, Us, info = t
    rnd = lambda a: np.asarray(a).astype(store).astype(np.complex128)
    return (rnd(G), [rnd(U) for U in Us], info)


def aca_tucker(get_row, get_col, n, q: int, m2: int, tol: float, max_rank: int, tucker_tol=None,
               store=None, trace=False, compress=None):
    """Algorithm 3: ACA of Z (q n_v x m2) with U assembled directly as Tucker tensors.

    Returns (tensors_u, V, info): tensors_u[l][k] = (G, [U1, U2, U3], hosvd_info).
    store: None (complex128 tensors) or np.complex64 (tensors rounded as a GPU handle stores them).
    trace: info["trace"][k] = {"r": row residual, "x": column residual, "nx", "ny", "s2"}.
    compress: callable(A, tol) -> (G, [U1, U2, U3], info) used for U's tensors in place of the
    truncated HOSVD (e.g. the randomized Tucker of oracle.randomized with its certified bound).
    """
    if compress is None:
        compress = tucker.hosvd
    n1, n2, n3 = n
    nv = n1 * n2 * n3
    m1 = q * nv
    ttol = 3.0 * tol if tucker_tol is None else tucker_tol
    steps = []
    Ut = []
    V = np.zeros((m2, 0), dtype=np.complex128)
    used_r, used_c = set(), set()
    s2 = 0.0
    i = 0
    pivots = []
    converged = False
    for k in range(min(m1, m2, max_rank)):
        while True:
            r = np.asarray(get_row(i), dtype=np.complex128).copy()
            if k > 0:
                kk, v = divmod(i, nv)
                f1, f2, f3 = v % n1, (v // n1) % n2, v // (n1 * n2)
                t = np.array([tucker.element(Ut[l][kk][0], Ut[l][kk][1], f1, f2, f3)
                              for l in range(len(Ut))])
                r -= t @ V.conj().T
            used_r.add(i)
            rr = np.abs(r).copy()
            if used_c:
                rr[list(used_c)] = 0.0
            if rr.max() > 0.0:
                break
            free = [t for t in range(m1) if t not in used_r]
            if not free:
                return Ut, V, {"rank": len(Ut), "pivots": pivots, "s2": s2, "converged": True}
            i = free[0]
        j = _argmax_abs(r, used_c)
        y = (r / r[j]).conj()
        x = np.asarray(get_col(j), dtype=np.complex128).copy()
        if k > 0:
            x -= products.matvec(Ut, n, V[j, :].conj()[:, None])[:, 0]
        nx, ny = np.linalg.norm(x), np.linalg.norm(y)
        s2 += (nx * ny) ** 2
        if k > 0:
            uhx = products.rmatvec(Ut, n, x[:, None])[:, 0]
            s2 += 2.0 * np.sum((uhx * (V.conj().T @ y).conj()).real)
        Ut.append([_stored(compress(tucker.fold(x[kk * nv:(kk + 1) * nv], n), ttol), store)
                   for kk in range(q)])
        V = np.concatenate([V, y[:, None]], axis=1)
        used_c.add(j)
        pivots.append((i, j))
        if trace:
            steps.append({"r": r, "x": x, "nx": nx, "ny": ny, "s2": s2})
        if nx * ny <= tol * np.sqrt(s2):
            converged = True
            break
        a = np.abs(x)
        i = _argmax_abs(a, used_r)
    info = {"rank": len(Ut), "pivots": pivots, "s2": s2, "converged": converged}
    if trace:
        info["trace"] = steps
    return Ut, V, info
