"""Fixed-width randomized range-finder Tucker with an HOSVD fallback (FP64).

Not in the paper: the paper compresses every tensor with a truncated HOSVD
(Sec. II.B.1) and names a cross-based Tucker as future work.  This follows the
randomized range finder of Halko, Martinsson and Tropp (2011, Alg. 4.1) applied
per mode as in the randomized HOSVD of Minster, Saibaba and Kilmer (2020):

  1. for each mode g: Y_g = A_(g) Omega_g[:, :l_g]  (l_g = predicted rank + oversampling),
     Q_g = orthonormal basis of range(Y_g)  (Householder QR);
  2. C = A x1 Q1^H x2 Q2^H x3 Q3^H  (l1 x l2 x l3);
  3. projection error e^2 = ||A||^2 - ||C||^2 (exact: Q_g orthonormal);
  4. if e^2 > tol^2 ||A||^2 the predicted width failed -> fallback to HOSVD;
  5. otherwise truncate C by HOSVD with the remaining budget (tol^2 ||A||^2 - e^2)/3
     per mode: U_g = Q_g W_g, G = C x W^H.  Total error <= tol ||A||_F.

Unfolding column order is fixed here (the sketches are inputs shared with the GPU):
  mode 1 columns (i2, i3) with i2 fastest; mode 2 columns (i1, i3) with i1 fastest;
  mode 3 columns (i1, i2) with i1 fastest.

Parity against the paper: unpinned (no counterpart); pinned instead by planted-rank
tensors, the error bound and agreement with HOSVD reconstructions.
"""
import numpy as np

from . import tucker


def unfold_f(A: np.ndarray, mode: int) -> np.ndarray:
    n1, n2, n3 = A.shape
    if mode == 0:
        return A.reshape(n1, n2 * n3, order="F")
    if mode == 1:
        return np.transpose(A, (1, 0, 2)).reshape(n2, n1 * n3, order="F")
    return np.transpose(A, (2, 0, 1)).reshape(n3, n1 * n2, order="F")


def randomized_tucker(A: np.ndarray, widths, sketches, tol: float):
    """Returns (G, [U1,U2,U3], info); info['fallback'] is True when step 4 failed
    (then the result is the plain HOSVD)."""
    A = np.asarray(A, dtype=np.complex128)
    norm2 = float(np.vdot(A, A).real)
    Qs = []
    for g in range(3):
        lg = int(min(widths[g], A.shape[g]))
        Y = unfold_f(A, g) @ np.asarray(sketches[g])[:, :lg]
        Q, _ = np.linalg.qr(Y)
        Qs.append(Q)
    C = tucker.mode_product(A, Qs[0].conj().T, 0)
    C = tucker.mode_product(C, Qs[1].conj().T, 1)
    C = tucker.mode_product(C, Qs[2].conj().T, 2)
    e2 = max(norm2 - float(np.vdot(C, C).real), 0.0)
    budget = tol * tol * norm2 - e2
    if budget < 0.0 or norm2 == 0.0:
        G, Us, info = tucker.hosvd(A, tol)
        info = dict(info)
        info.update(fallback=True, proj_err2=e2)
        return G, Us, info
    Ws, ranks, margins = [], [], []
    # truncation with per-mode threshold budget/3, i.e. tol_eff^2/3 * ||C||^2 = budget/3
    for g in range(3):
        U, s, _ = np.linalg.svd(tucker.unfold(C, g), full_matrices=False)
        s2 = s ** 2
        thr = budget / 3.0
        tail = np.zeros(s2.size + 1)
        tail[:s2.size] = np.cumsum(s2[::-1])[::-1]
        r = s2.size
        for cand in range(1, s2.size + 1):
            if tail[cand] <= thr:
                r = cand
                break
        mg = [abs(tail[r] - thr) / thr] if thr > 0 else [np.inf]
        if r - 1 >= 1 and thr > 0:
            mg.append(abs(tail[r - 1] - thr) / thr)
        Ws.append(U[:, :r])
        ranks.append(r)
        margins.append(float(min(mg)))
    G = tucker.mode_product(C, Ws[0].conj().T, 0)
    G = tucker.mode_product(G, Ws[1].conj().T, 1)
    G = tucker.mode_product(G, Ws[2].conj().T, 2)
    Us = [Qs[g] @ Ws[g] for g in range(3)]
    return G, Us, {"ranks": tuple(ranks), "margin": tuple(margins), "norm2": norm2,
                   "fallback": False, "proj_err2": e2}
