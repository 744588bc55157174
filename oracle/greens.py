"""Coupling-matrix entries from the free-space Green's function (FP64).

Paper: Eq. n6 gives the scalar Helmholtz kernel g = exp(-i k0 R) / (4 pi R); Eq. nNt
defines the N operator built on it and Eq. nKt the K operator (curl of the single-layer
potential) that maps coil currents to magnetic fields; Sec. III.A says each column of the
coupling matrix is the concatenation of q per-component vectors over the voxels, reshaped
column-major into n1 x n2 x n3 tensors (Fig. 2).

Point-matched form used here (one point per voxel; the segment either point-matched at its
centre or integrated with an nq-point Gauss-Legendre rule along it):
    Z[(k, v), e] = h^3 * len_e * sum_q (w_q / 2) [ Kern(r_v - p_eq) t_e ]_k,
    p_eq = c_e + (xi_q len_e / 2) t_e,   (xi_q, w_q) the Gauss-Legendre rule on [-1, 1],
with Kern = G = (I + grad grad / k0^2) g (the N operator) or Kern t = grad g x t (the K
operator, curl(g t) for a constant t).  For R = |r_v - p|, Rhat the unit vector, x = k0 R:
    G = g * [ (1 - i/x - 1/x^2) I + (-1 + 3i/x + 3/x^2) Rhat Rhat^T ],
    grad g = g' Rhat,   g' = -g (i k0 + 1/R).
The closed form of G follows from grad grad g = g'' Rhat Rhat + (g'/R)(I - Rhat Rhat).  One
point (xi = 0, w = 2) is the plain point-matched form.
Row index (k, v) -> k*n_v + v  (Algorithm 1: Y = [Y^1; ...; Y^q]).  For the piecewise-linear
basis (q = 12, Sec. II.A) each voxel carries phi_0 = 1 and the three linear functions
(x - x_c)/h, (y - y_c)/h, (z - z_c)/h per field component, integrated over the voxel with a
2 x 2 x 2 Gauss-Legendre rule; row block b = 3 l + k.
"""
import numpy as np

C0 = 299_792_458.0


def wavenumber(freq_hz: float) -> float:
    return 2.0 * np.pi * freq_hz / C0


def scalar_green(R: np.ndarray, k0: float) -> np.ndarray:
    """Eq. n6."""
    return np.exp(-1j * k0 * R) / (4.0 * np.pi * R)


def dyadic_green(r_obs: np.ndarray, r_src: np.ndarray, k0: float) -> np.ndarray:
    """(I + grad grad / k0^2) g evaluated at r_obs - r_src; inputs (..., 3), output (..., 3, 3)."""
    Rv = np.asarray(r_obs, dtype=np.float64) - np.asarray(r_src, dtype=np.float64)
    R = np.asarray(np.sqrt((Rv * Rv).sum(axis=-1)))
    Rh = Rv / R[..., None]
    x = k0 * R
    g = np.asarray(scalar_green(R, k0))
    a = np.asarray(1.0 - 1j / x - 1.0 / x ** 2)
    b = np.asarray(-1.0 + 3j / x + 3.0 / x ** 2)
    eye = np.eye(3)
    return g[..., None, None] * (a[..., None, None] * eye + b[..., None, None] * Rh[..., :, None] * Rh[..., None, :])


def curl_green(r_obs: np.ndarray, r_src: np.ndarray, t: np.ndarray, k0: float) -> np.ndarray:
    """grad g (r_obs - r_src) x t = curl(g t) for a constant t (Eq. nKt's kernel on a segment);
    inputs (..., 3), output (..., 3)."""
    Rv = np.asarray(r_obs, dtype=np.float64) - np.asarray(r_src, dtype=np.float64)
    R = np.asarray(np.sqrt((Rv * Rv).sum(axis=-1)))
    Rh = Rv / R[..., None]
    gp = -np.asarray(scalar_green(R, k0)) * (1j * k0 + 1.0 / R)    # g'(R)
    return gp[..., None] * np.cross(Rh, np.broadcast_to(t, Rh.shape))


def gauss_legendre(nq: int):
    """Nodes and weights of the nq-point Gauss-Legendre rule on [-1, 1] (library routine)."""
    x, w = np.polynomial.legendre.leggauss(int(nq))
    return x, w


def segment_field(rv: np.ndarray, centre, tangent, length, k0: float, operator: str, nq: int) -> np.ndarray:
    """sum_q (w_q / 2) Kern(rv - p_q) t over the segment's quadrature points; rv (nv, 3) -> (nv, 3)."""
    xs, ws = gauss_legendre(nq)
    f = np.zeros((rv.shape[0], 3), dtype=np.complex128)
    for xq, wq in zip(xs, ws):
        p = np.asarray(centre, dtype=np.float64) + 0.5 * xq * length * np.asarray(tangent, dtype=np.float64)
        if operator == "N":
            f += 0.5 * wq * (dyadic_green(rv, p[None, :], k0) @ tangent)
        elif operator == "K":
            f += 0.5 * wq * curl_green(rv, p[None, :], tangent, k0)
        else:
            raise ValueError(operator)
    return f


def pwl_field(rv: np.ndarray, h: float, centre, tangent, length, k0: float, operator: str, nq: int,
              nvq: int = 2) -> np.ndarray:
    """Piecewise-linear voxel basis (q = 12): for each voxel centre rv (nv, 3), the four basis
    functions phi_0 = 1, phi_1 = (x - x_c)/h, phi_2 = (y - y_c)/h, phi_3 = (z - z_c)/h integrated
    against the segment's field with an nvq^3 Gauss-Legendre rule over the voxel (mean over the
    voxel, i.e. divided by h^3).  Returns (nv, 4, 3): [basis l][component k]."""
    xs, ws = gauss_legendre(nvq)
    out = np.zeros((rv.shape[0], 4, 3), dtype=np.complex128)
    for ix, wx in zip(xs, ws):
        for iy, wy in zip(xs, ws):
            for iz, wz in zip(xs, ws):
                d = 0.5 * np.array([ix, iy, iz])            # offset / h, in [-1/2, 1/2]^3
                f = segment_field(rv + h * d[None, :], centre, tangent, length, k0, operator, nq)
                wgt = wx * wy * wz / 8.0                    # the rule's weights sum to 1
                for l, phi in enumerate((1.0, d[0], d[1], d[2])):
                    out[:, l, :] += wgt * phi * f
    return out


def voxel_centres(n1: int, n2: int, n3: int, h: float) -> np.ndarray:
    """(n_v, 3) centres, v = i1 + n1*(i2 + n2*i3), centred at the origin."""
    a1 = (np.arange(n1) - (n1 - 1) / 2.0) * h
    a2 = (np.arange(n2) - (n2 - 1) / 2.0) * h
    a3 = (np.arange(n3) - (n3 - 1) / 2.0) * h
    x = np.broadcast_to(a1[None, None, :], (n3, n2, n1)).reshape(-1)
    y = np.broadcast_to(a2[None, :, None], (n3, n2, n1)).reshape(-1)
    z = np.broadcast_to(a3[:, None, None], (n3, n2, n1)).reshape(-1)
    return np.stack([x, y, z], axis=1)


def voxel_mask(n1, n2, n3, h, mask_radius, mask_box=0.0) -> np.ndarray:
    """True for voxels kept; voxels with sqrt(x^2+y^2) > mask_radius (if > 0) or with
    max(|x|, |y|) > mask_box (if > 0) are dropped."""
    r = voxel_centres(n1, n2, n3, h)
    keep = np.ones(r.shape[0], dtype=bool)
    if mask_box > 0:
        keep &= (np.abs(r[:, 0]) <= mask_box) & (np.abs(r[:, 1]) <= mask_box)
    if mask_radius > 0:
        keep &= np.sqrt(r[:, 0] ** 2 + r[:, 1] ** 2) <= mask_radius
    return keep


def assemble_columns(n, h, centre, tangent, length, freq_hz, cols, q=3, mask_radius=0.0,
                     rows=None, operator="N", nq=1, mask_box=0.0) -> np.ndarray:
    """Dense columns Z[:, cols] of the (q*n_v) x m coupling matrix, complex128, column-major.

    rows: optional subset of voxel indices v; the result then has q*len(rows) rows
    ordered (k, row-position).  operator: "N" (Eq. nNt, the dyadic kernel) or "K" (Eq. nKt);
    nq: Gauss-Legendre points along each segment (1 = point-matched at the centre).
    q = 3: piecewise-constant basis, point-matched at the voxel centre.  q = 12: piecewise-linear
    basis (pwl_field, 2 x 2 x 2 Gauss points per voxel), row block b = 3 l + k for basis l and
    component k.
    """
    assert q in (3, 12)
    n1, n2, n3 = n
    k0 = wavenumber(freq_hz)
    rv = voxel_centres(n1, n2, n3, h)
    keep = voxel_mask(n1, n2, n3, h, mask_radius, mask_box)
    if rows is not None:
        rows = np.asarray(rows)
        rv = rv[rows]
        keep = keep[rows]
    nv = rv.shape[0]
    cols = np.atleast_1d(np.asarray(cols))
    out = np.zeros((q * nv, cols.size), dtype=np.complex128, order="F")
    for jj, e in enumerate(cols):
        if q == 12:
            f = pwl_field(rv, h, centre[e], tangent[e], length[e], k0, operator, nq).reshape(nv, 12)
        elif operator == "N" and nq == 1:
            f = dyadic_green(rv, centre[e][None, :], k0) @ tangent[e]   # (nv, 3)
        else:
            f = segment_field(rv, centre[e], tangent[e], length[e], k0, operator, nq)
        f *= h ** 3 * length[e]
        f[~keep] = 0.0
        for k in range(q):
            out[k * nv:(k + 1) * nv, jj] = f[:, k]
    return out


def assemble_row(n, h, centre, tangent, length, freq_hz, row, q=3, mask_radius=0.0, mask_box=0.0) -> np.ndarray:
    """One row Z[row, :] (all m columns), row = k*n_v + v."""
    n1, n2, n3 = n
    nv = n1 * n2 * n3
    k, v = divmod(int(row), nv)
    rv = voxel_centres(n1, n2, n3, h)[v]
    if not voxel_mask(n1, n2, n3, h, mask_radius, mask_box)[v]:
        return np.zeros(length.shape[0], dtype=np.complex128)
    G = dyadic_green(rv[None, :], centre, wavenumber(freq_hz))   # (m, 3, 3)
    f = np.einsum("eab,eb->ea", G, tangent) * (h ** 3 * length)[:, None]
    return f[:, k].copy()
