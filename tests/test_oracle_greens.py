"""Pins of the oracle's dyadic Green's function and column assembly (Eq. n6, Eq. nNt, Sec. III.A).

Each check compares against something other than the oracle's own closed form:
finite differences of the scalar kernel, textbook on-axis values, symmetry,
reciprocity and the far-field limit.
"""
import numpy as np
import pytest

from oracle import greens
from paper_2103_06393_gb300 import inputs

K0 = greens.wavenumber(298.2e6)


def test_wavenumber_value():
    # k0 = 2 pi f / c at 298.2 MHz
    assert abs(K0 - 6.249807) < 1e-5
    assert abs(2 * np.pi / K0 - 1.005340) < 1e-5


def _fd_dyadic(r, k0, step=1e-4):
    """(I + grad grad / k0^2) g by central second differences of the scalar kernel only."""
    def g(x):
        return greens.scalar_green(np.linalg.norm(x), k0)
    H = np.zeros((3, 3), dtype=complex)
    e = np.eye(3) * step
    for a in range(3):
        for b in range(3):
            H[a, b] = (g(r + e[a] + e[b]) - g(r + e[a] - e[b]) - g(r - e[a] + e[b]) + g(r - e[a] - e[b])) / (4 * step * step)
    return g(r) * np.eye(3) + H / k0 ** 2


@pytest.mark.parametrize("r", [np.array([0.05, -0.03, 0.02]), np.array([0.2, 0.1, -0.3]), np.array([0.0, 0.0, 0.4])])
def test_dyadic_matches_finite_differences(r):
    G = greens.dyadic_green(r, np.zeros(3), K0)
    Gfd = _fd_dyadic(r, K0, step=1e-4 * np.linalg.norm(r))
    assert np.max(np.abs(G - Gfd)) / np.max(np.abs(G)) < 1e-6


def test_on_axis_closed_form():
    R = 0.3
    G = greens.dyadic_green(np.array([0, 0, R]), np.zeros(3), K0)
    x = K0 * R
    g = np.exp(-1j * x) / (4 * np.pi * R)
    assert np.isclose(G[2, 2], g * (2j / x + 2 / x ** 2), rtol=1e-13)
    assert np.isclose(G[0, 0], g * (1 - 1j / x - 1 / x ** 2), rtol=1e-13)
    assert np.isclose(G[1, 1], G[0, 0], rtol=1e-13)
    off = [G[0, 1], G[0, 2], G[1, 2], G[1, 0], G[2, 0], G[2, 1]]
    assert max(abs(v) for v in off) < 1e-15 * abs(G[0, 0])


def test_symmetry_and_reciprocity():
    rng = np.random.default_rng(3)
    a, b = rng.normal(size=3) * 0.1, rng.normal(size=3) * 0.1 + 0.2
    G1 = greens.dyadic_green(a, b, K0)
    G2 = greens.dyadic_green(b, a, K0)
    assert np.allclose(G1, G1.T, rtol=1e-14, atol=0)
    assert np.allclose(G1, G2, rtol=1e-14, atol=0)


def test_far_field_is_transverse():
    # for k0 R >> 1, G -> g (I - Rhat Rhat^T)
    r = np.array([300.0, 400.0, 0.0])
    G = greens.dyadic_green(r, np.zeros(3), K0)
    R = np.linalg.norm(r)
    rh = r / R
    g = greens.scalar_green(R, K0)
    approx = g * (np.eye(3) - np.outer(rh, rh))
    assert np.max(np.abs(G - approx)) / abs(g) < 3.0 / (K0 * R)


def test_voxel_ordering_and_centres():
    c = greens.voxel_centres(3, 4, 5, 0.01)
    v = 2 + 3 * (1 + 4 * 3)     # i1=2, i2=1, i3=3
    assert np.allclose(c[v], [(2 - 1) * 0.01, (1 - 1.5) * 0.01, (3 - 2) * 0.01])


def test_assembly_entry_by_hand_and_row_column_consistency():
    w = inputs.scaled_workload("tiny", (5, 6, 7), m=8)
    g, s = w.grid, w.segments
    Z = greens.assemble_columns(g.shape, g.h, s.centre, s.tangent, s.length, w.freq_hz, np.arange(s.m))
    nv = g.nv
    # one entry from the on-axis/general closed form written per component
    v, e, k = 17, 3, 1
    rv = greens.voxel_centres(*g.shape, g.h)[v]
    R = rv - s.centre[e]
    Rn = np.linalg.norm(R)
    rh = R / Rn
    x = K0 * Rn
    gg = np.exp(-1j * x) / (4 * np.pi * Rn)
    val = gg * ((1 - 1j / x - 1 / x ** 2) * s.tangent[e][k]
                + (-1 + 3j / x + 3 / x ** 2) * rh[k] * (rh @ s.tangent[e]))
    assert np.isclose(Z[k * nv + v, e], g.h ** 3 * s.length[e] * val, rtol=1e-13)
    row = greens.assemble_row(g.shape, g.h, s.centre, s.tangent, s.length, w.freq_hz, k * nv + v)
    assert np.allclose(row, Z[k * nv + v, :], rtol=1e-14, atol=0)


def test_assembly_linear_in_tangent():
    g = inputs.Grid(4, 5, 6, 0.01)
    c = np.array([[0.2, 0.05, 0.0]])
    t1, t2 = np.array([[1.0, 0, 0]]), np.array([[0, 0.6, 0.8]])
    ln = np.array([0.01])
    z1 = greens.assemble_columns(g.shape, g.h, c, t1, ln, 3e8, [0])
    z2 = greens.assemble_columns(g.shape, g.h, c, t2, ln, 3e8, [0])
    z12 = greens.assemble_columns(g.shape, g.h, c, 0.3 * t1 + 0.7 * t2, ln, 3e8, [0])
    assert np.allclose(z12, 0.3 * z1 + 0.7 * z2, rtol=1e-13, atol=0)


def test_mask_zeroes_outer_voxels():
    g = inputs.Grid(10, 10, 4, 0.01, mask_radius=0.04)
    c = np.array([[0.3, 0.0, 0.0]])
    t = np.array([[0, 1.0, 0]])
    z = greens.assemble_columns(g.shape, g.h, c, t, np.array([0.01]), 3e8, [0], mask_radius=g.mask_radius)
    keep = greens.voxel_mask(*g.shape, g.h, g.mask_radius)
    assert keep.sum() < g.nv
    for k in range(3):
        seg = z[k * g.nv:(k + 1) * g.nv, 0]
        assert np.all(seg[~keep] == 0) and np.all(seg[keep] != 0)


def test_box_mask_is_separable_and_keeps_tucker_ranks():
    """The box mask drops exactly the voxels with max(|x|, |y|) > mask_box (a loop over voxels),
    and, being a product of per-axis indicators, it leaves the multilinear ranks of a column's
    tensor those of the unmasked field on the kept box, where a radial mask raises them."""
    from oracle import tucker
    g = inputs.Grid(16, 14, 6, 0.01, mask_box=0.045)
    keep = greens.voxel_mask(*g.shape, g.h, 0.0, g.mask_box)
    for v in range(g.nv):
        i1, i2 = v % g.n1, (v // g.n1) % g.n2
        x, y = (i1 - (g.n1 - 1) / 2.0) * g.h, (i2 - (g.n2 - 1) / 2.0) * g.h
        assert keep[v] == (abs(x) <= g.mask_box and abs(y) <= g.mask_box)
    assert 0 < keep.sum() < g.nv
    c = np.array([[0.15, 0.02, 0.01]])
    t = np.array([[0.0, 0.6, 0.8]])
    z = greens.assemble_columns(g.shape, g.h, c, t, np.array([0.01]), 3e8, [0], mask_box=g.mask_box)
    full = greens.assemble_columns(g.shape, g.h, c, t, np.array([0.01]), 3e8, [0])
    assert np.array_equal(z[np.tile(keep, 3), 0], full[np.tile(keep, 3), 0])
    assert np.all(z[~np.tile(keep, 3), 0] == 0)
    i1 = np.abs((np.arange(g.n1) - (g.n1 - 1) / 2.0) * g.h) <= g.mask_box
    i2 = np.abs((np.arange(g.n2) - (g.n2 - 1) / 2.0) * g.h) <= g.mask_box
    for k in range(3):
        A = tucker.fold(z[k * g.nv:(k + 1) * g.nv, 0], g.shape)
        B = tucker.fold(full[k * g.nv:(k + 1) * g.nv, 0], g.shape)[np.ix_(i1, i2, np.arange(g.n3))]
        _, _, ia = tucker.hosvd(A, 1e-6)
        _, _, ib = tucker.hosvd(B, 1e-6)
        assert tuple(ia["ranks"]) == tuple(ib["ranks"])
    zr = greens.assemble_columns(g.shape, g.h, c, t, np.array([0.01]), 3e8, [0], mask_radius=g.mask_box)
    _, _, ir = tucker.hosvd(tucker.fold(zr[:g.nv, 0], g.shape), 1e-6)
    _, _, ib = tucker.hosvd(tucker.fold(z[:g.nv, 0], g.shape), 1e-6)
    assert ir["ranks"][0] > ib["ranks"][0]


# ------------------------------------------------------------------------------------------------
# the K operator (Eq. nKt: curl of the single-layer potential) and the segment quadrature
# ------------------------------------------------------------------------------------------------

def _fd_grad(r, k0, step):
    """grad g by central first differences of the scalar kernel only."""
    def g(x):
        return greens.scalar_green(np.linalg.norm(x), k0)
    e = np.eye(3) * step
    return np.array([(g(r + e[a]) - g(r - e[a])) / (2 * step) for a in range(3)])


@pytest.mark.parametrize("r", [np.array([0.05, -0.03, 0.02]), np.array([0.2, 0.1, -0.3]), np.array([0.0, 0.0, 0.4])])
def test_curl_green_matches_finite_differences(r):
    t = np.array([0.3, -0.8, 0.52])
    t /= np.linalg.norm(t)
    K = greens.curl_green(r, np.zeros(3), t, K0)
    Kfd = np.cross(_fd_grad(r, K0, 1e-5 * np.linalg.norm(r)), t)
    assert np.max(np.abs(K - Kfd)) / np.max(np.abs(K)) < 1e-8


def test_curl_green_orthogonality_and_magnitude():
    # grad g x t is orthogonal to t and to Rhat; |grad g x t| = |g| |i k0 + 1/R| |Rhat x t|;
    # it vanishes for t along Rhat and changes sign with the source-observer swap
    rng = np.random.default_rng(5)
    for _ in range(5):
        r, c = rng.normal(size=3) * 0.2, rng.normal(size=3) * 0.05
        t = rng.normal(size=3)
        t /= np.linalg.norm(t)
        K = greens.curl_green(r, c, t, K0)
        R = r - c
        Rn = np.linalg.norm(R)
        assert abs(np.dot(K, t)) < 1e-13 * np.linalg.norm(K)
        assert abs(np.dot(K, R / Rn)) < 1e-13 * np.linalg.norm(K)
        mag = abs(greens.scalar_green(Rn, K0)) * abs(1j * K0 + 1 / Rn) * np.linalg.norm(np.cross(R / Rn, t))
        assert np.isclose(np.linalg.norm(K), mag, rtol=1e-13)
        assert np.allclose(greens.curl_green(c, r, t, K0), -K, rtol=1e-13, atol=0)
        assert np.max(np.abs(greens.curl_green(r, c, R / Rn, K0))) < 1e-15 * np.max(np.abs(K)) + 1e-300


def test_curl_of_k_field_is_k0_squared_times_n_field():
    # curl(curl(g t)) = curl curl (g t) = k0^2 (I + grad grad / k0^2) g t away from the source:
    # a finite-difference curl of the K kernel gives k0^2 times the N kernel (each operator is
    # pinned independently above; this ties the two together)
    t = np.array([0.1, 0.7, -0.2])
    t /= np.linalg.norm(t)
    r = np.array([0.12, -0.05, 0.2])
    step = 1e-5

    def Kf(x):
        return greens.curl_green(x, np.zeros(3), t, K0)
    e = np.eye(3) * step
    J = np.array([(Kf(r + e[a]) - Kf(r - e[a])) / (2 * step) for a in range(3)])   # J[a, b] = d_a K_b
    curl = np.array([J[1, 2] - J[2, 1], J[2, 0] - J[0, 2], J[0, 1] - J[1, 0]])
    N = greens.dyadic_green(r, np.zeros(3), K0) @ t
    assert np.max(np.abs(curl - K0 ** 2 * N)) / np.max(np.abs(K0 ** 2 * N)) < 1e-7


@pytest.mark.parametrize("operator", ["N", "K"])
def test_segment_quadrature(operator):
    # one Gauss-Legendre point is the point-matched form; nq points agree with a fine midpoint rule
    # along the segment (brute force), and 8 points already to 1e-12 for a voxel 20 lengths away
    rng = np.random.default_rng(9)
    c = np.array([0.1, 0.0, 0.02])
    t = rng.normal(size=3)
    t /= np.linalg.norm(t)
    L = 0.015
    rv = np.array([[0.4, 0.2, -0.1], [0.12, 0.01, 0.03]])
    one = greens.segment_field(rv, c, t, L, K0, operator, 1)
    if operator == "N":
        point = greens.dyadic_green(rv, c[None, :], K0) @ t
    else:
        point = greens.curl_green(rv, c[None, :], t, K0)
    assert np.allclose(one, point, rtol=1e-15, atol=0)
    nmid = 4000
    xs = (np.arange(nmid) + 0.5) / nmid * 2 - 1
    brute = np.zeros_like(one)
    for x in xs:
        p = c + 0.5 * x * L * t
        if operator == "N":
            brute += (greens.dyadic_green(rv, p[None, :], K0) @ t) / nmid
        else:
            brute += greens.curl_green(rv, p[None, :], t, K0) / nmid
    q8 = greens.segment_field(rv, c, t, L, K0, operator, 8)
    assert np.max(np.abs(q8 - brute)) / np.max(np.abs(brute)) < 1e-6          # the midpoint rule's own error
    q16 = greens.segment_field(rv[:1], c, t, L, K0, operator, 16)
    assert np.max(np.abs(q8[:1] - q16)) / np.max(np.abs(q16)) < 1e-12


def test_k_assembly_columns():
    # the K columns: entry by the closed form, orthogonal to the segment's tangent at every voxel
    w = inputs.scaled_workload("tiny", (6, 5, 4), m=3)
    g, s = w.grid, w.segments
    Z = greens.assemble_columns(g.shape, g.h, s.centre, s.tangent, s.length, w.freq_hz, np.arange(3), operator="K")
    nv = g.nv
    rv = greens.voxel_centres(*g.shape, g.h)
    for e in range(3):
        F = np.stack([Z[k * nv:(k + 1) * nv, e] for k in range(3)], axis=1)
        assert np.max(np.abs(F @ s.tangent[e])) < 1e-13 * np.max(np.abs(F))
        v = 17
        ref = g.h ** 3 * s.length[e] * greens.curl_green(rv[v], s.centre[e], s.tangent[e], greens.wavenumber(w.freq_hz))
        assert np.allclose(F[v], ref, rtol=1e-14, atol=0)


# ------------------------------------------------------------------------------------------------
# piecewise-linear voxel basis (q = 12)
# ------------------------------------------------------------------------------------------------

_C, _T, _L = np.array([0.15, 0.0, 0.0]), np.array([0.0, 1.0, 0.0]), 0.015
_RV = np.array([[0.0, 0.01, 0.0], [0.1, 0.02, -0.01], [0.05, -0.05, 0.03]])
_H = 0.005


@pytest.mark.parametrize("op", ["N", "K"])
def test_pwl_rule_against_a_high_order_rule(op):
    # the 2 x 2 x 2 Gauss rule against an 8 x 8 x 8 one (library nodes): the constant rows to the
    # rule's accuracy, the linear rows to its (lower) accuracy for the linear-times-field integrand
    a = greens.pwl_field(_RV, _H, _C, _T, _L, K0, op, 2, nvq=2)
    b = greens.pwl_field(_RV, _H, _C, _T, _L, K0, op, 2, nvq=8)
    assert np.max(np.abs(a[:, 0] - b[:, 0])) / np.max(np.abs(b[:, 0])) < 1e-4
    for l in range(1, 4):
        assert np.max(np.abs(a[:, l] - b[:, l])) / np.max(np.abs(b[:, l])) < 5e-3


@pytest.mark.parametrize("op", ["N", "K"])
def test_pwl_moments(op):
    # mean of f over the voxel = f(r_c) (1 - k0^2 h^2 / 24) + O(h^4) (the Laplacian of a Helmholtz
    # field is -k0^2 f); the linear rows are the first moments (h / 12) d_x f, (h / 12) d_y f,
    # (h / 12) d_z f + O(h^3), checked by central differences of the point-matched field
    a = greens.pwl_field(_RV, _H, _C, _T, _L, K0, op, 2)
    f0 = greens.segment_field(_RV, _C, _T, _L, K0, op, 2)
    assert np.max(np.abs(a[:, 0] - f0 * (1 - K0 ** 2 * _H ** 2 / 24))) / np.max(np.abs(f0)) < 1e-4
    e = 1e-6
    for ax in range(3):
        d = np.zeros(3)
        d[ax] = e
        df = (greens.segment_field(_RV + d, _C, _T, _L, K0, op, 2) - greens.segment_field(_RV - d, _C, _T, _L, K0, op, 2)) / (2 * e)
        assert np.max(np.abs(a[:, ax + 1] - _H / 12 * df)) / np.max(np.abs(_H / 12 * df)) < 1e-2


def test_pwl_assembly_layout():
    # q = 12 columns: row block b = 3 l + k holds basis l, component k of pwl_field, times h^3 len
    w = inputs.scaled_workload("tiny", (5, 4, 3), m=2)
    g, s = w.grid, w.segments
    Z = greens.assemble_columns(g.shape, g.h, s.centre, s.tangent, s.length, w.freq_hz, np.arange(2), q=12,
                                operator="K", nq=2)
    assert Z.shape == (12 * g.nv, 2)
    rv = greens.voxel_centres(*g.shape, g.h)
    F = greens.pwl_field(rv, g.h, s.centre[1], s.tangent[1], s.length[1], greens.wavenumber(w.freq_hz), "K", 2)
    for l in range(4):
        for k in range(3):
            b = 3 * l + k
            assert np.allclose(Z[b * g.nv:(b + 1) * g.nv, 1], g.h ** 3 * s.length[1] * F[:, l, k], rtol=1e-14, atol=0)
