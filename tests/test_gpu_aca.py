"""GPU ACA (plain, dense U then Tucker) and Algorithm 3 (Tucker-compressed U) against the
oracle's FP64 ACA on the same geometry: pivots, rank, norm estimate, approximation error and
the products on the resulting U V^H storage."""
import numpy as np
import pytest

from oracle import aca, greens, products, randomized, tucker
from paper_2103_06393_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import __graft_entry__  # noqa: E402

__graft_entry__.build()
from paper_2103_06393_gb300 import zbc  # noqa: E402


def _case(mask_radius=None, n=(12, 12, 10), m=64):
    w = inputs.scaled_workload("batching", n, m=m)
    g = w.grid
    if mask_radius is not None:
        g = inputs.Grid(g.n1, g.n2, g.n3, g.h, mask_radius)
    s = w.segments
    Z = greens.assemble_columns(g.shape, g.h, s.centre, s.tangent, s.length, w.freq_hz, np.arange(s.m),
                                mask_radius=g.mask_radius, mask_box=g.mask_box)
    return w, g, s, Z


def _uvh(h, g):
    tens, V = h.tensors()
    Zt = products.matvec(tens, g.shape, V.astype(np.complex128).conj().T)
    return Zt, tens, V


@pytest.mark.parametrize("tol", [1e-4, 1e-6])
def test_aca_dense_matches_oracle(tol):
    w, g, s, Z = _case()
    Uo, Vo, info = aca.aca_dense(lambda i: Z[i, :], lambda j: Z[:, j], Z.shape[0], Z.shape[1], tol, 64)
    h, st, piv = zbc.aca_compress(g, zbc.DeviceSegments(s), w.freq_hz, tol, 64, zbc.ACA_DENSE_U, tucker_tol=1e-10)
    assert st.rank == info["rank"]
    assert [tuple(p) for p in piv] == [tuple(p) for p in info["pivots"]]
    assert abs(st.s2 - info["s2"]) <= 1e-9 * info["s2"]
    Zt, _, _ = _uvh(h, g)
    ref = np.linalg.norm(Z - Uo @ Vo.conj().T) / np.linalg.norm(Z)
    err = np.linalg.norm(Z - Zt) / np.linalg.norm(Z)
    assert err <= ref + 1e-6 and err < 30 * tol


def test_aca_dense_masked_rows_and_products():
    w, g, s, Z = _case(mask_radius=0.008)
    assert np.all(Z[0, :] == 0)
    tol = 1e-5
    Uo, Vo, info = aca.aca_dense(lambda i: Z[i, :], lambda j: Z[:, j], Z.shape[0], Z.shape[1], tol, 64)
    h, st, piv = zbc.aca_compress(g, zbc.DeviceSegments(s), w.freq_hz, tol, 64, zbc.ACA_DENSE_U)
    assert st.row_restarts >= 1
    assert [tuple(p) for p in piv] == [tuple(p) for p in info["pivots"]]
    inf = h.info()
    assert inf.has_v == 1 and inf.m == s.m and inf.M == st.rank
    tens, V = h.tensors()
    X = inputs.cn01((s.m, 4), seed=1).astype(np.complex64)
    Y = zbc.colmajor(3 * g.nv, 4, torch.complex64)
    for prec in (zbc.FP32_SIMT, zbc.TF32X3, zbc.BF16X3):
        zbc.zbc_matvec(h, zbc.to_colmajor(X), Y, prec)
        torch.cuda.synchronize()
        Yo = products.matvec_aca(tens, V.astype(np.complex128), g.shape, X)
        e = np.linalg.norm(zbc.from_colmajor(Y) - Yo, axis=0) / np.linalg.norm(Yo, axis=0)
        assert e.max() < 1e-5
    Phi = inputs.cn01((3 * g.nv, 4), seed=2).astype(np.complex64)
    Psi = zbc.colmajor(s.m, 4, torch.complex64)
    zbc.zbc_rmatvec(h, zbc.to_colmajor(Phi), Psi, zbc.FP32_SIMT)
    torch.cuda.synchronize()
    Po = products.rmatvec_aca(tens, V.astype(np.complex128), g.shape, Phi)
    e = np.linalg.norm(zbc.from_colmajor(Psi) - Po, axis=0) / np.linalg.norm(Po, axis=0)
    assert e.max() < 1e-5


# Algorithm 3 on the GPU against the oracle.  The GPU stores U's tensors in
# complex64 and forms the residual column with Algorithm 1 in FP32, so its residuals differ from
# the oracle's (which stores the same complex64 roundings, store=np.complex64) by rounding: an
# entry whose value is a sum of terms of absolute size S moves by at most K_ERR * 2^-24 * S.
# K_ERR = 64 covers the complex64 storage of the four arrays an entry is evaluated from on each
# side (8 u), the FP32 sums of Algorithm 1 over the ranks and columns (tens of u) and the
# propagation of earlier columns' differences.  A pivot is decided when the gap between the
# largest and the second largest candidate exceeds twice that bound at both of them, and the stop
# test when |x||y| / (eps sqrt(s)) is further from 1 than four times the relative bound on |x|.
# Pivots must be bit-exact up to the first step that is not decided; after such a near-tie both
# runs are valid ACAs with different pivots, and r_c is accepted within R_WINDOW of the oracle's.
K_ERR = 64
U32 = 2.0 ** -24
R_WINDOW = 3


def _abs_columns(tens, shape):
    """Per stored column, the Tucker model evaluated on absolute values (|G| x1 |U1| x2 |U2| x3 |U3|):
    the absolute size of the terms that make up each entry."""
    return [np.concatenate([tucker.reconstruct(np.abs(G), [np.abs(U) for U in Us]).reshape(-1, order="F")
                            for G, Us in col]) for col in tens]


def _pick(vals, scale, excluded):
    """(argmax |vals| over the allowed entries, whether the storage-error margin decides it)."""
    a = np.abs(vals).astype(np.float64)
    if excluded:
        a[list(excluded)] = -np.inf
    order = np.argsort(-a, kind="stable")
    i1, i2 = int(order[0]), int(order[1])
    return i1, (a[i1] - a[i2]) > 2 * K_ERR * U32 * max(scale[i1], scale[i2])


def _check_alg3_against_oracle(w, g, s, Z, tol, h, st, piv, Ut, Vt, info, rank_tie=1e-5, min_decided=3):
    """Pivots bit-exact up to the first step whose argmax margin does not decide it against the
    complex64 storage error, r_c exact without a near-tie and within R_WINDOW after one; the
    approximation error tracks tol.  A Tucker rank of a new column's tensors decided within
    rank_tie of its threshold (relative: 1e-5 for the
    HOSVD; 1e-3 for the randomized Tucker, whose budget tol^2 ||A||^2 - e^2 carries the rounding
    of e^2) is a near-tie too: the steps after it are not compared."""
    assert st.row_restarts == 0
    tens = [[(G, Us) for G, Us, _ in col] for col in Ut]
    absU = _abs_columns(tens, g.shape)
    opiv = [tuple(p) for p in info["pivots"]]
    used_r, used_c = {0}, set()
    decided = 0          # leading pivots the storage-error margin decides
    tie = False
    why = ""
    for k, (i, j) in enumerate(opiv):
        tr = info["trace"][k]
        if k and min(min(t[2]["margin"]) for t in Ut[k - 1]) < rank_tie:
            tie, why = True, "rank"
            break
        rs = np.abs(Z[i, :]) + (np.array([absU[l][i] for l in range(k)]) @ np.abs(Vt[:, :k]).T if k else 0.0)
        jj, ok = _pick(tr["r"], rs, used_c)
        assert jj == j
        if not ok:
            tie, why = True, "column pivot"
            break
        assert tuple(piv[k]) == (i, j), (k, tuple(piv[k]), (i, j))
        decided = k + 1
        used_c.add(j)
        xs = np.abs(Z[:, j]) + (sum(absU[l] * abs(Vt[j, l]) for l in range(k)) if k else 0.0)
        relx = K_ERR * U32 * np.linalg.norm(xs) / tr["nx"]
        rho = tr["nx"] * tr["ny"] / (tol * np.sqrt(tr["s2"]))
        if abs(rho - 1.0) <= 4 * relx:
            tie, why = True, "stop test"
            break
        if k + 1 == len(opiv):
            break
        ii, ok = _pick(tr["x"], xs, used_r)
        assert ii == opiv[k + 1][0]
        if not ok:
            tie, why = True, "row pivot"
            break
        used_r.add(ii)
    print(f"tol {tol}: {decided} of {len(opiv)} pivots decided, near-tie: {tie} ({why}); "
          f"r_c GPU {st.rank} oracle {info['rank']}")
    assert decided >= min_decided
    if tie:
        assert [tuple(p) for p in piv[:decided]] == opiv[:decided]
        assert abs(st.rank - info["rank"]) <= R_WINDOW
    else:
        assert [tuple(p) for p in piv] == opiv and st.rank == info["rank"]
    Zt, _, _ = _uvh(h, g)
    err = np.linalg.norm(Z - Zt) / np.linalg.norm(Z)
    assert err < 30 * tol
    assert st.max_tucker_err <= 3 * tol * (1 + 1e-9)


@pytest.mark.parametrize("tol,n,m", [(1e-5, (12, 12, 10), 64), (1e-4, (14, 12, 8), 48), (1e-6, (10, 8, 8), 40)])
def test_algorithm3_pivots_exact_until_a_near_tie(tol, n, m):
    w, g, s, Z = _case(n=n, m=m)
    Ut, Vt, info = aca.aca_tucker(lambda i: Z[i, :], lambda j: Z[:, j], g.shape, 3, Z.shape[1], tol, 64,
                                  store=np.complex64, trace=True)
    h, st, piv = zbc.aca_compress(g, zbc.DeviceSegments(s), w.freq_hz, tol, 64, zbc.ACA_ALG3)
    _check_alg3_against_oracle(w, g, s, Z, tol, h, st, piv, Ut, Vt, info)


@pytest.mark.parametrize("width", [8, 12])
def test_algorithm3_with_randomized_tucker(width):
    """Algorithm 3 with U's tensors compressed by the fixed-width randomized Tucker (HOSVD fallback)
    against the oracle's Algorithm 3 with the oracle's randomized Tucker on the same sketches."""
    tol, n, m = 1e-5, (12, 12, 10), 64
    w, g, s, Z = _case(n=n, m=m)
    lmax = 16
    sk = inputs.mode_sketches(g, lmax, seed=21)
    skd = [zbc.to_colmajor(o) for o in sk]
    sk128 = [o.astype(np.complex128) for o in sk]
    wd = [min(width, ng) // 2 * 2 for ng in g.shape]
    fb = []

    def comp(A, t):
        G, Us, inf = randomized.randomized_tucker(A, wd, sk128, t)
        fb.append(inf["fallback"])
        return G, Us, inf

    Ut, Vt, info = aca.aca_tucker(lambda i: Z[i, :], lambda j: Z[:, j], g.shape, 3, Z.shape[1], tol, 64,
                                  store=np.complex64, trace=True, compress=comp)
    model = zbc.rank_model(skd, lmax, fixed_width=width)
    h, st, piv = zbc.aca_compress(g, zbc.DeviceSegments(s), w.freq_hz, tol, 64, zbc.ACA_ALG3,
                                  method=zbc.RANDOMIZED_FIXED, model=model)
    _check_alg3_against_oracle(w, g, s, Z, tol, h, st, piv, Ut, Vt, info, rank_tie=1e-3)
    if width == 8:
        assert st.tucker_fallbacks >= 1 and any(fb)   # too narrow for some of U's tensors


def test_aca_refuses_the_learned_method():
    w, g, s, Z = _case()
    lmax = 16
    skd = [zbc.to_colmajor(o) for o in inputs.mode_sketches(g, lmax, seed=21)]
    with pytest.raises(zbc.ZbcError) as e:
        zbc.aca_compress(g, zbc.DeviceSegments(s), w.freq_hz, 1e-5, 8, zbc.ACA_ALG3,
                         method=zbc.RANDOMIZED_LEARNED, model=zbc.rank_model(skd, lmax, fixed_width=8))
    assert e.value.status == zbc.ZBC_EINVAL
