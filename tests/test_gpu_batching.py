"""Batching and scheduling of the products: the autotuner (zbc_tune + ZBC_AUTO) and CUDA-graph
capture of mixed right-hand-side batches, against the FP64 oracle and the eager calls."""
import math

import numpy as np
import pytest

from oracle import greens, products, tucker
from paper_2103_06393_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import __graft_entry__  # noqa: E402

__graft_entry__.build()
from paper_2103_06393_gb300 import zbc  # noqa: E402

RTOL = 1e-5


def _handle(n=(40, 24, 20), m=20, tol=1e-6):
    w = inputs.scaled_workload("precision", n, m=m)
    g, s = w.grid, w.segments
    Z = greens.assemble_columns(g.shape, g.h, s.centre, s.tangent, s.length, w.freq_hz, np.arange(s.m))
    tens = tucker.compress_columns(Z, g.shape, 3, tol)
    tens = [[(t[0].astype(np.complex64).astype(np.complex128),
              [U.astype(np.complex64).astype(np.complex128) for U in t[1]]) for t in tj] for tj in tens]
    return zbc.zbc_create_from_host(g, 3, tens), tens, g


def _rel(a, b):
    return float(np.max(np.linalg.norm(a - b, axis=0) / np.linalg.norm(b, axis=0)))


@pytest.mark.parametrize("p", [1, 5, 16, 40])
def test_tune_then_auto_matches_oracle(p):
    h, tens, g = _handle()
    t = zbc.zbc_tune(h, p)
    assert set(t) == set(zbc.TUNE_VARIANTS)
    assert all(math.isfinite(t[k]) and t[k] > 0 for k in ("fwd_simt6", "fwd_simt9", "adj_simt6", "adj_simt9"))
    X = inputs.cn01((len(tens), p), seed=3).astype(np.complex64)
    Phi = inputs.cn01((3 * g.nv, p), seed=4).astype(np.complex64)
    Y = zbc.colmajor(3 * g.nv, p, torch.complex64)
    Psi = zbc.colmajor(len(tens), p, torch.complex64)
    zbc.zbc_matvec(h, zbc.to_colmajor(X), Y, zbc.AUTO)
    zbc.zbc_rmatvec(h, zbc.to_colmajor(Phi), Psi, zbc.AUTO)
    zbc.zbc_product_status(h)
    assert _rel(zbc.from_colmajor(Y), products.matvec(tens, g.shape, X)) < RTOL
    assert _rel(zbc.from_colmajor(Psi), products.rmatvec(tens, g.shape, Phi)) < RTOL


def test_tune_releases_operands_of_unselected_forms():
    """zbc_tune frees the per-handle operands of the forms it did not select; a later call of such a
    form builds them again and gives the same bits as before."""
    h, tens, g = _handle()
    p = 5
    X = zbc.to_colmajor(inputs.cn01((len(tens), p), seed=7).astype(np.complex64))
    outs = {}
    for code in (zbc.TC_MODE1, zbc.TC_DC, zbc.TC2):
        Y = zbc.colmajor(3 * g.nv, p, torch.complex64)
        zbc.zbc_matvec(h, X, Y, code)
        outs[code] = Y.clone()
    Phi = zbc.to_colmajor(inputs.cn01((3 * g.nv, p), seed=8).astype(np.complex64))
    Psi = zbc.colmajor(len(tens), p, torch.complex64)
    zbc.zbc_rmatvec(h, Phi, Psi, zbc.TC_MODE1)
    zbc.zbc_product_status(h)
    before = h.device_bytes()["caches"]
    t = zbc.zbc_tune(h, p)
    fwd = min((k for k in t if k.startswith("fwd_")), key=lambda k: t[k])
    after = h.device_bytes()["caches"]
    # at most one of the three forward forms' operands stays
    assert after < before, (before, after, fwd)
    for code in (zbc.TC_MODE1, zbc.TC_DC, zbc.TC2):
        Y = zbc.colmajor(3 * g.nv, p, torch.complex64)
        zbc.zbc_matvec(h, X, Y, code)
        zbc.zbc_product_status(h)
        assert torch.equal(Y, outs[code]), code
    assert h.device_bytes()["caches"] >= before


def test_adjoint_rejects_tensor_core_forms():
    h, tens, g = _handle(n=(8, 8, 8), m=3)
    Phi = zbc.colmajor(3 * g.nv, 2, torch.complex64)
    Psi = zbc.colmajor(len(tens), 2, torch.complex64)
    with pytest.raises(zbc.ZbcError) as e:
        zbc.zbc_rmatvec(h, Phi, Psi, zbc.BF16X3)
    assert e.value.status == zbc.ZBC_EINVAL


def test_graph_capture_of_mixed_batches():
    # one CUDA graph holding forward and adjoint products for a mix of right-hand-side counts;
    # its replay must reproduce the eager calls bit for bit (same kernels, same order of sums)
    h, tens, g = _handle()
    ps = [16, 1, 3, 8, 40]
    Xs = [zbc.to_colmajor(inputs.cn01((len(tens), p), seed=10 + p).astype(np.complex64)) for p in ps]
    Phis = [zbc.to_colmajor(inputs.cn01((3 * g.nv, p), seed=20 + p).astype(np.complex64)) for p in ps]
    Ys = [zbc.colmajor(3 * g.nv, p, torch.complex64) for p in ps]
    Psis = [zbc.colmajor(len(tens), p, torch.complex64) for p in ps]
    for p in ps:
        zbc.zbc_tune(h, p)

    def run_all():
        for X, Phi, Y, Psi in zip(Xs, Phis, Ys, Psis):
            zbc.zbc_matvec(h, X, Y, zbc.AUTO)
            zbc.zbc_rmatvec(h, Phi, Psi, zbc.AUTO)

    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        run_all()                       # eager, on the stream that will be captured
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    eager = [(zbc.from_colmajor(Y), zbc.from_colmajor(Psi)) for Y, Psi in zip(Ys, Psis)]
    for Y, Psi in zip(Ys, Psis):
        Y.fill_(float("nan"))
        Psi.fill_(float("nan"))
    graph = torch.cuda.CUDAGraph()
    l0 = zbc.kernel_launches()
    with torch.cuda.graph(graph):
        run_all()
    launches = zbc.kernel_launches() - l0
    assert launches >= 2 * len(ps)
    graph.replay()
    torch.cuda.synchronize()
    zbc.zbc_product_status(h)
    for (Ye, Pe), Y, Psi in zip(eager, Ys, Psis):
        assert np.array_equal(zbc.from_colmajor(Y), Ye)
        assert np.array_equal(zbc.from_colmajor(Psi), Pe)
    # and the replay is right, not only repeatable
    X0, Phi0 = zbc.from_colmajor(Xs[0]), zbc.from_colmajor(Phis[0])
    assert _rel(eager[0][0], products.matvec(tens, g.shape, X0)) < RTOL
    assert _rel(eager[0][1], products.rmatvec(tens, g.shape, Phi0)) < RTOL
