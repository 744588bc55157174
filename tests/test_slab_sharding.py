"""Voxel-slab sharding (paper_2103_06393_gb300/shard.py) simulated on the host with the FP64 oracle:
each rank's share of the tensors gives Y's rows of its slab (Algorithm 1 needs no exchange) and a
partial adjoint whose sum over the ranks is Psi (Algorithm 2: one all_reduce).  In one process for
several world sizes and uneven splits, then across two gloo ranks that really exchange the
partials."""
import os
import socket

import numpy as np
import pytest

from oracle import greens, products, tucker
from paper_2103_06393_gb300 import inputs, shard

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

SHAPE = (12, 10, 7)     # n3 = 7: uneven slabs for 2 and 3 ranks


def _problem(seed=0):
    w = inputs.scaled_workload("precision", SHAPE, m=5)
    g, s = w.grid, w.segments
    Z = greens.assemble_columns(g.shape, g.h, s.centre, s.tangent, s.length, w.freq_hz, np.arange(s.m))
    tens = tucker.compress_columns(Z, g.shape, 3, 1e-6)
    X = inputs.cn01((s.m, 3), seed=seed + 1)
    Phi = inputs.cn01((3 * g.nv, 3), seed=seed + 2)
    return tens, X, Phi


def test_slab_ranges_cover_the_grid():
    for n3, world in ((7, 2), (7, 3), (96, 8), (5, 5), (3, 4)):
        spans = [shard.slab_range(n3, r, world) for r in range(world)]
        assert spans[0][0] == 0 and spans[-1][1] == n3
        assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
        sizes = [e - s for s, e in spans]
        assert max(sizes) - min(sizes) <= 1
        rows = np.concatenate([shard.slab_rows((4, 3, n3), 3, r, world) for r in range(world)])
        assert np.array_equal(np.sort(rows), np.arange(3 * 4 * 3 * n3))
    with pytest.raises(ValueError):
        shard.slab_range(7, 2, 2)


@pytest.mark.parametrize("world", [1, 2, 3, 7])
def test_slabs_reproduce_both_products(world):
    tens, X, Phi = _problem()
    n1, n2, n3 = SHAPE
    Y = products.matvec(tens, SHAPE, X)
    Psi = products.rmatvec(tens, SHAPE, Phi)
    Yr = np.zeros_like(Y)
    Psi_sum = np.zeros_like(Psi)
    for r in range(world):
        s, e = shard.slab_range(n3, r, world)
        sub = shard.slab_tensors(tens, n3, r, world)
        rows = shard.slab_rows(SHAPE, 3, r, world)
        Yr[rows] = products.matvec(sub, (n1, n2, e - s), X)
        Psi_sum += products.rmatvec(sub, (n1, n2, e - s), Phi[rows])
    assert np.allclose(Yr, Y, rtol=0, atol=1e-13 * np.abs(Y).max())
    assert np.allclose(Psi_sum, Psi, rtol=0, atol=1e-13 * np.abs(Psi).max())


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    tens, X, Phi = _problem()
    n1, n2, n3 = SHAPE
    s, e = shard.slab_range(n3, rank, world)
    sub = shard.slab_tensors(tens, n3, rank, world)
    rows = shard.slab_rows(SHAPE, 3, rank, world)
    # the adjoint's one exchange: all_reduce(sum) of the m x p partials (real and imaginary parts)
    part = products.rmatvec(sub, (n1, n2, e - s), Phi[rows])
    t = torch.from_numpy(np.stack([part.real, part.imag]))
    dist.all_reduce(t)
    # Y stays distributed; gather the slabs only to check them
    slabs = [None] * world
    dist.all_gather_object(slabs, (rows, products.matvec(sub, (n1, n2, e - s), X)))
    if rank == 0:
        Y = np.zeros((3 * n1 * n2 * n3, X.shape[1]), dtype=np.complex128)
        for rr, yr in slabs:
            Y[rr] = yr
        out.put((t[0].numpy() + 1j * t[1].numpy(), Y))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_exchange_the_adjoint_partials():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    Psi_d, Y_d = q.get(timeout=180)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    tens, X, Phi = _problem()
    Y = products.matvec(tens, SHAPE, X)
    Psi = products.rmatvec(tens, SHAPE, Phi)
    assert np.allclose(Psi_d, Psi, rtol=0, atol=1e-13 * np.abs(Psi).max())
    assert np.allclose(Y_d, Y, rtol=0, atol=1e-13 * np.abs(Y).max())
