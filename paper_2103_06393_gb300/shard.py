"""Voxel-slab sharding of the compressed coupling matrix across ranks (one GPU per rank).

Rank r of R owns the voxels with i3 in [s_r, e_r), s_r = floor(r n3 / R).  Its share of every
Tucker tensor keeps the factors U1, U2 whole and only rows s_r .. e_r - 1 of U3, re-orthonormalised
(U3[s:e] = Q R, Q with min(e - s, r3) columns, and R folded into the core: G x3 R), so it is the
coupling matrix restricted to the slab's rows (the rows of each component block whose
voxel index v = i1 + n1 (i2 + n2 i3) falls in the slab, contiguous because i3 varies slowest).
Algorithm 1 is then slab-local: rank r computes Y's rows of its slab and nothing is exchanged.
Algorithm 2 sums over voxels, so each rank computes the partial Psi_r = Z_r^H Phi_r from its
slab of Phi and one all_reduce (sum) of the m x p partials gives Psi.  The cores, U1, U2, X and
V are replicated; only U3 and the slabs of Y and Phi are split.
"""
from __future__ import annotations

import numpy as np


def slab_range(n3: int, rank: int, world: int) -> tuple[int, int]:
    """[s, e) of the i3 planes owned by `rank` of `world` (contiguous, sizes differ by at most 1)."""
    if not 0 <= rank < world:
        raise ValueError(f"rank {rank} not in [0, {world})")
    return rank * n3 // world, (rank + 1) * n3 // world


def slab_rows(n, q: int, rank: int, world: int) -> np.ndarray:
    """Row indices, in the (q n_v)-row layout of Y and Phi, of the slab's rows in the order the
    slab's own (q n1 n2 (e - s))-row layout uses: component block by block."""
    n1, n2, n3 = n
    s, e = slab_range(n3, rank, world)
    nv, plane = n1 * n2 * n3, n1 * n2
    return np.concatenate([k * nv + np.arange(s * plane, e * plane) for k in range(q)])


def _slab_tensor(G, Us, s, e):
    """(G x3 R, [U1, U2, Q]) with U3[s:e] = Q R (reduced QR): the same entries on planes s .. e-1,
    with a mode-3 rank of at most e - s (a handle needs every rank within its mode size)."""
    U3 = np.asarray(Us[2][s:e], dtype=np.complex128)
    Q, R = np.linalg.qr(U3)                                   # (e-s) x r', r' x r3
    Gs = np.tensordot(np.asarray(G, dtype=np.complex128), R, axes=([2], [1]))   # r1 x r2 x r'
    return (Gs, [Us[0], Us[1], Q])


def slab_tensors(tensors, n3: int, rank: int, world: int):
    """The slab's share of every tensor in the oracle's / export format (a list over columns of a
    list over components of (G, [U1, U2, U3], ...)): U3 cut to the slab's rows and
    re-orthonormalised, its triangular factor folded into the core; U1, U2 shared."""
    s, e = slab_range(n3, rank, world)
    return [[_slab_tensor(t[0], t[1], s, e) for t in tj] for tj in tensors]


def slab_handle(h, grid, rank: int, world: int):
    """A handle over rank `rank`'s slab of handle h (a copy in device memory: cores, U1, U2, V
    whole, U3 cut).  Its zbc_matvec gives Y's rows slab_rows(...) and its zbc_rmatvec the partial
    Psi_r to sum over the ranks."""
    from . import inputs, zbc
    s, e = slab_range(grid.n3, rank, world)
    if e - s < 2:
        raise ValueError(f"rank {rank} of {world} would own {e - s} of the {grid.n3} i3 planes; a handle "
                         "needs at least 2 (use at most n3 // 2 ranks)")
    tens, V = h.tensors()
    sub = inputs.Grid(grid.n1, grid.n2, e - s, grid.h)
    return zbc.zbc_create_from_host(sub, h.info().q, slab_tensors(tens, grid.n3, rank, world), V)
