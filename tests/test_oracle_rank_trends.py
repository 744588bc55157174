"""Tucker-rank studies of Sec. IV.A (Figs. 4-6) as regression tests of the compressor, scaled
down to grids the FP64 oracle compresses in seconds, with the K operator of Eq. nKt (the
paper's Z_bc) and 4- or 8-point Gauss-Legendre rules along the segments.

  Rank vs distance (Sec. IV.A.1, Fig. 4): a loop of radius 0.5 m in the plane y = d beside a 1 m
    cube; the maximum Tucker rank and the compressed storage fall as d grows.
  Rank vs frequency (Sec. IV.A.2, Fig. 5): voxels of lambda / 20; rank and storage grow with the
    frequency.
  Rank vs surface mesh (Sec. IV.A.3, Fig. 6): an equilateral triangle (centroid (0, 0.55, 0),
    a vertex at (0, 0.55, 0.5)) whose sides are cut into finer segments; the rank falls.
The paper gives the trends (its exact values come from RWG meshes and 5D integrals, not
reproduced); the values asserted here are this oracle's on these synthetic inputs."""
import numpy as np

from oracle import greens, tucker
from paper_2103_06393_gb300 import inputs

F7T = 298.06e6


def _study(n, h, segs, freq, nq, tol):
    Z = greens.assemble_columns(n, h, segs.centre, segs.tangent, segs.length, freq, np.arange(segs.m),
                                operator="K", nq=nq)
    tens = tucker.compress_columns(Z, n, 3, tol)
    max_rank = max(max(U.shape[1] for U in t[1]) for tj in tens for t in tj)
    storage = sum(int(np.prod(t[0].shape)) + sum(U.size for U in t[1]) for tj in tens for t in tj)
    return max_rank, storage


def test_rank_falls_with_distance():
    n, h = (16, 16, 16), 1.0 / 16
    res = [_study(n, h, inputs.loop_coil_y(0.5, d, 24), F7T, 4, 1e-8) for d in (0.55, 0.7, 0.85, 1.0)]
    ranks, store = [r for r, _ in res], [s for _, s in res]
    assert all(a >= b for a, b in zip(ranks, ranks[1:])) and ranks[-1] < ranks[0], ranks
    assert all(a > b for a, b in zip(store, store[1:])), store
    assert ranks == [16, 15, 13, 11]


def test_rank_grows_with_frequency():
    res = []
    for f in (300e6, 600e6, 900e6):
        h = 299_792_458.0 / f / 20
        nn = int(round(0.5 / h)) + 1
        res.append(_study((nn, nn, nn), h, inputs.loop_coil_y(0.25, 0.3, 16), f, 4, 1e-8))
    ranks, store = [r for r, _ in res], [s for _, s in res]
    assert all(a < b for a, b in zip(ranks, ranks[1:])), ranks
    assert all(a < b for a, b in zip(store, store[1:])), store
    assert ranks == [11, 20, 24]


def test_rank_falls_with_surface_mesh_refinement():
    n, h = (28, 28, 28), 1.0 / 28
    ranks = [_study(n, h, inputs.triangle_coil_y(0.5, 0.55, k), F7T, 8, 1e-6)[0] for k in (1, 2, 4, 8)]
    assert all(a >= b for a, b in zip(ranks, ranks[1:])) and ranks[-1] < ranks[0], ranks
    assert ranks == [27, 24, 21, 20]
