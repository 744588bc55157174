"""Pins of Algorithms 1 and 2 in the oracle (Sec. III.B): brute-force dense products,
the adjoint identity, sampled rows, the ACA wrappers and the Table II byte counts."""
import os

import numpy as np
import pytest

from oracle import greens, memory, products, tucker
from paper_2103_06393_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))


def _dense_case(n=(6, 7, 8), m=10, tol=1e-12):
    w = inputs.scaled_workload("precision", n, m=m)
    g, s = w.grid, w.segments
    Z = greens.assemble_columns(g.shape, g.h, s.centre, s.tangent, s.length, w.freq_hz, np.arange(s.m))
    tens = tucker.compress_columns(Z, g.shape, 3, tol)
    return g, Z, tens


def test_brute_force_matvec_and_rmatvec():
    g, Z, tens = _dense_case()
    X = inputs.cn01((Z.shape[1], 3), seed=0)
    Phi = inputs.cn01((Z.shape[0], 3), seed=1)
    Y = products.matvec(tens, g.shape, X)
    Psi = products.rmatvec(tens, g.shape, Phi)
    assert np.linalg.norm(Y - Z @ X) <= 1e-11 * np.linalg.norm(Z @ X)
    assert np.linalg.norm(Psi - Z.conj().T @ Phi) <= 1e-11 * np.linalg.norm(Z.conj().T @ Phi)


def test_adjoint_identity_fp64():
    g, Z, tens = _dense_case(tol=1e-4)
    X = inputs.cn01((Z.shape[1], 2), seed=5)
    Phi = inputs.cn01((Z.shape[0], 2), seed=6)
    lhs = np.vdot(Phi, products.matvec(tens, g.shape, X))       # <Z~X, Phi>
    rhs = np.vdot(products.rmatvec(tens, g.shape, Phi), X)      # <X, Z~^H Phi>
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


def test_matvec_rows_matches_full():
    g, Z, tens = _dense_case(tol=1e-6)
    X = inputs.cn01((Z.shape[1], 2), seed=2)
    Y = products.matvec(tens, g.shape, X)
    rows = np.array([0, 5, g.nv + 7, 2 * g.nv + g.nv - 1, 100])
    assert np.allclose(products.matvec_rows(tens, g.shape, X, rows), Y[rows], rtol=1e-13, atol=1e-25)


def test_aca_wrappers():
    rng = np.random.default_rng(4)
    g, Z, tens = _dense_case(tol=1e-12)
    V = rng.normal(size=(5, Z.shape[1])) + 1j * rng.normal(size=(5, Z.shape[1]))  # m x r_c with r_c = 10
    X = inputs.cn01((5, 2), seed=3)
    Y = products.matvec_aca(tens, V, g.shape, X)
    assert np.allclose(Y, Z @ (V.conj().T @ X), rtol=1e-10, atol=0)
    Phi = inputs.cn01((Z.shape[0], 2), seed=4)
    assert np.allclose(products.rmatvec_aca(tens, V, g.shape, Phi), V @ (Z.conj().T @ Phi), rtol=1e-10, atol=0)


def test_table_memory_values():
    """Table IV and Table VIII printed sizes equal the Table II formulas at 16 B per entry."""
    n_rows = 0
    with open(os.path.join(HERE, "golden", "table_memory.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            tab, form, n1, n2, n3, q, m, rc, val = line.split()
            nv = int(n1) * int(n2) * int(n3)
            q, m, rc = int(q), int(m), int(rc)
            if form == "full":
                ent = memory.full_entries(q, nv, m)
            else:
                ent = memory.aca_entries(q, nv, m, rc)
            got = memory.gib(ent)
            dec = len(val.split(".")[1]) if "." in val else 0
            # the tables mostly truncate (6.1858 -> 6.18) but sometimes round (10194.77 -> 10195):
            # accept anything within one unit of the last printed digit
            assert abs(got - float(val)) < 10 ** (-dec), (line, got)
            n_rows += 1
    assert n_rows == 24


def test_tucker_entries_exact():
    assert memory.tucker_entries([(2, 3, 4)], (10, 11, 12)) == 24 + 20 + 33 + 48
    assert memory.tucker_entries_uniform(3, 10, 2, 5) == 3 * (8 + 60) * 5
