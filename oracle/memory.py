"""Storage model of Table II (Sec. III.A), in bytes.

Full:        q n_v m entries
ACA:         q n_v r_c + m r_c
Tucker:      q (r^3 + 3 n r) m             (uniform ranks, cubic tensors)
ACA+Tucker:  q (r^3 + 3 n r) r_c + m r_c
The exact per-tensor count with uneven ranks is r1 r2 r3 + n1 r1 + n2 r2 + n3 r3.
"""


def full_entries(q, nv, m):
    return q * nv * m


def aca_entries(q, nv, m, rc):
    return q * nv * rc + m * rc


def tucker_entries_uniform(q, n, r, m):
    return q * (r ** 3 + 3 * n * r) * m


def aca_tucker_entries_uniform(q, n, r, m, rc):
    return q * (r ** 3 + 3 * n * r) * rc + m * rc


def tucker_entries(ranks, n):
    """Exact entry count for a list of per-tensor ranks (r1, r2, r3)."""
    n1, n2, n3 = n
    return sum(r1 * r2 * r3 + n1 * r1 + n2 * r2 + n3 * r3 for (r1, r2, r3) in ranks)


def gib(entries, bytes_per_entry=16):
    return entries * bytes_per_entry / 2.0 ** 30
