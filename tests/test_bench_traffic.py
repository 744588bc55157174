"""The bench's recorded DRAM traffic (profiles/traffic.txt): well-formed records, each used only
while the kernel's source file still hashes to the recorded prefix."""
import os

import bench


def _records():
    path = os.path.join(bench.ROOT, "profiles", "traffic.txt")
    out = []
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        out.append(line.split())
    return out


def test_records_are_well_formed():
    recs = _records()
    assert recs
    for f in recs:
        assert len(f) == 4, f
        kernel, workload, sha, nbytes = f
        assert kernel in bench.KERNEL_SOURCES, kernel
        assert workload in ("large", "precision", "batching", "learned"), workload
        assert len(sha) == 16 and all(c in "0123456789abcdef" for c in sha), sha
        assert float(nbytes) > 0


def test_record_used_only_while_the_source_matches():
    for kernel, workload, sha, nbytes in _records():
        got = bench.recorded_traffic(kernel, workload)
        if bench.source_sha16(kernel) == sha:
            assert got == float(nbytes)
        else:
            assert got is None
    assert bench.recorded_traffic("matvec_dc_kernel", "no-such-workload") is None
    assert bench.recorded_traffic("no_such_kernel", "large") is None
