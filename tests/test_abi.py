"""The C-ABI library builds for sm_103a, loads, and exports every symbol its headers declare
(no compute call: this runs without a GPU)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^(?:const\s+)?[A-Za-z_][\w]*\s*\**\s+\**\s*([A-Za-z_]\w*)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_headers_declare_the_boundary():
    names = declared_functions()
    for required in ("vsie_assemble_columns", "tucker_compress", "aca_compress", "zbc_matvec", "zbc_rmatvec",
                     "zbc_free", "zbc_save", "zbc_load", "zbc_memory_bytes"):
        assert required in names, required


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2103_06393_gb300 import build
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_2103_06393_gb300 import zbc
    monkeypatch.setattr(zbc, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(zbc, "_lib", None)
    with pytest.raises(ImportError):
        zbc.lib()


def test_binding_enums_match_the_header():
    # the Python binding's integer constants are the header's enum values (zbc_precision and the
    # status codes), and zbc_tune's variant list has the length the header documents
    from paper_2103_06393_gb300 import zbc
    text = open(os.path.join(ROOT, "include", "zbc.h")).read()
    values = {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(ZBC_[A-Z0-9_]+)\s*=\s*(-?\d+)", text)}
    for name in ("FP32_SIMT", "TF32X3", "BF16X3", "AUTO", "TC2", "TC_MODE1", "TC_DC"):
        assert getattr(zbc, name) == values["ZBC_" + name], name
    for name in ("ZBC_OK", "ZBC_EINVAL"):
        assert getattr(zbc, name) == values[name], name
    m = re.search(r"times_ms_host : optional float\[(\d+)\]", text)
    assert m and int(m.group(1)) == len(zbc.TUNE_VARIANTS)
