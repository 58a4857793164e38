"""The C ABI library loads (no GPU needed) and exports every function include/wroute.h declares."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "wroute.h")


def declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(wr_[a-z_]+)\s*\(", text)
    return sorted(set(n for n in names if n not in ("wr_consume_fn",)))


@pytest.fixture(scope="module")
def lib():
    from paper_2504_20655_gb300 import build, wroute
    build.build()
    return wroute.load_library()


def test_header_lists_the_entry_points():
    names = declared()
    for n in ("wr_create", "wr_load_graph", "wr_route_orders", "wr_distance_rows", "wr_bf_rows", "wr_tour_eval",
              "wr_sync", "wr_strerror", "wr_destroy"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2504_20655_gb300 import wroute
    out = subprocess.run(["nm", "-D", "--defined-only", wroute.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (wr_[a-z_]+)\b", out))
    missing = [n for n in declared() if n not in exported]
    assert not missing, missing
    for n in declared():
        assert hasattr(lib, n)
    assert set(wroute.EXPORTS) == set(declared())


def test_strerror_is_host_only(lib):
    from paper_2504_20655_gb300 import wroute
    assert wroute.strerror(0) == "ok"
    assert "timed out" in wroute.strerror(wroute.WR_ETIMEOUT)


def test_no_fallback_when_library_missing(tmp_path):
    from paper_2504_20655_gb300 import wroute
    saved = wroute._lib
    try:
        wroute._lib = None
        with pytest.raises(ImportError):
            wroute.load_library(str(tmp_path / "missing.so"))
    finally:
        wroute._lib = saved


def test_product_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2504_20655_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cpp", ".h", ".cuh")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "oracle.h" not in text, f
