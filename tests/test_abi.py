"""The C-ABI library builds, loads and exports every entry point include/*.h declares (no GPU
needed: nothing here launches work)."""
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        names |= set(re.findall(r"MHD_API\s+[\w\s\*]*?\b(mhd_\w+)\s*\(", text))
    return names


def test_header_declares_the_boundary():
    names = declared_symbols()
    for core in ("mhd_init", "mhd_set_state", "mhd_rhs", "mhd_step", "mhd_diagnostics", "mhd_destroy"):
        assert core in names


def test_library_exports_every_declared_symbol():
    from paper_1810_12707_gb300 import build_lib, mhd
    build_lib.build()
    lib = mhd.load_library()
    missing = [n for n in sorted(declared_symbols()) if not hasattr(lib, n)]
    assert missing == []
    assert set(mhd.EXPORTS) == declared_symbols()


def test_footprint_is_pure_host_arithmetic():
    from paper_1810_12707_gb300 import mhd
    assert mhd.mhd_footprint_bytes(48, 0, 1) == 0          # not a power of two
    assert mhd.mhd_footprint_bytes(256, 0, 0) == 0         # no instance
    f256 = mhd.mhd_footprint_bytes(256, 0, 1)
    assert 2e9 < f256 < 3e9
    assert mhd.mhd_footprint_bytes(1024, 0, 1) < 200e9     # the largest grid fits in HBM
