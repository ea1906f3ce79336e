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
    assert mhd.mhd_footprint_bytes(8, 0, 1) == 0           # below the smallest grid, 16
    assert mhd.mhd_footprint_bytes(2048, 0, 1) == 0        # above the largest, 1024
    assert mhd.mhd_footprint_bytes(256, 0, 0) == 0         # no instance
    assert mhd.mhd_footprint_bytes(256, 3, 1) == 0         # no such precision
    f256 = mhd.mhd_footprint_bytes(256, 0, 1)
    assert 2e9 < f256 < 3e9
    # the double-float mode stores FP64-sized values: FP64's footprint plus its twiddle table
    # and the FP64 copy of one instance's state
    k = (256 - 1) // 3
    spec = (2 * k + 1) ** 2 * (k + 1)
    assert mhd.mhd_footprint_bytes(256, 2, 1) == f256 + 256 * 16 + 7 * spec * 16
    assert mhd.mhd_footprint_bytes(1024, 0, 1) < 200e9     # the largest grid fits in HBM


def test_shell_count_is_pure_host_arithmetic(oracle_mod):
    """Shells s = 0 .. round(sqrt(3) K) hold the modes of the 2/3-truncated cube (K = (N - 1) // 3):
    the corner mode (K, K, K) lies in shell round(sqrt(3) K).  The library's count agrees with the
    oracle's and with that closed form, and is 0 for sizes the library does not take."""
    import math
    from paper_1810_12707_gb300 import mhd
    for n in (16, 32, 64, 128, 256, 512, 1024):
        k = (n - 1) // 3
        assert mhd.mhd_num_shells(n) == int(math.floor(math.sqrt(3) * k + 0.5)) + 1
        assert mhd.mhd_num_shells(n) == oracle_mod._load().or_num_shells(n)
    for n in (0, 8, 48, 2048):
        assert mhd.mhd_num_shells(n) == 0
