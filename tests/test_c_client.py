"""The C ABI from a plain C99 program (tests/abi_example.c, built with gcc -std=c99 -Wall -Wextra
-Werror against include/mhd.h and linked to the library): the header compiles as C, the host-only
entry points answer as the Python binding does, and without a GPU mhd_init returns MHD_ECUDA
(there is no CPU fallback); with one, a context steps."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_c_client(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not found")
    from paper_1810_12707_gb300 import build_lib, mhd
    build_lib.build()
    libdir = os.path.dirname(build_lib.LIB)
    exe = tmp_path / "abi_example"
    subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "abi_example.c"), "-L", libdir, "-l:" + os.path.basename(build_lib.LIB),
                    "-Wl,-rpath," + libdir, "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True, timeout=120).stdout
    got = {line.split()[0]: line.split()[1:] for line in out.splitlines()}
    assert int(got["footprint"][0]) == mhd.mhd_footprint_bytes(64, mhd.MHD_FP64, 2) > 0
    assert int(got["footprint_bad"][0]) == 0
    assert int(got["shells"][0]) == mhd.mhd_num_shells(64)
    assert int(got["init_bad"][0]) == mhd.MHD_EINVAL
    init = int(got["init"][0])
    if init == mhd.MHD_OK:  # a GPU is present: the context stepped
        assert got["set"] == ["0"] and got["step"] == ["0"] and got["sync"] == ["0"]
        assert got["diag"] == ["0", "3"]
    else:
        assert init == mhd.MHD_ECUDA
