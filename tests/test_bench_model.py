"""bench.py's bookkeeping, no GPU: the algorithmic bytes of each kernel of the FP64 step against a
count of what each pass must read and write, those counts against the DRAM reads ncu measured at
256^3, and the rule that a stored traffic figure is dropped once its kernel's sources change."""
import pytest

import bench

N, K = 256, 85
NX, NK = K + 1, 2 * K + 1
SPEC = NK * NK * NX
C = 16  # bytes of an FP64 complex value

# what each pass reads and writes, in complex values (one instance)
COUNTS = {
    "inverse_z": (7 * SPEC, 7 * N * NK * NX),
    "inverse_y": (7 * N * NK * NX, 7 * N * N * NX),
    "flux_x": (7 * N * N * NX, 12 * N * N * NX),
    "forward_y": (12 * N * N * NX, 12 * N * NK * NX),
    "forward_z": (12 * N * NK * NX, 12 * SPEC),
    "assemble_ab2": (26 * SPEC, 14 * SPEC),
    "assemble_iz": (26 * SPEC, 14 * SPEC + 7 * N * NK * NX),
}

# dram__bytes_read.sum of one launch at 256^3 FP64 (ncu --set full; profiles/)
NCU_READ = {"inverse_z": 281.798e6, "inverse_y": 421.688e6, "flux_x": 634.282e6, "forward_y": 1082.209e6,
            "forward_z": 723.134e6, "assemble_ab2": 1046.350e6}


def test_model_bytes_equal_the_pass_counts():
    model = bench.kernel_model(N, 1, "fp64")
    for kernel, (r, w) in COUNTS.items():
        assert model[kernel][0] == pytest.approx((r + w) * C, rel=1e-12), kernel


def test_measured_reads_equal_the_algorithmic_reads():
    """Every pass reads its inputs from HBM once: within 0.1 % for the column passes and the
    assembly, within 1 % for the flux pass (0.5 % measured: about three 32-byte sectors per
    block beyond its inputs)."""
    for kernel, (r, _) in COUNTS.items():
        if kernel not in NCU_READ:
            continue
        assert NCU_READ[kernel] == pytest.approx(r * C, rel=1e-2 if kernel == "flux_x" else 1e-3), kernel


def test_batch_scales_the_model():
    one, eight = bench.kernel_model(64, 1, "fp32"), bench.kernel_model(64, 8, "fp32")
    for kernel in one:
        assert eight[kernel][0] == pytest.approx(8 * one[kernel][0])
        assert eight[kernel][1] == pytest.approx(8 * one[kernel][1])


def test_traffic_is_dropped_when_sources_change(monkeypatch):
    key = ("flux_x", 64, 1, "fp64")
    current = bench.sources_hash("flux_x")
    monkeypatch.setitem(bench.TRAFFIC, key, (123, current, "capture"))
    assert bench.measured_traffic("flux_x", 64, 1, "fp64") == (123, "capture")
    monkeypatch.setitem(bench.TRAFFIC, key, (123, "0" * 16, "capture"))
    nbytes, why = bench.measured_traffic("flux_x", 64, 1, "fp64")
    assert nbytes is None and "changed" in why
    nbytes, why = bench.measured_traffic("flux_x", 48, 1, "fp64")
    assert nbytes is None and "no capture" in why


def test_double_float_model():
    """The double-float mode moves FP64-sized values, so its bytes are the FP64 model's; its
    operation count per transform follows the radix plan: N = 8 one untwiddled radix-8 DFT (432
    FP32 operations), N = 16 two of them and eight twiddled radix-2 butterflies (64 each), N = 32
    four and eight twiddled radix-4 butterflies (224 each), N = 64 eight untwiddled and eight
    twiddled radix-8 DFTs (656 each)."""
    assert bench.dfloat_fft_ops(8) == 432
    assert bench.dfloat_fft_ops(16) == 2 * 432 + 8 * 64
    assert bench.dfloat_fft_ops(32) == 4 * 432 + 8 * 224
    assert bench.dfloat_fft_ops(64) == 8 * 432 + 8 * 656
    assert bench.dfloat_fft_ops(512) == 64 * 432 + 2 * 64 * 656
    fp64, df = bench.kernel_model(N, 1, "fp64"), bench.kernel_model(N, 1, "fp64df")
    for kernel in fp64:
        assert df[kernel][0] == fp64[kernel][0]
    ops = bench.dfloat_ops(N)
    assert df["inverse_y"][1] == ops["inverse_y"] == 7 * N * NX * (bench.dfloat_fft_ops(N) + 6 * N)
